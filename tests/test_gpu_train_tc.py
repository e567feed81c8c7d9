"""GPU parity of the tensor-core training path (SDF_BF16 and SDF_FP16 operands, FP32
accumulation): the forward with saved pre-activations against the FP64 oracle, the
backward against the FP32 path and against FP64 central differences of the oracle's
objective on 1024 parameters, chunking, the autograd wrapper and a short fit.

Tolerances, in units of the operand type's unit roundoff u (2^-9 bfloat16, 2^-12
half).  Each hidden-layer contraction rounds both operands to 16 bits and
accumulates in FP32, so a value or a tangent carries a relative error of a few u;
f: 4 u of its scale.  The parameter gradient from fixed adjoints sums such terms
over thousands of points: 8 u of each parameter block's RMS.  Against finite
differences of the FP64 objective (the adjoints then differ too, through f and
grad f): 32 u of the RMS.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_09147_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

LAM_N, LAM_E = 0.1, 0.05
UNIT = {1: 2.0 ** -9, 3: 2.0 ** -12}  # SDF_BF16, SDF_FP16 unit roundoff
PRECISIONS = [1, 3]
IDS = ["bf16", "fp16"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


NETS = [("siren64x1", lambda: inputs.net_to_bytes(inputs.siren_init(11, 64, 1))),
        ("scene64x2", lambda: (workloads.SCENES / "s8_64x2.sdfn").read_bytes()),
        ("scene128x2", lambda: (workloads.SCENES / "s8_128x2.sdfn").read_bytes()),
        ("scene256x3", lambda: (workloads.SCENES / "s8_256x3.sdfn").read_bytes())]


@pytest.mark.parametrize("precision", PRECISIONS, ids=IDS)
@pytest.mark.parametrize("name,make", NETS, ids=[n for n, _ in NETS])
def test_tc_forward_matches_oracle(sdf, precision, name, make):
    """f and grad f of the tensor-core training forward (3001 points: several tiles and a
    ragged tail) against FP64.  f to 4 u of the scale of f.  grad f: the training forward makes
    the roundings of the 16-bit normal-mapping kernel up to the last hidden layer and then runs
    the output layer in FP32, so its error may not exceed that kernel's on the same points
    (p99.9, relative; that kernel is held to the stated normal bounds in the parity tests).
    Points uniform in the cube, where the networks are not Eikonal and grad f is a sum with
    cancellation that amplifies every rounding."""
    b = make()
    shape, theta = sdf.theta_from_sdfn(b)
    pts = inputs.random_points(21, 3001)
    f, g, _ = sdf.train_forward(shape, _dev(theta), _dev(pts), precision=precision)
    g_inf = sdf.normals(sdf.Net(b, precision), _dev(pts))
    sdf.sync_status()
    ref_g, ref_f = oracle.Net(b).grad_batch(pts.astype(np.float64), with_value=True)
    u = UNIT[precision]
    fe = np.abs(f.cpu().numpy() - ref_f)
    gn = np.linalg.norm(ref_g, axis=0)
    den = np.maximum(gn, 1e-3 * np.median(gn))
    ge = np.quantile(np.linalg.norm(g.cpu().numpy() - ref_g, axis=0) / den, 0.999)
    ge_inf = np.quantile(np.linalg.norm(g_inf.cpu().numpy() - ref_g, axis=0) / den, 0.999)
    print(name, precision, "f err max", fe.max(), "f scale", np.abs(ref_f).max(), "grad rel p99.9", ge,
          "normal-mapping kernel", ge_inf)
    assert fe.max() <= 4 * u * max(1.0, np.abs(ref_f).max())
    assert ge <= max(1.25 * ge_inf, 2 * u)


def _grad(sdf, b, pts, tf, tg, near, precision):
    shape, theta = sdf.theta_from_sdfn(b)
    th = _dev(theta)
    f, g, ws = sdf.train_forward(shape, th, _dev(pts), precision=precision)
    d_f, d_g, loss = sdf.fit_loss(f, g, _dev(tf), _dev(tg), _dev(near), LAM_N, LAM_E)
    d_theta = sdf.train_backward(shape, th, _dev(pts), d_f, d_g, ws, precision=precision)
    sdf.sync_status()
    return d_theta.cpu().numpy().astype(np.float64), loss.cpu().numpy()


@pytest.mark.parametrize("precision", PRECISIONS, ids=IDS)
@pytest.mark.parametrize("name", ["s8_64x2", "s8_128x2", "s8_256x2", "s8_256x3"])
def test_tc_backward_matches_fp32_backward(sdf, precision, name):
    """The backward's arithmetic: dL/dtheta from the same seeded adjoints (dL/df, dL/d grad f:
    normal draws / n; the backward is linear in them) through the 16-bit tensor-core path and
    through the FP32 path (itself checked against FP64 finite differences), 4096 points, per
    parameter block relative to the block's RMS.  Random adjoints keep the sums free of the
    cancellation a fitted network's gradient has near its optimum, which would amplify any
    rounding.  The objective of the same points is compared too (its value, not its kinks)."""
    b = (workloads.SCENES / f"{name}.sdfn").read_bytes()
    n = 4096
    pts, tf, tg, near = inputs.fit_batch(inputs.sphere_scene(1), 5, n)
    u1, u2 = inputs.uniform01(6, 4 * n), inputs.uniform01(7, 4 * n)
    z = (np.sqrt(-2.0 * np.log(np.maximum(u1, 1e-300))) * np.cos(2.0 * np.pi * u2) / n).astype(np.float32)
    d_f, d_g = _dev(z[:n]), _dev(z[n:].reshape(3, n))
    shape, theta = sdf.theta_from_sdfn(b)
    th, dp = _dev(theta), _dev(pts)
    out = {}
    for prec in (sdf.SDF_FP32, precision):
        f, g, ws = sdf.train_forward(shape, th, dp, precision=prec)
        _, _, loss = sdf.fit_loss(f, g, _dev(tf), _dev(tg), _dev(near), LAM_N, LAM_E)
        out[prec] = (sdf.train_backward(shape, th, dp, d_f, d_g, ws, precision=prec).cpu().numpy().astype(np.float64),
                     loss.cpu().numpy())
        del ws
    sdf.sync_status()
    (g32, l32), (g16, l16) = out[sdf.SDF_FP32], out[precision]
    u = UNIT[precision]
    print(name, precision, "loss fp32", l32, "16-bit", l16)
    assert abs(l16[3] - l32[3]) <= 8 * u * abs(l32[3])
    in_dim, w, k = shape
    blocks = [("W0", 0, w * in_dim), ("b0", w * in_dim, w * in_dim + w)]
    o = w * in_dim + w
    for li in range(k):
        blocks += [(f"W{li + 1}", o, o + w * w), (f"b{li + 1}", o + w * w, o + w * w + w)]
        o += w * w + w
    blocks += [("wout", o, o + w), ("bout", o + w, o + w + 1)]
    for label, lo, hi in blocks:
        ref, got = g32[lo:hi], g16[lo:hi]
        rms = np.sqrt(np.mean(ref ** 2))
        err = np.sqrt(np.mean((got - ref) ** 2)) / max(rms, 1e-30)
        print(f"  {label}: rms {rms:.3e} rel rms err {err:.3e}")
        assert err <= 8 * u


@pytest.mark.parametrize("precision", PRECISIONS, ids=IDS)
def test_tc_backward_matches_fp64_finite_differences(sdf, precision):
    """Config 5's check: dL/dtheta on 1024 sampled parameters of a fitted (64,2) against central
    differences of the FP64 oracle objective (steps of 2^-12 on the float32 parameters)."""
    b = (workloads.SCENES / "s8_64x2.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    pts, tf, tg, near = inputs.fit_batch(inputs.sphere_scene(1), 3, 512)
    rg, rf = oracle.Net(sdf.sdfn_from_theta(shape, theta)).grad_batch(pts.astype(np.float64), with_value=True)
    keep = (np.abs(rf - tf) > 1e-2) & (np.abs(np.linalg.norm(rg, axis=0) - 1.0) > 5e-2)
    pts, tf, tg, near = pts[:, keep].copy(), tf[keep].copy(), tg[:, keep].copy(), near[keep].copy()
    gpu, _ = _grad(sdf, b, pts, tf, tg, near, precision)
    idx = np.unique((inputs.uniform01(77, 1400) * theta.size).astype(np.int64))[:1024]
    assert idx.size == 1024
    h = np.float32(2.0 ** -12)
    fd = np.empty(idx.size)
    for q, j in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        lp, _ = oracle.fit_loss(sdf.sdfn_from_theta(shape, tp), pts, tf, tg, near, LAM_N, LAM_E)
        lm, _ = oracle.fit_loss(sdf.sdfn_from_theta(shape, tm), pts, tf, tg, near, LAM_N, LAM_E)
        fd[q] = (lp - lm) / (float(tp[j]) - float(tm[j]))
    err = np.abs(gpu[idx] - fd)
    scale = np.sqrt(np.mean(fd ** 2))
    u = UNIT[precision]
    rel = np.sqrt(np.mean(err ** 2)) / scale
    print(precision, "rms fd", scale, "rel rms err", rel, "max err / rms", err.max() / scale)
    assert rel <= 32 * u
    assert np.all(err <= 0.25 * np.abs(fd) + 64 * u * scale)


@pytest.mark.parametrize("precision", PRECISIONS, ids=IDS)
def test_tc_chunks_accumulate_to_the_whole_batch(sdf, precision):
    """Points are independent: two chunks (ragged, not multiples of a tile) add up to the whole
    batch, with the FP32 accumulation order as the only difference; per-point time (4-D)."""
    b = (workloads.SCENES / "a8_64x1_t.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    th = _dev(theta)
    pts = _dev(inputs.random_points(23, 1000))
    times = _dev((inputs.uniform01(24, 1000)).astype(np.float32))
    f, g, ws = sdf.train_forward(shape, th, pts, pt_time=times, precision=precision)
    d_f = (2.0 * f).contiguous()
    c = torch.linspace(-1.0, 1.0, 3, device="cuda")[:, None]
    d_g = c.expand_as(g).contiguous()
    whole = sdf.train_backward(shape, th, pts, d_f, d_g, ws, pt_time=times, precision=precision)
    acc = torch.zeros_like(whole)
    for lo, hi in ((0, 613), (613, 1000)):
        p = pts[:, lo:hi].contiguous()
        t = times[lo:hi].contiguous()
        _, _, w = sdf.train_forward(shape, th, p, pt_time=t, precision=precision)
        sdf.train_backward(shape, th, p, d_f[lo:hi].contiguous(), d_g[:, lo:hi].contiguous(), w, acc, pt_time=t,
                           precision=precision)
    sdf.sync_status()
    rel = ((acc - whole).norm() / whole.norm()).item()
    print("chunks vs whole", rel)
    assert rel <= 1e-5
    # the 4-D forward against the oracle at each point's time
    onet = oracle.Net(b)
    ph, th_ = pts.cpu().numpy().astype(np.float64), times.cpu().numpy().astype(np.float64)
    ref = np.array([onet.eval([*ph[:, i], th_[i]]) for i in range(0, 1000, 97)])
    assert np.abs(f.cpu().numpy()[::97] - ref).max() <= 4 * UNIT[precision] * max(1.0, np.abs(ref).max())


def test_tc_autograd_function(sdf):
    """SineMLP with precision SDF_BF16 inside a torch graph gives the library's backward."""
    b = (workloads.SCENES / "s8_128x2.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    pts = _dev(inputs.random_points(25, 777))
    th = _dev(theta).requires_grad_(True)
    f, g = sdf.SineMLP.apply(th, pts, shape, None, sdf.SDF_BF16)
    c = torch.linspace(-1.0, 1.0, 3, device="cuda")[:, None]
    (f.square().sum() + (g * c).sum()).backward()
    f2, g2, ws = sdf.train_forward(shape, th.detach(), pts, precision=sdf.SDF_BF16)
    ref = sdf.train_backward(shape, th.detach(), pts, (2.0 * f2).contiguous(), c.expand_as(g2).contiguous(), ws,
                             precision=sdf.SDF_BF16)
    sdf.sync_status()
    assert torch.allclose(th.grad, ref, rtol=1e-5, atol=1e-5 * ref.abs().max().item())


def test_tc_native_fit_descends_like_fp32(sdf):
    """200 native steps from one SIREN (64,2) initialisation on the same batches: the BF16
    tensor-core path and the FP32 path reach objectives within 5 % of each other, both well
    below the start."""
    shape, theta0 = sdf.theta_from_sdfn(inputs.net_to_bytes(inputs.siren_init(0, 64, 2)))
    ends = {}
    for prec in (sdf.SDF_FP32, sdf.SDF_BF16):
        th = _dev(theta0)
        m, v = torch.zeros_like(th), torch.zeros_like(th)
        ws, first = None, None
        for it in range(200):
            pts, tf, tg, near = (_dev(x) for x in inputs.fit_batch(inputs.sphere_scene(1), 1000 + it, 1 << 12))
            loss, ws = sdf.fit_step(shape, th, m, v, it + 1, pts, tf, tg, near, lr=1e-4, workspace=ws,
                                    precision=prec)
            if first is None:
                first = loss[3].item()
        sdf.sync_status()
        ends[prec] = (first, loss[3].item())
    print(ends)
    (f32a, f32b), (bfa, bfb) = ends[sdf.SDF_FP32], ends[sdf.SDF_BF16]
    assert abs(f32a - bfa) <= 0.05 * f32a
    assert f32b < 0.7 * f32a and bfb < 0.7 * bfa
    assert abs(bfb - f32b) <= 0.05 * f32b
