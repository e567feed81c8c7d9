"""GPU parity of the training path (FP32): forward with tangents, the fitting
objective, the backward pass against FP64 finite differences of the oracle's
objective, the autograd wrapper, Adam, and a short native fit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_09147_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu

LAM_N, LAM_E = 0.1, 0.05


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("make", [lambda: inputs.siren_init(11, 64, 1), lambda: inputs.siren_init(12, 128, 2),
                                  lambda: inputs.siren_init(13, 256, 3),
                                  lambda: (workloads.SCENES / "s8_256x3.sdfn").read_bytes()],
                         ids=["siren64x1", "siren128x2", "siren256x3", "scene256x3"])
def test_train_forward_matches_oracle(sdf, make):
    net = make()
    b = net if isinstance(net, bytes) else inputs.net_to_bytes(net)
    shape, theta = sdf.theta_from_sdfn(b)
    pts = inputs.random_points(21, 3001)
    f, g, _ = sdf.train_forward(shape, _dev(theta), _dev(pts))
    torch.cuda.synchronize()
    ref_g, ref_f = oracle.Net(b).grad_batch(pts.astype(np.float64), with_value=True)
    fe = np.abs(f.cpu().numpy() - ref_f)
    ge = np.linalg.norm(g.cpu().numpy() - ref_g, axis=0) / np.maximum(np.linalg.norm(ref_g, axis=0), 1e-3)
    print(shape, "f err max", fe.max(), "grad rel p99.9", np.quantile(ge, 0.999))
    assert fe.max() <= 2e-4 * max(1.0, np.abs(ref_f).max())
    assert np.quantile(ge, 0.999) <= 2e-4


def test_train_forward_4d_per_point_time(sdf):
    b = (workloads.SCENES / "a8_64x1_t.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    pts = inputs.random_points(22, 2000)
    times = np.repeat(np.array([0.1, 0.6], np.float32), 1000)
    f, g, _ = sdf.train_forward(shape, _dev(theta), _dev(pts), pt_time=_dev(times))
    f, g = f.cpu().numpy(), g.cpu().numpy()
    on = oracle.Net(b)
    for lo, t in ((0, 0.1), (1000, 0.6)):
        rg, rf = on.grad_batch(pts[:, lo:lo + 1000].astype(np.float64), time=float(np.float32(t)), with_value=True)
        assert np.abs(f[lo:lo + 1000] - rf).max() <= 2e-4
        assert np.abs(g[:, lo:lo + 1000] - rg).max() <= 2e-4 * max(1.0, np.abs(rg).max())


def _loss_inputs(n, seed=0):
    sc = inputs.sphere_scene(1)
    return inputs.fit_batch(sc, seed, n)


def test_fit_loss_matches_oracle_and_its_derivative(sdf):
    b = (workloads.SCENES / "s8_64x2.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    pts, tf, tg, near = _loss_inputs(4096)
    f, g, _ = sdf.train_forward(shape, _dev(theta), _dev(pts))
    d_f, d_g, loss = sdf.fit_loss(f, g, _dev(tf), _dev(tg), _dev(near), LAM_N, LAM_E)
    torch.cuda.synchronize()
    L, parts = oracle.fit_loss(b, pts, tf, tg, near, LAM_N, LAM_E)
    got = loss.cpu().numpy()
    print(got, L, parts)
    assert np.allclose(got[:3], parts, rtol=1e-4, atol=1e-6) and abs(got[3] - L) <= 1e-4 * abs(L)
    # the adjoints are the derivatives of the objective in (f, grad f) (FP64, from the definition)
    fv, gv = f.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    n = fv.size
    nn = near.astype(bool)
    exp_df = np.sign(fv - tf) / n
    na = np.linalg.norm(gv, axis=0)
    nb = np.linalg.norm(tg.astype(np.float64), axis=0)
    cos = np.sum(gv * tg, axis=0) / (na * nb)
    exp_dg = LAM_E / n * np.sign(na - 1.0) * gv / na
    exp_dg[:, nn] -= LAM_N / nn.sum() * (tg[:, nn] / (na * nb)[nn] - cos[nn] * gv[:, nn] / na[nn] ** 2)
    assert np.allclose(d_f.cpu().numpy(), exp_df, rtol=1e-6, atol=1e-12)
    assert np.allclose(d_g.cpu().numpy(), exp_dg, rtol=1e-4, atol=1e-9)


def test_backward_matches_fp64_finite_differences(sdf):
    """dL/dtheta of the objective on 1024 parameters against central differences of
    the FP64 oracle objective (exact steps of 2^-12 on the float32 parameters)."""
    b = (workloads.SCENES / "s8_64x2.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    pts, tf, tg, near = _loss_inputs(512, seed=3)
    # keep points away from the kinks of |.| so that the objective is smooth around theta
    rg, rf = oracle.Net(sdf.sdfn_from_theta(shape, theta)).grad_batch(pts.astype(np.float64), with_value=True)
    keep = (np.abs(rf - tf) > 1e-2) & (np.abs(np.linalg.norm(rg, axis=0) - 1.0) > 5e-2)
    pts, tf, tg, near = pts[:, keep].copy(), tf[keep].copy(), tg[:, keep].copy(), near[keep].copy()
    th = _dev(theta)
    f, g, ws = sdf.train_forward(shape, th, _dev(pts))
    d_f, d_g, _ = sdf.fit_loss(f, g, _dev(tf), _dev(tg), _dev(near), LAM_N, LAM_E)
    d_theta = sdf.train_backward(shape, th, _dev(pts), d_f, d_g, ws)
    sdf.sync_status()
    gpu = d_theta.cpu().numpy().astype(np.float64)
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
    print("rms fd", scale, "max err", err.max(), "p99 rel", np.quantile(err / (np.abs(fd) + 1e-2 * scale), 0.99))
    assert np.all(err <= 2e-3 * np.abs(fd) + 2e-3 * scale)


def test_autograd_function_and_chunks(sdf):
    """SineMLP in a torch graph gives the library's backward; two chunks of the points
    accumulate to the whole batch."""
    b = (workloads.SCENES / "s8_128x2.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    pts = _dev(inputs.random_points(23, 1000))
    th = _dev(theta).requires_grad_(True)
    f, g = sdf.SineMLP.apply(th, pts, shape)
    c = torch.linspace(-1.0, 1.0, 3, device="cuda")[:, None]
    (f.square().sum() + (g * c).sum()).backward()
    f2, g2, ws = sdf.train_forward(shape, th.detach(), pts)
    d_f = (2.0 * f2).contiguous()
    d_g = c.expand_as(g2).contiguous()
    ref = sdf.train_backward(shape, th.detach(), pts, d_f, d_g, ws)
    assert torch.allclose(th.grad, ref, rtol=1e-5, atol=1e-5)
    acc = torch.zeros_like(ref)
    for lo, hi in ((0, 600), (600, 1000)):
        p = pts[:, lo:hi].contiguous()
        _, _, w = sdf.train_forward(shape, th.detach(), p)
        sdf.train_backward(shape, th.detach(), p, d_f[lo:hi].contiguous(), d_g[:, lo:hi].contiguous(), w, acc)
    torch.cuda.synchronize()
    assert torch.allclose(acc, ref, rtol=1e-4, atol=1e-4 * ref.abs().max().item())


def test_adam_matches_oracle(sdf):
    rng = np.random.default_rng(6)
    theta = rng.normal(size=5000).astype(np.float32)
    th, m, v = _dev(theta), torch.zeros(5000, device="cuda"), torch.zeros(5000, device="cuda")
    rt, rm, rv = theta.astype(np.float64), np.zeros(5000), np.zeros(5000)
    for k in range(1, 4):
        gk = rng.normal(size=5000).astype(np.float32)
        sdf.adam_step(th, _dev(gk), m, v, k, 1e-3)
        rt, rm, rv = oracle.adam_step(rt, gk, rm, rv, k, 1e-3)
    torch.cuda.synchronize()
    assert np.allclose(th.cpu().numpy(), rt, rtol=0, atol=2e-6)


def _torch_objective(theta, pts, shape, tf, tg, near):
    """The same network and objective written with torch autograd (FP32 reference)."""
    in_dim, W, k = shape
    o = 0
    x = pts.T.clone().requires_grad_(True)
    w0 = theta[o:o + W * in_dim].view(W, in_dim)
    o += W * in_dim
    b0 = theta[o:o + W]
    o += W
    h = torch.sin(x @ w0.T + b0)
    for _ in range(k):
        wl = theta[o:o + W * W].view(W, W)
        o += W * W
        bl = theta[o:o + W]
        o += W
        h = torch.sin(h @ wl.T + bl)
    f = h @ theta[o:o + W] + theta[o + W]
    (g,) = torch.autograd.grad(f.sum(), x, create_graph=True)
    nrm = g.norm(dim=1)
    nb = tg.T.norm(dim=1)
    cos = (g * tg.T).sum(dim=1) / (nrm * nb)
    nf = near.bool()
    return ((f - tf).abs().mean() + LAM_N * (1.0 - cos[nf]).mean() + LAM_E * (nrm - 1.0).abs().mean())


def test_native_fit_matches_torch_reference(sdf):
    """Native steps (forward, objective, backward, Adam) against the same objective and
    torch.optim.Adam through torch autograd, from one SIREN (64,1) initialisation."""
    shape, theta = sdf.theta_from_sdfn(inputs.net_to_bytes(inputs.siren_init(0, 64, 1)))
    th = _dev(theta)
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    pts, tf, tg, near = (_dev(x) for x in _loss_inputs(1 << 13, seed=9))
    ref = _dev(theta).requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=1e-4)
    # the first gradient itself
    f, g, ws = sdf.train_forward(shape, th, pts)
    d_f, d_g, _ = sdf.fit_loss(f, g, tf, tg, near, LAM_N, LAM_E)
    d0 = sdf.train_backward(shape, th, pts, d_f, d_g, ws)
    _torch_objective(ref, pts, shape, tf, tg, near).backward()
    rel = (d0 - ref.grad).norm() / ref.grad.norm()
    print("first gradient rel diff", rel.item())
    assert rel.item() <= 1e-4
    opt.zero_grad()
    objs = []
    for step in range(1, 101):
        loss, ws = sdf.fit_step(shape, th, m, v, step, pts, tf, tg, near, lr=1e-4, workspace=ws)
        opt.zero_grad()
        lt = _torch_objective(ref, pts, shape, tf, tg, near)
        lt.backward()
        opt.step()
        objs.append((loss[3].item(), lt.item()))
    sdf.sync_status()
    objs = np.array(objs)
    print("objective native / torch", objs[0], objs[-1])
    assert np.all(np.abs(objs[:, 0] - objs[:, 1]) <= 2e-3 * objs[:, 1])
    assert objs[-1, 0] < 0.8 * objs[0, 0]
    assert (th - ref.detach()).abs().max().item() <= 1e-3 * ref.detach().abs().max().item()


def test_full_batch_objective_and_chunking(sdf):
    """2^20 points (the benchmark's batch) of a (64,2): the objective matches the FP64 oracle,
    and the gradient of the whole batch equals the sum over four chunks."""
    b = (workloads.SCENES / "s8_64x2.sdfn").read_bytes()
    shape, theta = sdf.theta_from_sdfn(b)
    n = 1 << 20
    pts, tf, tg, near = _loss_inputs(n, seed=11)
    th = _dev(theta)
    dp, dtf, dtg, dnear = _dev(pts), _dev(tf), _dev(tg), _dev(near)
    f, g, ws = sdf.train_forward(shape, th, dp)
    d_f, d_g, loss = sdf.fit_loss(f, g, dtf, dtg, dnear, LAM_N, LAM_E)
    whole = sdf.train_backward(shape, th, dp, d_f, d_g, ws)
    torch.cuda.synchronize()
    L, parts = oracle.fit_loss(b, pts, tf, tg, near, LAM_N, LAM_E)
    got = loss.cpu().numpy()
    print(got, L)
    assert np.allclose(got[:3], parts, rtol=2e-4) and abs(got[3] - L) <= 2e-4 * abs(L)
    del ws
    acc = torch.zeros_like(whole)
    q = n // 4
    for c in range(4):
        sl = slice(c * q, (c + 1) * q)
        p = dp[:, sl].contiguous()
        _, _, w = sdf.train_forward(shape, th, p)
        sdf.train_backward(shape, th, p, d_f[sl].contiguous(), d_g[:, sl].contiguous(), w, acc)
        del w
    sdf.sync_status()
    rel = (acc - whole).norm() / whole.norm()
    print("chunked vs whole rel", rel.item())
    assert rel.item() <= 1e-4


def test_native_fitter_produces_a_loadable_network(sdf, tmp_path):
    """fit.py --native path: a few steps give an SDFN network the renderer and the oracle load."""
    from paper_2201_09147_gb300 import fit
    net = fit.fit_net_native(inputs.sphere_scene(1), 64, 1, 30, batch=1 << 12, log_every=0)
    b = inputs.net_to_bytes(net)
    assert oracle.Net(b).width == 64
    n = sdf.Net(b, sdf.SDF_BF16)
    assert n.lipschitz > 0
