"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check uses a closed form,
an independent library routine (LAPACK SVD, torch autograd, numpy roots),
brute force, or a property the paper states (Props. 1-2, the Lipschitz step).
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2201_09147_gb300 import inputs

GOLDEN = Path(__file__).resolve().parent / "golden"


def folded_arrays(net: inputs.SineNet):
    Ws, bs = [], []
    for i, (w, b) in enumerate(zip(net.weights[:-1], net.biases[:-1])):
        s = 1.0 if net.folded else (net.omega0 if i == 0 else net.omega)
        Ws.append(s * w.astype(np.float64))
        bs.append(s * b.astype(np.float64))
    return Ws, bs, net.weights[-1][0].astype(np.float64), float(net.biases[-1][0])


# ---------------------------------------------------------------------------
# P1: the (w, k) reading reproduces the paper's memory column
# ---------------------------------------------------------------------------

def test_param_counts_match_paper_memory_column():
    rows = json.loads((GOLDEN / "mem_column.json").read_text())["rows"]
    for row in rows:
        kib = sum(inputs.param_count(3, w, k) for w, k in row["nets"]) * 4 / 1024
        assert abs(kib - row["mem_kb"]) <= row["tol_kb"], (row, kib)


def test_netfile_roundtrip_and_size():
    net = inputs.siren_init(0, 64, 1)
    b = inputs.net_to_bytes(net)
    assert len(b) == 32 + 4 * 4481
    back = inputs.net_from_bytes(b)
    for w0, w1 in zip(net.weights, back.weights):
        assert np.array_equal(w0.astype(np.float32), w1)


# ---------------------------------------------------------------------------
# P2: network value and gradient in closed form
# ---------------------------------------------------------------------------

def single_sine_layer_net(seed, width):
    """f(p) = sum_k c_k sin(w_k . p + b_k) + b: a (width, 0) network, omega = 1."""
    return inputs.random_plain_net(seed, width, 0, scale=1.5)


def test_single_layer_value_and_gradient_closed_form():
    net = single_sine_layer_net(21, 16)
    on = oracle.Net(inputs.net_to_bytes(net))
    W = net.weights[0].astype(np.float64)
    b = net.biases[0].astype(np.float64)
    c = net.weights[1][0].astype(np.float64)
    b_out = float(net.biases[1][0])
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = rng.uniform(-1, 1, 3)
        a = W @ p + b
        assert abs(on.eval(p) - (c @ np.sin(a) + b_out)) <= 1e-13
        g_ref = (c * np.cos(a)) @ W
        assert np.max(np.abs(on.grad(p) - g_ref)) <= 1e-13


def test_zero_hidden_weights_reduce_to_bias_chain():
    net = inputs.random_plain_net(22, 8, 2, scale=0.9)
    for i in (1, 2):
        net.weights[i][:] = 0.0
    on = oracle.Net(inputs.net_to_bytes(net))
    b2, b1 = net.biases[2].astype(np.float64), net.biases[1].astype(np.float64)
    expect = net.weights[3][0].astype(np.float64) @ np.sin(b2) + float(net.biases[3][0])
    for p in ([0.1, -0.2, 0.3], [0.9, 0.9, -0.9]):
        assert abs(on.eval(np.array(p)) - expect) <= 1e-14
        assert np.all(on.grad(np.array(p)) == 0.0)
    del b1


def test_frequency_folding_matches_unfolded_definition():
    """Layer 0 scaled by omega0, hidden layers by omega, output linear (SIREN, Sec. 2)."""
    net = inputs.siren_init(4, 64, 2, omega0=30.0, omega=20.0)
    on = oracle.Net(inputs.net_to_bytes(net))
    W = [w.astype(np.float64) for w in net.weights]
    b = [x.astype(np.float64) for x in net.biases]
    p = np.array([0.2, -0.4, 0.1])
    x = np.sin(30.0 * (W[0] @ p + b[0]))
    x = np.sin(20.0 * (W[1] @ x + b[1]))
    x = np.sin(20.0 * (W[2] @ x + b[2]))
    f = W[3][0] @ x + b[3][0]
    assert abs(on.eval(p) - f) <= 1e-12


# ---------------------------------------------------------------------------
# P3: the analytic gradient (Alg. 2) against independent differentiation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(64, 1), (64, 3), (128, 2)])
def test_gradient_matches_torch_autograd(shape):
    torch = pytest.importorskip("torch")
    net = inputs.siren_init(8, *shape)
    on = oracle.Net(inputs.net_to_bytes(net))
    Ws, bs, wo, bo = folded_arrays(net)
    Wt = [torch.tensor(w) for w in Ws]
    bt = [torch.tensor(x) for x in bs]
    rng = np.random.default_rng(1)
    for _ in range(10):
        p = rng.uniform(-1, 1, 3)
        x = torch.tensor(p, requires_grad=True)
        h = x
        for w, b in zip(Wt, bt):
            h = torch.sin(w @ h + b)
        f = torch.tensor(wo) @ h + bo
        (g,) = torch.autograd.grad(f, x)
        ref = g.numpy()
        assert abs(on.eval(p) - f.item()) <= 1e-12 * max(1.0, abs(f.item()))
        assert np.max(np.abs(on.grad(p) - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(64, 1), (256, 3)])
def test_gradient_matches_central_differences(shape):
    net = inputs.siren_init(9, *shape)
    on = oracle.Net(inputs.net_to_bytes(net))
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(4):
        p = rng.uniform(-1, 1, 3)
        g = on.grad(p)
        fd = np.array([(on.eval(p + h * e) - on.eval(p - h * e)) / (2 * h) for e in np.eye(3)])
        assert np.linalg.norm(g - fd) <= 1e-5 * np.linalg.norm(g)


def test_gradient_batch_equals_single_point():
    net = inputs.siren_init(10, 64, 2)
    on = oracle.Net(inputs.net_to_bytes(net))
    pts = inputs.random_points(3, 37)
    g, v = on.grad_batch(pts, with_value=True, threads=3)
    for i in (0, 17, 36):
        assert np.array_equal(g[:, i], on.grad(pts[:, i].astype(np.float64)))
        assert v[i] == on.eval(pts[:, i].astype(np.float64))


def test_hadamard_identity_of_sec_5_1():
    """(W (.) cos[a|...|a]) G = (W G) (.) cos(a), the identity behind Alg. 2."""
    rng = np.random.default_rng(3)
    W = rng.normal(size=(7, 5))
    a = rng.normal(size=7)
    G = rng.normal(size=(5, 3))
    lhs = (W * np.cos(a)[:, None]) @ G
    rhs = (W @ G) * np.cos(a)[:, None]
    assert np.allclose(lhs, rhs, atol=1e-14)


def test_4d_network_time_input():
    net = inputs.siren_init(12, 64, 1, in_dim=4)
    on = oracle.Net(inputs.net_to_bytes(net))
    sdf = oracle.SDF.of_net(on, time=0.25)
    p = np.array([0.1, 0.2, -0.3])
    assert sdf.value(p) == on.eval(np.array([0.1, 0.2, -0.3, 0.25]))
    g = on.grad_batch(p[:, None], time=0.25)[:, 0]
    assert np.allclose(g, on.grad(np.array([0.1, 0.2, -0.3, 0.25]))[:3], rtol=0, atol=0)


# ---------------------------------------------------------------------------
# P4: Alg. 1 on exact SDFs
# ---------------------------------------------------------------------------

def ray_sphere(o, v, c, r):
    oc = o - c
    b = oc @ v
    disc = b * b - (oc @ oc - r * r)
    if disc < 0:
        return None
    t = -b - math.sqrt(disc)
    return t if t >= 0 else None


def test_sphere_hit_matches_quadratic_root():
    c, r = np.array([0.1, -0.05, 0.0]), 0.5
    tp = oracle.TraceParams([oracle.SDF.sphere(c, r)], [0.0], [200], [1.0], 1e-6)
    o_all, v_all = inputs.random_rays(5, 400)
    n_hit = 0
    for i in range(o_all.shape[1]):
        o = o_all[:, i].astype(np.float64)
        v = v_all[:, i].astype(np.float64)
        v /= np.linalg.norm(v)
        t_ref = ray_sphere(o, v, c, r)
        res = tp.trace_ray(o, v)
        if t_ref is None:
            assert res.hit == 0
            continue
        cosang = abs((o + t_ref * v - c) @ v) / r
        if cosang < 0.2:
            continue  # grazing: convergence along the ray is slow
        n_hit += 1
        assert res.hit == 1
        assert abs(res.tau - t_ref) <= 1e-6 / cosang + 1e-12
        assert np.allclose(res.p, o + res.tau * v, atol=1e-12)
    assert n_hit > 100


def ray_torus_roots(o, v, R, r):
    """Real roots t of |(o + t v) - torus| = 0 (torus about z), via the quartic."""
    ox, oy, oz = o
    vx, vy, vz = v
    # (|p|^2 + R^2 - r^2)^2 = 4 R^2 (x^2 + y^2)
    a2 = vx * vx + vy * vy + vz * vz
    a1 = 2 * (ox * vx + oy * vy + oz * vz)
    a0 = ox * ox + oy * oy + oz * oz + R * R - r * r
    q = np.polymul([a2, a1, a0], [a2, a1, a0])
    q = np.polysub(q, 4 * R * R * np.array([vx * vx + vy * vy, 2 * (ox * vx + oy * vy), ox * ox + oy * oy]))
    roots = np.roots(q)
    return sorted(x.real for x in roots if abs(x.imag) < 1e-9 and x.real >= 0)


def test_torus_hit_matches_quartic_and_dense_march():
    R, r = 0.5, 0.2
    tor = oracle.SDF.torus((0, 0, 0), R, r)
    tp = oracle.TraceParams([tor], [0.0], [400], [1.0], 1e-7)
    o_all, v_all = inputs.random_rays(6, 300)
    checked = 0
    for i in range(o_all.shape[1]):
        o = o_all[:, i].astype(np.float64)
        v = v_all[:, i].astype(np.float64)
        v /= np.linalg.norm(v)
        roots = ray_torus_roots(o, v, R, r)
        res = tp.trace_ray(o, v)
        if not roots:
            assert res.hit == 0
            continue
        t_ref = roots[0]
        t_dm = oracle.first_root(tor, o, v, 0.0, 6.0, h=1e-4, tol=1e-13)
        p = o + t_ref * v
        q = np.array([p[0], p[1]]) * (1 - R / math.hypot(p[0], p[1]))
        nrm = np.array([q[0], q[1], p[2]]) / r
        cosang = abs(nrm @ v)
        if cosang < 0.3:
            continue
        checked += 1
        assert t_dm is not None and abs(t_dm - t_ref) <= 1e-9
        assert res.hit == 1
        assert abs(res.tau - t_ref) <= 1e-7 / cosang + 1e-10
    assert checked > 50


def test_nested_sphere_shells_equal_single_level():
    """f_1 = sphere of radius r + delta_1 nests the sphere f_2 of radius r (Eq. 1)."""
    c, r, d1 = np.zeros(3), 0.45, 0.03
    f1 = oracle.SDF.sphere(c, r + d1)
    f2 = oracle.SDF.sphere(c, r)
    two = oracle.TraceParams([f1, f2], [d1, 0.0], [100, 100], [1.0, 1.0], 1e-8)
    one = oracle.TraceParams([f2], [0.0], [200], [1.0], 1e-8)
    o_all, v_all = inputs.random_rays(7, 300)
    for i in range(o_all.shape[1]):
        o = o_all[:, i].astype(np.float64)
        v = v_all[:, i].astype(np.float64)
        v /= np.linalg.norm(v)
        a, b = two.trace_ray(o, v), one.trace_ray(o, v)
        t_ref = ray_sphere(o, v, c, r)
        if t_ref is None:
            # the coarse shell may be hit while the fine sphere is missed
            assert b.hit == 0
            continue
        cosang = abs((o + t_ref * v - c) @ v) / r
        if cosang < 0.2:
            continue
        assert a.hit == 1 and b.hit == 1
        assert abs(a.tau - t_ref) <= 1e-8 / cosang + 1e-12
        assert abs(a.tau - b.tau) <= 2e-8 / cosang + 1e-12


def test_final_mode_stops_on_the_last_shell_and_mode_0_ignores_it():
    """delta_m is used only with final_mode 1 (reading R4): on the exact sphere SDF |p - c| - r a
    level with final_mode 1 and delta 0.1 ends on the sphere of radius r + 0.1 (the first root of
    f - delta, a quadratic), while final_mode 0 ends on the surface itself whatever delta_m says."""
    c, r, d = np.array([0.05, 0.0, -0.1]), 0.4, 0.1
    shell = oracle.TraceParams([oracle.SDF.sphere(c, r)], [d], [300], [1.0], 1e-9, final_mode=1)
    surface = oracle.TraceParams([oracle.SDF.sphere(c, r)], [d], [300], [1.0], 1e-9, final_mode=0)
    o_all, v_all = inputs.random_rays(8, 300)
    checked = 0
    for i in range(o_all.shape[1]):
        o = o_all[:, i].astype(np.float64)
        v = v_all[:, i].astype(np.float64)
        v /= np.linalg.norm(v)
        t_shell, t_surf = ray_sphere(o, v, c, r + d), ray_sphere(o, v, c, r)
        a, b = shell.trace_ray(o, v), surface.trace_ray(o, v)
        if t_shell is None:
            assert a.hit == 0 and b.hit == 0
            continue
        cos_shell = abs((o + t_shell * v - c) @ v) / (r + d)
        if cos_shell < 0.2 or (t_surf is not None and abs((o + t_surf * v - c) @ v) / r < 0.2):
            continue  # grazing
        checked += 1
        assert a.hit == 1 and abs(a.tau - t_shell) <= 1e-9 / cos_shell + 1e-12
        assert abs(np.linalg.norm(a.p - c) - (r + d)) <= 1e-9
        if t_surf is None:
            assert b.hit == 0
        else:
            assert b.hit == 1 and abs(np.linalg.norm(b.p - c) - r) <= 1e-9
    assert checked > 50


def test_normal_map_is_the_unit_gradient_masked_and_zero_at_critical_points():
    """Normal mapping (Sec. 5, reading R10) on a (w, 0) network whose gradient is known in closed
    form, sum_k c_k cos(w_k . p + b_k) w_k: the unit vector where the mask is set, (0, 0, 0) where it
    is not, and (0, 0, 0) where |grad f| < 1e-12 (output weights scaled to make the gradient vanish)."""
    net = single_sine_layer_net(23, 16)
    W = net.weights[0].astype(np.float64)
    b = net.biases[0].astype(np.float64)
    cw = net.weights[1][0].astype(np.float64)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, (3, 40))
    mask = (np.arange(40) % 3 != 0).astype(np.uint8)
    out = oracle.Net(inputs.net_to_bytes(net)).normal_map(pts, mask)
    for i in range(40):
        if not mask[i]:
            assert np.all(out[:, i] == 0.0)
            continue
        g = (cw * np.cos(W @ pts[:, i] + b)) @ W
        assert np.max(np.abs(out[:, i] - g / np.linalg.norm(g))) <= 1e-12
    # a network with a vanishing gradient everywhere, and one just above the threshold
    for scale, zero in ((1e-16, True), (1e-6, False)):
        tiny = single_sine_layer_net(23, 16)
        tiny.weights[1] = (tiny.weights[1].astype(np.float64) * scale).astype(tiny.weights[1].dtype)
        got = oracle.Net(inputs.net_to_bytes(tiny)).normal_map(pts[:, :5])
        if zero:
            assert np.all(got == 0.0)
        else:
            assert np.allclose(np.linalg.norm(got, axis=0), 1.0, atol=1e-12)


def test_batch_driver_is_the_pinned_single_ray_trace():
    """The threaded batch driver (all rays, or an index subset, several threads) gives, in list order,
    exactly the single-ray trace that the closed-form pins above check."""
    c, r = np.array([0.0, 0.1, 0.0]), 0.45
    tp = oracle.TraceParams([oracle.SDF.sphere(c, r + 0.05), oracle.SDF.sphere(c, r)], [0.05, 0.0], [60, 60],
                            [1.0, 1.0], 1e-7)
    o_all, v_all = inputs.random_rays(9, 257)
    o32, v32 = o_all.astype(np.float32), v_all.astype(np.float32)
    idx = np.array([256, 3, 3, 100, 0, 17], np.int64)
    for sel, threads in ((None, 5), (idx, 3)):
        res = tp.trace_batch(o32, v32, idx=sel, threads=threads)
        rows = range(o32.shape[1]) if sel is None else sel
        for k, i in enumerate(rows):
            one = tp.trace_ray(o32[:, i].astype(np.float64), v32[:, i].astype(np.float64))
            assert res["hit"][k] == one.hit and res["iters"][k] == one.iters
            assert np.array_equal(res["pos"][:, k], np.array(one.p[:3]))


def test_alg1_steps_before_testing():
    """Alg. 1 applies p = p + t v before re-testing t: one step lands exactly on a plane SDF."""
    # a sphere of huge radius is a plane to within 1e-12 near the ray
    c = np.array([0.0, 0.0, -1e6])
    f = oracle.SDF.sphere(c, 1e6 + 0.2)  # surface near z = 0.2
    tp = oracle.TraceParams([f], [0.0], [10], [1.0], 1e-9, box=(-1, 1))
    res, traj, _ = tp.trace_ray(np.array([0.0, 0.0, 2.0]), np.array([0.0, 0.0, -1.0]), traj_cap=10)
    assert res.hit == 1
    assert len(traj) == 2  # one step to the surface, one more to measure t <= eps
    assert abs(res.p[2] - 0.2) <= 1e-9


# ---------------------------------------------------------------------------
# P5/P6: the Lipschitz step never crosses the surface; brute force first hit
# ---------------------------------------------------------------------------

def test_lipschitz_bound_matches_lapack():
    from paper_2201_09147_gb300 import workloads
    net = workloads.random_siren_64x1()
    on = oracle.Net(inputs.net_to_bytes(net))
    Ws, _, wo, _ = folded_arrays(net)
    ref = np.prod([np.linalg.norm(w, 2) for w in Ws]) * np.linalg.norm(wo)
    assert abs(on.lipschitz() - ref) <= 1e-10 * ref


def slab_entry(o, v, lo=-1.0, hi=1.0):
    with np.errstate(divide="ignore"):
        t1, t2 = (lo - o) / v, (hi - o) / v
    return max(0.0, float(np.max(np.minimum(t1, t2))))


def test_lipschitz_steps_never_cross_and_find_first_root():
    """With s = 1/L no step crosses the zero set (|f(p + t v / L) - f(p)| <= |t|)."""
    from paper_2201_09147_gb300 import workloads
    wl = workloads.get("random_siren_64x1", 20, 20)
    on = oracle.Net(inputs.net_to_bytes(wl.levels[0]))
    L = on.lipschitz()
    sdf = oracle.SDF.of_net(on)
    tp = oracle.TraceParams([sdf], [0.0], [600], [1.0 / L], 1e-3)
    orig, dirs = wl.rays()
    n_hits = 0
    for i in range(orig.shape[1]):
        o = orig[:, i].astype(np.float64)
        v = dirs[:, i].astype(np.float64)
        res, traj, _ = tp.trace_ray(o, v, traj_cap=600)
        if len(traj) < 2:
            continue
        vals = np.array([on.eval(q) for q in traj])
        # every iterate stays on the side of the zero set where the ray started
        assert np.all(vals * vals[0] >= 0.0), i
        if res.hit and vals[0] > 0:
            n_hits += 1
            assert abs(on.eval(res.p)) <= 1e-3 + 1e-9
            # the first root along the ray lies at or beyond the end point
            t_end = float((res.p - o) @ v)
            t_in = slab_entry(o, v)
            t_root = oracle.first_root(sdf, o, v, t_in, t_end + 1e-3, h=1e-4, tol=1e-12)
            assert t_root is None or t_root >= t_end - 1e-9
    assert n_hits > 3


def test_box_exit_means_no_root_on_the_path():
    """A Lipschitz-stepped ray that leaves the box passed no root (dense march over the path)."""
    from paper_2201_09147_gb300 import workloads
    wl = workloads.get("random_siren_64x1", 16, 16)
    on = oracle.Net(inputs.net_to_bytes(wl.levels[0]))
    sdf = oracle.SDF.of_net(on)
    L = on.lipschitz()
    tp = oracle.TraceParams([sdf], [0.0], [400], [1.0 / L], 1e-3)
    orig, dirs = wl.rays()
    exits = 0
    for i in range(orig.shape[1]):
        o = orig[:, i].astype(np.float64)
        v = dirs[:, i].astype(np.float64)
        res = tp.trace_ray(o, v)
        if res.hit or res.iters == 0:
            continue
        t_in = slab_entry(o, v)
        if on.eval(o + t_in * v) <= 0:
            continue
        exits += 1
        t_root = oracle.first_root(sdf, o, v, t_in, res.tau - 2e-3, h=2e-4, tol=1e-9)
        assert t_root is None
    assert exits > 20


# ---------------------------------------------------------------------------
# P7: threshold recurrences of Props. 1 and 2 imply the nesting of Eq. 1
# ---------------------------------------------------------------------------

def _nested(f_coarse, d_coarse, f_fine, d_fine):
    inner = np.abs(f_fine) <= d_fine
    return np.all(np.abs(f_coarse[inner]) <= d_coarse)


def test_prop2_thresholds_nest_approximations_of_one_surface():
    rng = np.random.default_rng(4)
    P = rng.uniform(-1, 1, (200000, 3))
    f = np.linalg.norm(P, axis=1) - 0.5
    eps = np.array([0.05, 0.02, 0.008])
    fs = [f + e * np.sin(7 * k + 11 * P[:, 0]) * np.cos(5 * P[:, 1] - k) * 0.999 for k, e in enumerate(eps)]
    delta = oracle.thresholds_prop2(eps)
    assert np.all(np.diff(delta) < 0)
    for j in range(len(eps) - 1):
        assert _nested(fs[j], delta[j], fs[j + 1], delta[j + 1])
    # shrinking a threshold below the recurrence breaks the nesting for adversarial errors
    adv = [f + eps[0] * 0.999, f - eps[1] * 0.999]
    d2 = oracle.thresholds_prop2(eps[:2])
    assert _nested(adv[0], d2[0], adv[1], d2[1])
    assert not _nested(adv[0], d2[0] * 0.98, adv[1], d2[1])


def test_prop1_thresholds_nest_successive_differences():
    rng = np.random.default_rng(5)
    P = rng.uniform(-1, 1, (200000, 3))
    base = np.linalg.norm(P - 0.1, axis=1) - 0.4
    eps = np.array([0.0, 0.03, 0.01, 0.004])  # eps[0] unused by Prop. 1
    fs = [base]
    for k in range(1, len(eps)):
        fs.append(fs[-1] + eps[k] * 0.999 * np.sin(3 * k + 9 * P[:, 2]))
    delta = oracle.thresholds_prop1(eps)
    for j in range(len(eps) - 1):
        assert _nested(fs[j], delta[j], fs[j + 1], delta[j + 1])
    adv = [base, base + eps[1] * 0.999]
    d2 = oracle.thresholds_prop1(eps[:2])
    assert _nested(adv[0], d2[0], adv[1], d2[1])
    assert not _nested(adv[0], d2[0] * 0.97, adv[1], d2[1])


# ---------------------------------------------------------------------------
# fitting objective and optimiser step (the training path)
# ---------------------------------------------------------------------------

def _two_layer_by_hand(net, P):
    """f and grad f of a (w, 1) plain network (omega = 1) at points P (n, 3) by
    reverse-mode differentiation written out: grad f = W0^T [cos A0 (.) W1^T (cos A1 (.) w)]."""
    W0, b0 = net.weights[0].astype(np.float64), net.biases[0].astype(np.float64)
    W1, b1 = net.weights[1].astype(np.float64), net.biases[1].astype(np.float64)
    wo, bo = net.weights[2][0].astype(np.float64), float(net.biases[2][0])
    f, g = [], []
    for p in P:
        a0 = W0 @ p + b0
        a1 = W1 @ np.sin(a0) + b1
        f.append(wo @ np.sin(a1) + bo)
        g.append(W0.T @ (np.cos(a0) * (W1.T @ (np.cos(a1) * wo))))
    return np.array(f), np.array(g).T


def test_fit_loss_matches_hand_computation():
    net = inputs.random_plain_net(31, 5, 1, scale=1.2)
    b = inputs.net_to_bytes(net)
    rng = np.random.default_rng(3)
    P = rng.uniform(-1, 1, (40, 3))
    f, g = _two_layer_by_hand(net, P)
    tf = rng.normal(size=40)
    tg = rng.normal(size=(3, 40))
    near = rng.uniform(size=40) < 0.4
    lam_n, lam_e = 0.1, 0.05
    l_val = np.mean(np.abs(f - tf))
    cos = [np.dot(g[:, i], tg[:, i]) / np.linalg.norm(g[:, i]) / np.linalg.norm(tg[:, i]) for i in range(40)]
    l_dir = np.mean([1.0 - c for c, m in zip(cos, near) if m])
    l_eik = np.mean(np.abs(np.linalg.norm(g, axis=0) - 1.0))
    L, parts = oracle.fit_loss(b, P.T.copy(), tf, tg, near, lam_n, lam_e)
    assert np.allclose(parts, (l_val, l_dir, l_eik), rtol=1e-12, atol=1e-14)
    assert abs(L - (l_val + lam_n * l_dir + lam_e * l_eik)) <= 1e-12


def test_fit_loss_vanishes_on_the_network_itself():
    """Targets equal to f and to any positive multiple of grad f zero the value and
    direction terms; with no near points the direction term is 0."""
    net = inputs.random_plain_net(32, 6, 1, scale=1.0)
    b = inputs.net_to_bytes(net)
    P = np.random.default_rng(4).uniform(-1, 1, (25, 3))
    f, g = _two_layer_by_hand(net, P)
    L, (lv, ld, le) = oracle.fit_loss(b, P.T.copy(), f, 3.0 * g, np.ones(25, bool), 0.1, 0.05)
    assert lv <= 1e-14 and ld <= 1e-13
    assert abs(le - np.mean(np.abs(np.linalg.norm(g, axis=0) - 1.0))) <= 1e-13
    _, (_, ld0, _) = oracle.fit_loss(b, P.T.copy(), f, -g, np.zeros(25, bool), 0.1, 0.05)
    assert ld0 == 0.0
    _, (_, ld2, _) = oracle.fit_loss(b, P.T.copy(), f, -g, np.ones(25, bool), 0.1, 0.05)
    assert abs(ld2 - 2.0) <= 1e-12  # opposite directions: 1 - cos = 2


def test_adam_step_matches_torch_optimizer():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    theta0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(4)]
    t = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for k, gk in enumerate(grads, start=1):
        t.grad = torch.tensor(gk, dtype=torch.float64)
        opt.step()
        th, m, v = oracle.adam_step(th, gk, m, v, k, 1e-3)
    assert np.allclose(t.detach().numpy(), th, rtol=0, atol=1e-15)


def test_sine_arguments_of_the_committed_networks_stay_in_the_tested_range():
    """Every sine argument (pre-activation W_l x + b_l, frequencies folded) of every committed
    network at 2 * 10^5 points of the cube lies within |x| <= 256, the range over which the
    kernels' sine and cosine are tested against FP64 on the GPU."""
    import numpy as np

    import oracle
    from paper_2201_09147_gb300 import inputs, workloads
    pts = inputs.random_points(17, 200_000).astype(np.float64)
    for path in sorted(workloads.SCENES.glob("*.sdfn")):
        b = path.read_bytes()
        p = pts if oracle._parse_sdfn(b)[0] == 3 else np.vstack([pts, inputs.uniform01(18, pts.shape[1])[None, :]])
        m = oracle.max_preactivation(b, p)
        print(path.name, [round(float(v), 1) for v in m])
        assert max(m) <= 256.0


# ---------------------------------------------------------------------------
# 16-bit weight image (reference-only mode: weight rounding vs arithmetic error)
# ---------------------------------------------------------------------------

def test_round_bf16_ties_to_even_and_matches_torch():
    """Hand cases of round-to-nearest-even at 8 significand bits, then random float32 values
    against torch's own float32 -> bfloat16 conversion (a library routine)."""
    torch = pytest.importorskip("torch")
    h = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 1 + 2 ** -8 + 2 ** -20, 2 ** -130], np.float32)
    assert oracle.round_bf16(h).tolist() == [1.0, 1.0, 1 + 2 ** -6, -1.0, 1 + 2 ** -7, 2 ** -130]
    x = (np.random.default_rng(5).standard_normal(200_000) * 30).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.round_bf16(x), ref)


def _params(data):
    in_dim, width, n_hidden, layers, w_out, b_out = oracle._parse_sdfn(data)
    return layers, w_out, b_out


def test_quantised_image_rounds_only_the_hidden_weights():
    """Hidden weights: the 16-bit rounding of float32(omega W) (within half an ulp, exactly
    representable); layer 0, biases and the output row: float32 of the folded values."""
    b = inputs.net_to_bytes(inputs.siren_init(3, 64, 2))
    ref_layers, ref_wo, ref_bo = _params(b)
    for fmt, ulp_bits in (("bf16", 8), ("f16", 11)):
        layers, w_out, b_out = _params(oracle.quantised_image(b, fmt))
        for li, ((W, bb), (W0, b0)) in enumerate(zip(layers, ref_layers)):
            f32 = W0.astype(np.float32).astype(np.float64)
            assert np.array_equal(bb, b0.astype(np.float32).astype(np.float64))
            if li == 0:
                assert np.array_equal(W, f32)
                continue
            # half an ulp: relative 2^-(bits) for normal values; half the smallest subnormal (2^-25)
            # below half's normal range (bfloat16 has float32's exponent range)
            err, mag = np.abs(W - f32), np.abs(f32)
            normal = mag >= (2.0 ** -14 if fmt == "f16" else 2.0 ** -126)
            assert (err[normal] / mag[normal]).max() <= 2.0 ** -ulp_bits * 1.0000001
            assert np.all(err[~normal] <= 2.0 ** -25)
            assert not np.array_equal(W, f32)  # a random layer is not 16-bit exact
            if fmt == "bf16":
                assert np.all((W.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)
            else:
                assert np.array_equal(W.astype(np.float16).astype(np.float64), W)
        assert np.array_equal(w_out, ref_wo.astype(np.float32).astype(np.float64)) and b_out == np.float32(ref_bo)


def test_quantised_image_of_a_16bit_exact_net_evaluates_unchanged():
    """A folded network whose hidden weights are already bfloat16 values is its own 16-bit image:
    the oracle's f at random points is then identical, bit for bit."""
    net = inputs.siren_init(4, 64, 2)
    folded = inputs.SineNet(net.in_dim, net.width, net.n_hidden, net.omega0, net.omega,
                            [w.astype(np.float64) * (net.omega0 if i == 0 else (net.omega if i <= net.n_hidden else 1.0))
                             for i, w in enumerate(net.weights)],
                            [b.astype(np.float64) * (net.omega0 if i == 0 else (net.omega if i <= net.n_hidden else 1.0))
                             for i, b in enumerate(net.biases)], folded=True)
    for i in range(1, net.n_hidden + 1):
        folded.weights[i] = oracle.round_bf16(np.asarray(folded.weights[i], np.float32))
    b = inputs.net_to_bytes(folded)
    pts = inputs.random_points(9, 2000).astype(np.float64)
    assert np.array_equal(oracle.eval_batch(oracle.quantised_image(b), pts), oracle.eval_batch(b, pts))
