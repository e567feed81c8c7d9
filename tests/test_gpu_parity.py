"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (tests/parity.py, per precision): hit/miss agreement; on rays both
sides call hits, end-point distance p99.9; normal angle at the same point
p99.9.  FP32: 99.9 %, 1e-5, 0.01 deg.  FP16: 99.9 %, 1e-3, 0.5 deg.  BF16:
bounds scaled by its 8x larger unit roundoff.
"""
import ctypes as C
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2201_09147_gb300 import inputs, workloads
from parity import (DECISION_MARGIN, FP8_ANGLE_MEDIAN_DEG, FP8_ANGLE_P999_DEG, FP8_MAGNITUDE_REL, FP8_TRACE_AGREEMENT,
                    FP8_TRACE_POS_MEDIAN, FP8_TRACE_POS_P99, HIT_AGREEMENT,
                    PRECISION_IDS, PRECISIONS, RANDOM_NET_ANGLE_FACTOR, TOL, angle_report, bf16_within_fp16,
                    capped_report, trace_report)

pytestmark = pytest.mark.gpu


def gpu_trace(sdf, level_bytes, precision, wl, orig, dirs, step_scale="wl"):
    nets = [sdf.Net(b, precision) for b in level_bytes]
    o = torch.from_numpy(np.ascontiguousarray(orig)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(dirs)).cuda()
    ss = wl.step_scale if step_scale == "wl" else step_scale
    pos, t, hit, iters = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, o, d, step_scale=ss,
                                              final_mode=wl.final_mode)
    sdf.sync_status()
    return {"pos": pos.cpu().numpy(), "t": t.cpu().numpy(), "hit": hit.cpu().numpy(),
            "iters": iters.cpu().numpy().astype(np.int64), "nets": nets, "pos_dev": pos, "hit_dev": hit}


def oracle_trace(level_bytes, wl, orig, dirs, idx=None):
    onets = [oracle.Net(b) for b in level_bytes]
    scales = wl.step_scale if wl.step_scale is not None else [1.0 / n.lipschitz() for n in onets]
    tp = oracle.TraceParams([oracle.SDF.of_net(n) for n in onets], wl.delta, wl.caps, scales, wl.eps,
                            final_mode=wl.final_mode)
    return tp.trace_batch(orig, dirs, idx=idx)


def fp16_twin(sdf, net_bytes, pts_dev, mask_dev=None, time_dev=None):
    """Unit normals of the same network with FP16 operands at the same device points (host array)."""
    net = sdf.Net(net_bytes, sdf.SDF_FP16)
    out = (sdf.normal_map(net, pts_dev, mask_dev) if time_dev is None
           else sdf.normal_map_timed(net, pts_dev, time_dev, mask_dev))
    sdf.sync_status()
    return out.cpu().numpy()


def assert_bf16_ratio(ar_bf16, ar_fp16, label=""):
    print(label, "normal p99.9 bf16", ar_bf16["angle_p999"], "fp16", ar_fp16["angle_p999"])
    assert bf16_within_fp16(ar_bf16["angle_p999"], ar_fp16["angle_p999"])


def check_trace(g, o, precision, label):
    agree_tol, pos_tol, _ = TOL[precision]
    rep = trace_report(g["pos"], g["hit"], o["pos"], o["hit"])
    print(label, {k: v for k, v in rep.items() if k != "both"})
    assert rep["agree"] >= agree_tol, (label, rep["agree"])
    assert rep["pos_p999"] <= pos_tol, (label, rep["pos_p999"])
    return rep


# ---------------------------------------------------------------------------
# network preparation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(64, 1), (128, 2), (256, 3), (256, 4)])
def test_lipschitz_matches_oracle(sdf, shape):
    b = inputs.net_to_bytes(inputs.siren_init(3, shape[0], shape[1]))
    n = sdf.Net(b, sdf.SDF_FP32)
    ref = oracle.Net(b).lipschitz()
    assert abs(n.lipschitz - ref) <= 1e-9 * ref
    assert (n.in_dim, n.width, n.n_hidden) == (3, shape[0], shape[1])


def test_load_rejects_bad_input(sdf):
    b = inputs.net_to_bytes(inputs.siren_init(0, 64, 1))
    with pytest.raises(sdf.SdfError) as e:
        sdf.Net(b[:-4], sdf.SDF_BF16)
    assert e.value.code == -3
    bad = bytearray(b)
    bad[40:44] = np.array([np.nan], np.float32).tobytes()
    with pytest.raises(sdf.SdfError) as e:
        sdf.Net(bytes(bad), sdf.SDF_BF16)
    assert e.value.code == -5
    with pytest.raises(sdf.SdfError) as e:
        sdf.Net(b, sdf.SDF_FP8)
    assert e.value.code == -7
    odd = inputs.net_to_bytes(inputs.siren_init(0, 96, 1))
    with pytest.raises(sdf.SdfError) as e:
        sdf.Net(odd, sdf.SDF_FP32)
    assert e.value.code == -7


# ---------------------------------------------------------------------------
# analytic normals (Alg. 2)
# ---------------------------------------------------------------------------

NORMAL_NETS = [("siren64x1", lambda: inputs.net_to_bytes(workloads.random_siren_64x1())),
               ("siren128x2", lambda: inputs.net_to_bytes(inputs.siren_init(5, 128, 2))),
               ("siren256x3", lambda: inputs.net_to_bytes(inputs.siren_init(6, 256, 3))),
               ("siren256x4", lambda: inputs.net_to_bytes(inputs.siren_init(7, 256, 4))),
               ("scene256x3", lambda: (workloads.SCENES / "s8_256x3.sdfn").read_bytes()),
               ("scene64x1", lambda: (workloads.SCENES / "s8_64x1.sdfn").read_bytes())]


@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
@pytest.mark.parametrize("name,make", NORMAL_NETS, ids=[n for n, _ in NORMAL_NETS])
def test_normals_vs_oracle(sdf, precision, name, make):
    b = make()
    n = 4096 + 37  # several tiles and a ragged tail
    pts = inputs.random_points(11, n, -1.0, 1.0)
    net = sdf.Net(b, precision)
    g = sdf.normals(net, torch.from_numpy(pts).cuda())
    nm = sdf.normal_map(net, torch.from_numpy(pts).cuda())
    sdf.sync_status()
    g = g.cpu().numpy()
    nm = nm.cpu().numpy()
    ref = oracle.Net(b).grad_batch(pts)
    tol = TOL[precision][2] * (RANDOM_NET_ANGLE_FACTOR if name.startswith("siren") and precision else 1.0)
    ok = np.linalg.norm(ref, axis=0) > 1e-3 * np.median(np.linalg.norm(ref, axis=0))
    rep = angle_report(g, ref, ok)
    print(name, precision, rep)
    assert rep["angle_p999"] <= tol
    rel = np.linalg.norm(g - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert np.quantile(rel[ok], 0.999) <= np.radians(tol) * 4 + 1e-4
    # normal map = unit gradient
    unit = ref / np.linalg.norm(ref, axis=0, keepdims=True)
    ar_nm = angle_report(nm, unit, ok)
    assert ar_nm["angle_p999"] <= tol
    assert np.allclose(np.linalg.norm(nm, axis=0)[ok], 1.0, atol=1e-5)
    if precision == sdf.SDF_BF16:
        assert_bf16_ratio(ar_nm, angle_report(fp16_twin(sdf, b, torch.from_numpy(pts).cuda()), unit, ok), name)


@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_normal_map_mask(sdf, precision):
    b = (workloads.SCENES / "s8_256x3.sdfn").read_bytes()
    n = 3000
    pts = inputs.random_points(12, n, -0.8, 0.8)
    mask = (inputs.uniform01(13, n) < 0.4).astype(np.uint8)
    net = sdf.Net(b, precision)
    out = torch.full((3, n), 7.0, device="cuda")
    sdf.normal_map(net, torch.from_numpy(pts).cuda(), torch.from_numpy(mask).cuda(), out=out)
    sdf.sync_status()
    out = out.cpu().numpy()
    m = mask.astype(bool)
    assert np.all(out[:, ~m] == 0.0)
    ref = oracle.Net(b).normal_map(pts, mask)
    ar = angle_report(out, ref, m)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        twin = fp16_twin(sdf, b, torch.from_numpy(pts).cuda(), torch.from_numpy(mask).cuda())
        assert_bf16_ratio(ar, angle_report(twin, ref, m), "mask")


# ---------------------------------------------------------------------------
# multiscale sphere tracing (Alg. 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_trace_random_siren(sdf, precision):
    """128 x 128 rays, Lipschitz steps, 32 iterations: trajectories must agree."""
    wl = workloads.get("random_siren_64x1")
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    o = oracle_trace(lb, wl, orig, dirs)
    check_trace(g, o, precision, f"random_siren p={precision}")
    same_iters = np.mean(g["iters"] == o["iters"])
    print("same iteration count", same_iters)
    if precision == 0:
        assert same_iters >= HIT_AGREEMENT
        # every ray, hit or miss, ends at the same point
        d = np.linalg.norm(g["pos"] - o["pos"], axis=0)
        assert np.quantile(d, 0.999) <= 1e-4
    # normals of the traced net at the GPU's own hit points
    hit = g["hit"].astype(bool)
    nrm = sdf.normal_map(g["nets"][0], g["pos_dev"], g["hit_dev"])
    sdf.sync_status()
    ref = oracle.Net(lb[0]).normal_map(g["pos"].astype(np.float64), g["hit"])
    tol = TOL[precision][2] * (RANDOM_NET_ANGLE_FACTOR if precision else 1.0)
    ar = angle_report(nrm.cpu().numpy(), ref, hit)
    assert ar["angle_p999"] <= tol
    if precision == sdf.SDF_BF16:
        assert_bf16_ratio(ar, angle_report(fp16_twin(sdf, lb[0], g["pos_dev"], g["hit_dev"]), ref, hit), "siren")


@pytest.mark.parametrize("name", ["normal_map_1080p", "normal_map_1080p_c64x2", "normal_map_1080p_zero"])
@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_normal_map_workload_small(sdf, precision, name):
    """Coarse (64,1) to its delta shell, then (256,3) normals (Sec. 5), 200 x 113 rays; and config 3's
    other readings: the (64,2) as the coarse net, and the (64,1) traced to its zero set."""
    wl = workloads.get(name, 200, 113)
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    o = oracle_trace(lb, wl, orig, dirs)
    rep = check_trace(g, o, precision, f"{name} small p={precision}")
    assert rep["n_both"] > 1000
    fine = sdf.Net(wl.fine_bytes(), precision)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"])
    sdf.sync_status()
    nrm = nrm.cpu().numpy()
    hit = g["hit"].astype(bool)
    assert np.all(nrm[:, ~hit] == 0.0)
    ref = oracle.Net(wl.fine_bytes()).normal_map(g["pos"].astype(np.float64), g["hit"])
    ar = angle_report(nrm, ref, hit)
    print(ar)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        twin = fp16_twin(sdf, wl.fine_bytes(), g["pos_dev"], g["hit_dev"])
        assert_bf16_ratio(ar, angle_report(twin, ref, hit), name)


@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_nested_3level_small(sdf, precision):
    """(64,2) |> (128,2) |> (256,2) at 96 x 96 rays, then the finest net's normals at the hits."""
    wl = workloads.get("nested_3level_512", 96, 96)
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    o = oracle_trace(lb, wl, orig, dirs)
    rep = check_trace(g, o, precision, f"nested_3level p={precision}")
    assert rep["n_both"] > 500
    fine = sdf.Net(wl.fine_bytes(), precision)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"])
    sdf.sync_status()
    ref = oracle.Net(wl.fine_bytes()).normal_map(g["pos"].astype(np.float64), g["hit"])
    ar = angle_report(nrm.cpu().numpy(), ref, g["hit"].astype(bool))
    print(ar)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        twin = fp16_twin(sdf, wl.fine_bytes(), g["pos_dev"], g["hit_dev"])
        assert_bf16_ratio(ar, angle_report(twin, ref, g["hit"].astype(bool)), wl.name)


@pytest.mark.parametrize("name", ["three_level_512", "silhouette_512"])
@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_three_level_normal_map_small(sdf, precision, name):
    """(64,1) |> (256,1 or 2), 20 + 5 steps to the delta shells, then (256,3) normals (Tab. 3), 128 x 128."""
    wl = workloads.get(name, 128, 128)
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    o = oracle_trace(lb, wl, orig, dirs)
    rep = check_trace(g, o, precision, f"{name} p={precision}")
    assert rep["n_both"] > 1500
    assert g["iters"].max() <= sum(wl.caps)
    if precision == 0:
        assert np.mean(g["iters"] == o["iters"]) >= 0.99
    fine = sdf.Net(wl.fine_bytes(), precision)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"])
    sdf.sync_status()
    ref = oracle.Net(wl.fine_bytes()).normal_map(g["pos"].astype(np.float64), g["hit"])
    ar = angle_report(nrm.cpu().numpy(), ref, g["hit"].astype(bool))
    print(ar)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        twin = fp16_twin(sdf, wl.fine_bytes(), g["pos_dev"], g["hit_dev"])
        assert_bf16_ratio(ar, angle_report(twin, ref, g["hit"].astype(bool)), wl.name)


@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_plain_256x3_small(sdf, precision):
    """The single-network (256,3) tracer (streamed weights on the tensor cores), 120 x 68 rays."""
    wl = workloads.get("plain_256x3_1080p", 120, 68)
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    o = oracle_trace(lb, wl, orig, dirs)
    rep = check_trace(g, o, precision, f"plain_256x3 p={precision}")
    assert rep["n_both"] > 500


@pytest.mark.parametrize("precision", [1, 3], ids=["bf16", "fp16"])
def test_normal_map_1080p_sampled(sdf, precision):
    """Full 1920 x 1080 frame in the benchmark's launch configuration; oracle on 3000 sampled rays."""
    wl = workloads.get("normal_map_1080p")
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    fine = sdf.Net(wl.fine_bytes(), precision)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"])
    sdf.sync_status()
    idx = np.sort(np.unique((inputs.uniform01(99, 3000) * wl.n_rays).astype(np.int64)))
    o = oracle_trace(lb, wl, orig, dirs, idx=idx)
    gs = {"pos": g["pos"][:, idx], "hit": g["hit"][idx]}
    rep = check_trace(gs, o, precision, f"1080p sampled p={precision}")
    assert rep["n_both"] > 300
    hit = gs["hit"].astype(bool)
    ref = oracle.Net(wl.fine_bytes()).normal_map(gs["pos"].astype(np.float64), gs["hit"])
    ar = angle_report(nrm.cpu().numpy()[:, idx], ref, hit)
    print(ar)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        twin = fp16_twin(sdf, wl.fine_bytes(), g["pos_dev"], g["hit_dev"])[:, idx]
        assert_bf16_ratio(ar, angle_report(twin, ref, hit), "1080p sampled")
    # every ray of the frame got a decision and misses carry zero normals
    allhit = g["hit"].astype(bool)
    assert set(np.unique(g["hit"])) <= {0, 1}
    assert np.all(nrm.cpu().numpy()[:, ~allhit] == 0.0)


@pytest.mark.parametrize("name", ["nested_3level_512", "three_level_512", "silhouette_512"])
@pytest.mark.parametrize("precision", [1, 3], ids=["bf16", "fp16"])
def test_512_workloads_full_size_sampled(sdf, precision, name):
    """The 512 x 512 workloads at full size as the benchmark runs them; oracle on 2,000 sampled rays,
    every one of them checked.  Capped schedules (Alg. 1 with the iteration counts of Sec. 6) end
    rays at the eps threshold, where the decision depends on the last bits of the value: a ray whose
    FP64 decision flips when eps moves by the path's value error is ambiguous.  Asserted: the
    decision on every unambiguous ray (agreement bound of the precision); for every GPU hit and for
    every ambiguous ray, that the GPU's own end point lies, in FP64, within eps + 2 margin of the last
    level's level set (the ray really stopped at the threshold); the end points of the common hits.
    The ambiguous share is reported, not bounded."""
    wl = workloads.get(name)
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, precision, wl, orig, dirs)
    fine = sdf.Net(wl.fine_bytes(), precision)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"])
    sdf.sync_status()
    idx = np.sort(np.unique((inputs.uniform01(123, 2000) * wl.n_rays).astype(np.int64)))
    o = oracle_trace(lb, wl, orig, dirs, idx=idx)
    gs = {"pos": g["pos"][:, idx], "hit": g["hit"][idx]}
    m = DECISION_MARGIN[precision]
    lo = oracle_trace(lb, dataclasses.replace(wl, eps=wl.eps - m), orig, dirs, idx=idx)
    hi = oracle_trace(lb, dataclasses.replace(wl, eps=wl.eps + m), orig, dirs, idx=idx)
    d_last = wl.delta[-1] if wl.final_mode == 1 else 0.0
    _, v_end = oracle.Net(lb[-1]).grad_batch(gs["pos"].astype(np.float64), with_value=True)
    rep = capped_report(gs["pos"], gs["hit"], o, lo, hi, v_end - d_last, wl.eps, m)
    print(name, precision, rep)
    agree_tol, pos_tol, _ = TOL[precision]
    assert rep["agree_unambiguous"] >= agree_tol
    assert rep["hit_residual_max"] <= rep["residual_bound"]
    assert rep["ambiguous_residual_max"] <= rep["residual_bound"]
    assert rep["pos_p999"] <= pos_tol
    assert rep["n_both"] > 150
    ref = oracle.Net(wl.fine_bytes()).normal_map(gs["pos"].astype(np.float64), gs["hit"])
    ar = angle_report(nrm.cpu().numpy()[:, idx], ref, gs["hit"].astype(bool))
    print(ar)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        twin = fp16_twin(sdf, wl.fine_bytes(), g["pos_dev"], g["hit_dev"])[:, idx]
        assert_bf16_ratio(ar, angle_report(twin, ref, gs["hit"].astype(bool)), name)


@pytest.mark.parametrize("precision", PRECISIONS, ids=PRECISION_IDS)
def test_mesh_normal_map(sdf, precision):
    """Neural normal mapping onto mesh vertices (Sec. 5): displaced icosphere, subdivision 5."""
    pts, frac = workloads.mesh_points(subdivisions=5)
    assert frac > 0.9
    fine_b = (workloads.SCENES / "s8_256x3.sdfn").read_bytes()
    fine = sdf.Net(fine_b, precision)
    out = sdf.normal_map(fine, torch.from_numpy(pts).cuda())
    sdf.sync_status()
    ref = oracle.Net(fine_b).normal_map(pts.astype(np.float64))
    ar = angle_report(out.cpu().numpy(), ref)
    print(ar)
    assert ar["angle_p999"] <= TOL[precision][2]
    if precision == sdf.SDF_BF16:
        assert_bf16_ratio(ar, angle_report(fp16_twin(sdf, fine_b, torch.from_numpy(pts).cuda()), ref), "mesh5")


_MESH7 = {}


@pytest.mark.parametrize("precision", [1, 3], ids=["bf16", "fp16"])
def test_mesh_normal_map_full_size_sampled(sdf, precision):
    """Neural normal mapping onto the full-size mesh (displaced icosphere, subdivision 7: 163,842
    vertices, the benchmark's size): every normal unit length, the oracle on 3,000 sampled vertices."""
    if "pts" not in _MESH7:
        _MESH7["pts"], _MESH7["frac"] = workloads.mesh_points(subdivisions=7)
    pts = _MESH7["pts"]
    assert pts.shape[1] == 163842 and _MESH7["frac"] > 0.9
    fine_b = (workloads.SCENES / "s8_256x3.sdfn").read_bytes()
    fine = sdf.Net(fine_b, precision)
    out = sdf.normal_map(fine, torch.from_numpy(pts).cuda()).cpu().numpy()
    sdf.sync_status()
    assert np.allclose(np.linalg.norm(out, axis=0), 1.0, atol=1e-5)
    idx = np.sort(np.unique((inputs.uniform01(77, 3000) * pts.shape[1]).astype(np.int64)))
    ref = oracle.Net(fine_b).normal_map(pts[:, idx].astype(np.float64))
    ar = angle_report(out[:, idx], ref)
    print(ar)
    # the stated 0.5 deg for both operand types (BF16 measured 0.47 deg p99.9 on 18,836 vertices)
    assert ar["angle_p999"] <= 0.5


_HITS = {}

# Neural normal mapping of the fitted networks (Sec. 5), p99.9 angle against FP64 at the same points.
# The error of a 16-bit path scales with its operand type's unit roundoff, which is 8x larger for
# bfloat16 than for half: BF16 is held to 12x the FP16 error of the same network at the same points
# (the factor 8, and 1.5 for the shape of the error distribution), FP16 to 0.1 deg, and the
# benchmark's fine (256,3) to the stated 0.5 deg in BF16.  Whether BF16 meets 0.5 deg depends on the
# network (the cancellation in its gradient): it is reported, not asserted, for the others.
FITTED_NORMAL_NETS = ["s8_256x1", "s8_256x2", "s8_256x3", "s8_128x2"]


@pytest.mark.parametrize("name", FITTED_NORMAL_NETS)
def test_normal_bound_per_fitted_network(sdf, name):
    """The coarse (64,1) hits of the 1920 x 1080 frame (every 8th hit) and 20,000 sampled vertices of
    the full-size mesh, BF16 and FP16 operands."""
    if "hits" not in _HITS:
        wl = workloads.get("normal_map_1080p")
        orig, dirs = wl.rays()
        g = gpu_trace(sdf, wl.level_bytes(), sdf.SDF_BF16, wl, orig, dirs)
        hidx = np.nonzero(g["hit"])[0][::8]
        _HITS["hits"] = np.ascontiguousarray(g["pos"][:, hidx])
        mesh = _MESH7.get("pts")
        if mesh is None:
            mesh, _MESH7["frac"] = workloads.mesh_points(subdivisions=7)
            _MESH7["pts"] = mesh
        midx = np.sort(np.unique((inputs.uniform01(77, 20000) * mesh.shape[1]).astype(np.int64)))
        _HITS["mesh"] = np.ascontiguousarray(mesh[:, midx])
    b = (workloads.SCENES / f"{name}.sdfn").read_bytes()
    onet = oracle.Net(b)
    for label in ("hits", "mesh"):
        pts = _HITS[label]
        ref = onet.normal_map(pts.astype(np.float64))
        p999 = {}
        for prec in (sdf.SDF_FP16, sdf.SDF_BF16):
            out = sdf.normal_map(sdf.Net(b, prec), torch.from_numpy(pts).cuda()).cpu().numpy()
            sdf.sync_status()
            p999[prec] = angle_report(out, ref)["angle_p999"]
        print(name, label, "p99.9 deg: fp16", p999[sdf.SDF_FP16], "bf16", p999[sdf.SDF_BF16],
              "(bf16 within 0.5 deg)" if p999[sdf.SDF_BF16] <= 0.5 else "(bf16 above 0.5 deg)")
        assert p999[sdf.SDF_FP16] <= 0.1
        assert p999[sdf.SDF_BF16] <= 12.0 * p999[sdf.SDF_FP16]
        if name == "s8_256x3":
            assert p999[sdf.SDF_BF16] <= 0.5


@pytest.mark.parametrize("name", ["s8_256x3", "s8_256x2", "s8_128x2", "s8_256x1"])
def test_fp8_gradients_vs_oracle(sdf, name):
    """E4M3 hidden layers (kind::f8f6f4) against FP64: surface points of the displaced
    icosphere and uniform points of the box; the unnormalised gradient checks the scales."""
    b = (workloads.SCENES / f"{name}.sdfn").read_bytes()
    net = sdf.Net(b, sdf.SDF_FP8)
    surf, _ = workloads.mesh_points(subdivisions=5)
    box = inputs.random_points(7, 20000)
    onet = oracle.Net(b)
    for label, pts in (("surface", surf), ("box", box)):
        d = torch.from_numpy(pts).cuda()
        g = sdf.normals(net, d)
        nm = sdf.normal_map(net, d)
        sdf.sync_status()
        g, nm = g.cpu().numpy(), nm.cpu().numpy()
        ref = onet.grad_batch(pts.astype(np.float64))
        ar = angle_report(nm, ref)
        mag = np.abs(np.linalg.norm(g, axis=0) / np.linalg.norm(ref, axis=0) - 1.0)
        print(name, label, ar, "mag p99.9", float(np.quantile(mag, 0.999)))
        assert ar["angle_median"] <= FP8_ANGLE_MEDIAN_DEG
        if label == "surface":
            assert ar["angle_p999"] <= FP8_ANGLE_P999_DEG
            assert float(np.quantile(mag, 0.999)) <= FP8_MAGNITUDE_REL
        # normal_map is the normalised gradient of the same kernel
        assert np.allclose(nm, g / np.maximum(np.linalg.norm(g, axis=0), 1e-12), atol=1e-5)


def test_fp8_limits(sdf):
    """E4M3 covers the gradients of width 128 / 256 networks and tracing with width 256."""
    with pytest.raises(sdf.SdfError) as e:
        sdf.Net((workloads.SCENES / "s8_64x1.sdfn").read_bytes(), sdf.SDF_FP8)
    assert e.value.code == -7
    net = sdf.Net((workloads.SCENES / "s8_128x2.sdfn").read_bytes(), sdf.SDF_FP8)
    d = torch.zeros((3, 16), device="cuda")
    with pytest.raises(sdf.SdfError) as e:
        sdf.trace_multiscale([net], [0.0], [8], 1e-3, d, d)
    assert e.value.code == -7


def test_fp8_trace_plain_256x3(sdf):
    """The single-network (256,3) tracer with E4M3 hidden layers (kind::f8f6f4) against FP64, 120 x 68
    rays: the error is stated, not held to the 16-bit bounds (3 mantissa bits)."""
    wl = workloads.get("plain_256x3_1080p", 120, 68)
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, sdf.SDF_FP8, wl, orig, dirs)
    o = oracle_trace(lb, wl, orig, dirs)
    rep = trace_report(g["pos"], g["hit"], o["pos"], o["hit"])
    both = rep["both"]
    dist = np.linalg.norm(g["pos"][:, both].astype(np.float64) - o["pos"][:, both], axis=0)
    print("plain_256x3 e4m3", {k: v for k, v in rep.items() if k != "both"}, "median", float(np.median(dist)),
          "p99", float(np.quantile(dist, 0.99)))
    assert rep["n_both"] > 500
    assert rep["agree"] >= FP8_TRACE_AGREEMENT
    assert float(np.median(dist)) <= FP8_TRACE_POS_MEDIAN
    assert float(np.quantile(dist, 0.99)) <= FP8_TRACE_POS_P99


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_edge_cases(sdf):
    wl = workloads.get("random_siren_64x1")
    b = wl.level_bytes()[0]
    net = sdf.Net(b, sdf.SDF_BF16)
    # n = 0
    z = torch.empty((3, 0), device="cuda")
    sdf.trace_multiscale([net], [0.0], [32], 1e-3, z, z)
    sdf.normals(net, z)
    # host pointers are rejected before any launch
    host = torch.zeros((3, 4))
    with pytest.raises(sdf.SdfError) as e:
        sdf.normals(net, host, out=torch.zeros((3, 4)))
    assert e.value.code == -1
    # bad parameters
    d = torch.zeros((3, 4), device="cuda")
    with pytest.raises(sdf.SdfError):
        sdf.trace_multiscale([net], [0.0], [32], 0.0, d, d)
    with pytest.raises(sdf.SdfError):
        sdf.trace_multiscale([net, net], [-1.0, 0.0], [8, 8], 1e-3, d, d)
    # rays that miss the box, start inside it, or get zero iterations
    o = np.array([[0.0, 0.0, 5.0], [0.0, 0.0, 0.0], [0.3, 0.1, -0.2], [2.0, 2.0, 2.0]], np.float32).T.copy()
    v = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.6, 0.8], [1.0, 0.0, 0.0]], np.float32).T.copy()
    for caps in ([32], [0]):
        w2 = workloads.Workload("edge", [b], [0.0], caps, 1e-3, None, 0, 1, 1, b)
        g = gpu_trace(sdf, [b], 0, w2, o, v)
        r = oracle_trace([b], w2, o, v)
        assert np.array_equal(g["hit"], r["hit"])
        assert np.array_equal(g["iters"], r["iters"])
        assert np.allclose(g["pos"], r["pos"], atol=1e-5)
    assert g["hit"][0] == 0 and g["iters"][0] == 0  # misses the box: no evaluation
    sdf.sync_status()


def _degenerate_rays():
    """Unit rays that exercise every branch of the box-entry (slab) test of Alg. 1's ray setup."""
    rays = []
    for ax in range(3):  # along each axis, from outside, through the interior
        for s in (-1.0, 1.0):
            o, v = [0.1, -0.2, 0.3], [0.0, 0.0, 0.0]
            o[ax], v[ax] = -2.5 * s, s
            rays.append((o, v))
    for ax in range(3):  # parallel to a slab and outside it: a miss with no evaluation
        o, v = [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]
        o[ax], o[(ax + 1) % 3], v[(ax + 1) % 3] = 1.5, 2.5, -1.0
        rays.append((o, v))
    rays += [([1.0, 0.3, 2.5], [0.0, 0.0, -1.0]),     # parallel, on a face of the closed slab
             ([-1.0, 0.3, 2.5], [0.0, 0.0, -1.0]),
             ([1.0, 1.0, 2.5], [0.0, 0.0, -1.0]),      # parallel along an edge: enters at a corner
             ([0.2, 0.1, 1.0], [0.0, 0.0, -1.0]),      # starts on a face, pointing in
             ([0.0, 0.0, 0.95], [0.0, 0.0, 1.0]),      # starts inside, pointing out
             ([0.0, 0.0, 0.0], [0.6, 0.0, 0.8]),       # starts at the centre
             ([0.3, 0.2, 2.5], [1e-30, 1e-30, -1.0]),  # tiny normal components
             ([0.3, 0.2, 2.5], [1e-40, -1e-40, -1.0]),  # subnormal components: parallel to their slabs
             ([1.5, 0.2, 2.5], [1e-40, 0.0, -1.0])]    # subnormal and outside its slab: a miss
    o = np.array([r[0] for r in rays], np.float32).T.copy()
    v = np.array([r[1] for r in rays], np.float32).T.copy()
    ro, rv = inputs.random_rays(11, 64)  # oblique rays from every side
    return np.concatenate([o, ro], axis=1), np.concatenate([v, rv], axis=1)


@pytest.mark.parametrize("kernel", ["simt_fp32", "tc_w64_bf16", "tc_w128_bf16", "stream_w256_bf16"])
def test_box_entry_of_degenerate_rays(sdf, kernel):
    """A level with no iterations passes its rays on at their entry into the box, so the end points
    are the slab test's entry points (Alg. 1's ray setup): the FP64 oracle's to a few FP32 units in
    the last place of the entry distance (<= 5); rays that miss the box end at their origin with no
    evaluation and no hit, and with 32 iterations allowed they still take none."""
    width, n_hidden, precision = {"simt_fp32": (64, 1, sdf.SDF_FP32), "tc_w64_bf16": (64, 1, sdf.SDF_BF16),
                                  "tc_w128_bf16": (128, 2, sdf.SDF_BF16),
                                  "stream_w256_bf16": (256, 1, sdf.SDF_BF16)}[kernel]
    b = inputs.net_to_bytes(inputs.siren_init(4, width, n_hidden, out_shift=0.3))
    o, v = _degenerate_rays()
    w0 = workloads.Workload("entry", [b], [0.0], [0], 1e-3, None, 0, 1, 1, b)
    g = gpu_trace(sdf, [b], precision, w0, o, v)
    r = oracle_trace([b], w0, o, v)
    assert np.array_equal(g["iters"], r["iters"]) and not g["hit"].any() and not r["hit"].any()
    assert np.abs(g["pos"].astype(np.float64) - r["pos"]).max() <= 4e-6
    miss = np.all(r["pos"] == o.astype(np.float64), axis=0) & (np.abs(o).max(axis=0) > 1.0)
    assert miss.sum() >= 4  # the parallel and subnormal misses above
    assert np.array_equal(g["pos"][:, miss], o[:, miss])
    w32 = workloads.Workload("entry32", [b], [0.0], [32], 1e-3, None, 0, 1, 1, b)
    g32 = gpu_trace(sdf, [b], precision, w32, o, v)
    assert (g32["iters"][miss] == 0).all() and not g32["hit"][miss].any()
    assert np.array_equal(g32["pos"][:, miss], o[:, miss])


@pytest.mark.parametrize("memory", ["pinned", "pageable", "mixed"])
@pytest.mark.parametrize("size", [(160, 90), (640, 480), (1920, 1080)], ids=["1chunk", "2chunks", "4chunks"])
def test_render_host_matches_device(sdf, size, memory):
    """The host-buffer frame equals the device calls bit for bit: with page-locked buffers the kernels
    read the rays and write the normals in host memory directly; otherwise (pageable, or any one buffer
    pageable) the frame goes through the chunked copy pipeline."""
    wl = workloads.get("normal_map_1080p", *size)
    _render_host_vs_device(sdf, wl, memory)


@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_render_host_three_levels(sdf, memory):
    """Three levels through sdf_render_host: later levels re-read the directions through the ray queues."""
    _render_host_vs_device(sdf, workloads.get("three_level_512"), memory)


@pytest.mark.parametrize("precision", [0, 3], ids=["fp32", "fp16"])
def test_render_host_other_precisions(sdf, precision):
    """Page-locked host frames with the FP32 (SIMT) and FP16 kernels equal their device calls."""
    _render_host_vs_device(sdf, workloads.get("normal_map_1080p", 160, 90), "pinned", precision)


def _render_host_vs_device(sdf, wl, memory, precision=None):
    precision = sdf.SDF_BF16 if precision is None else precision
    orig, dirs = wl.rays()
    nets = [sdf.Net(b, precision) for b in wl.level_bytes()]
    fine = sdf.Net(wl.fine_bytes(), precision)
    n = orig.shape[1]
    pin = (lambda t: t.pin_memory()) if memory == "pinned" else (lambda t: t)
    hp = pin(torch.full((3, n), float("nan")))
    hh = pin(torch.full((n,), 7, dtype=torch.uint8))
    hn = torch.full((3, n), float("nan"))
    hn = hn if memory == "mixed" else pin(hn)
    ho = torch.from_numpy(orig)
    ho = ho.pin_memory() if memory in ("pinned", "mixed") else ho
    sdf.render_host(nets, wl.delta, wl.caps, wl.eps, fine, ho, pin(torch.from_numpy(dirs)), hp, hh, hn,
                    step_scale=wl.step_scale, final_mode=wl.final_mode)
    o = torch.from_numpy(orig).cuda()
    d = torch.from_numpy(dirs).cuda()
    pos, _, hit, _ = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, o, d, step_scale=wl.step_scale,
                                          final_mode=wl.final_mode)
    nrm = sdf.normal_map(fine, pos, hit)
    sdf.sync_status()
    assert torch.equal(hh, hit.cpu())
    assert torch.equal(hp, pos.cpu())
    assert torch.equal(hn, nrm.cpu())


def test_concurrent_streams_match_one_call(sdf):
    """Chunks of a frame traced and normal-mapped on two streams at once (each call with its own
    scratch from the library's pool) equal the single call bit for bit."""
    wl = workloads.get("normal_map_1080p", 640, 480)
    orig, dirs = wl.rays()
    nets = [sdf.Net(b, sdf.SDF_BF16) for b in wl.level_bytes()]
    fine = sdf.Net(wl.fine_bytes(), sdf.SDF_BF16)
    o = torch.from_numpy(orig).cuda()
    d = torch.from_numpy(dirs).cuda()
    kw = dict(step_scale=wl.step_scale, final_mode=wl.final_mode, want_iters=False)
    pos, _, hit, _ = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, o, d, **kw)
    nrm = sdf.normal_map(fine, pos, hit)
    n = orig.shape[1]
    cuts = [0, n // 3 + 5, 2 * n // 3 - 7, n]  # ragged chunks
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    chunks = [(o[:, a:b].contiguous(), d[:, a:b].contiguous()) for a, b in zip(cuts, cuts[1:])]
    start = torch.cuda.Event()
    start.record(main)
    outs = []
    for c, (oc, dc) in enumerate(chunks):
        s = streams[c % 2]
        s.wait_event(start)
        with torch.cuda.stream(s):
            pc, _, hc, _ = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, oc, dc, stream=s, **kw)
            outs.append((pc, hc, sdf.normal_map(fine, pc, hc, stream=s)))
    for s in streams:
        main.wait_stream(s)
    sdf.sync_status()
    assert torch.equal(torch.cat([x[0] for x in outs], 1), pos)
    assert torch.equal(torch.cat([x[1] for x in outs]), hit)
    assert torch.equal(torch.cat([x[2] for x in outs], 1), nrm)


def test_headline_bf16_frame_meets_the_stated_bounds(sdf):
    """The benchmark frame (BF16 coarse trace + BF16 (256,3) normal mapping, 1920 x 1080, full size)
    against the FP64 oracle on every 32nd image row (65,280 rays): hit/miss agreement >= 99.9 %,
    hit point <= 1e-3 and normal angle <= 0.5 deg at p99.9, the bounds stated for this frame rather
    than the precision-scaled BF16 bounds of the other tests."""
    wl = workloads.get("normal_map_1080p")
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, sdf.SDF_BF16, wl, orig, dirs)
    fine = sdf.Net(wl.fine_bytes(), sdf.SDF_BF16)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"]).cpu().numpy()
    sdf.sync_status()
    rows = np.arange(0, wl.height, 32)
    idx = (rows[:, None] * wl.width + np.arange(wl.width)[None, :]).ravel()
    o = oracle_trace(lb, wl, orig, dirs, idx=idx)
    rep = trace_report(g["pos"][:, idx], g["hit"][idx], o["pos"], o["hit"])
    print({k: v for k, v in rep.items() if k != "both"})
    assert rep["n_both"] > 10000
    assert rep["agree"] >= 0.999 and rep["pos_p999"] <= 1e-3
    hit = g["hit"][idx].astype(bool)
    ref = oracle.Net(wl.fine_bytes()).normal_map(g["pos"][:, idx].astype(np.float64), g["hit"][idx])
    ar = angle_report(nrm[:, idx], ref, hit)
    print(ar)
    assert ar["angle_p999"] <= 0.5


def test_headline_bf16_full_frame_against_the_oracle(sdf):
    """Every ray of the benchmark frame (2,073,600 rays: BF16 coarse trace + BF16 (256,3) normal mapping)
    against the FP64 oracle run on the whole frame: hit/miss agreement, hit point and normal angle at the
    same point over all common hits, with the bounds stated for this frame."""
    wl = workloads.get("normal_map_1080p")
    orig, dirs = wl.rays()
    lb = wl.level_bytes()
    g = gpu_trace(sdf, lb, sdf.SDF_BF16, wl, orig, dirs)
    fine = sdf.Net(wl.fine_bytes(), sdf.SDF_BF16)
    nrm = sdf.normal_map(fine, g["pos_dev"], g["hit_dev"]).cpu().numpy()
    sdf.sync_status()
    o = oracle_trace(lb, wl, orig, dirs)
    rep = trace_report(g["pos"], g["hit"], o["pos"], o["hit"])
    print({k: v for k, v in rep.items() if k != "both"})
    assert rep["n_both"] > 300000
    assert rep["agree"] >= 0.999 and rep["pos_p999"] <= 1e-3
    hit = g["hit"].astype(bool)
    ref = oracle.Net(wl.fine_bytes()).normal_map(g["pos"].astype(np.float64), g["hit"])
    ar = angle_report(nrm, ref, hit)
    print(ar)
    assert ar["angle_p999"] <= 0.5
