"""Benchmark: Mrays/s to hit + normal at 1920 x 1080.

One step renders one frame of the ``normal_map_1080p`` workload through the
C ABI: multiscale sphere tracing of the coarse (64,1) network until its
delta-shell (Alg. 1, BF16 tensor-core hidden layer) followed by neural normal
mapping of the fine (256,3) network at every hit (Sec. 5, Alg. 2 on the
tensor cores).  Inputs are resident in HBM; the L2 is flushed between timed
steps.  Also reported: the same frame end to end from host buffers (frames
back to back through a frame queue, and one sdf_render_host call per frame),
the plain FP32 (256,3) single-network tracer, the error
against the FP64 oracle on a sample of rays, and the oracle's own speed on the
host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Mrays/s to hit+normal at 1080p (multiscale BF16 vs plain FP32, same GPU, stated error)"
UNIT = "Mrays/s"
WORKLOAD = "normal_map_1080p"
ORACLE_ROW_STRIDE = 32  # the CPU-baseline sample: every 32nd image row
SCHEDULE_ROW_STRIDE = 32  # error of the 512 x 512 schedules against the oracle: every 32nd row
VARIANT_ROW_STRIDE = 64  # error of config 3's other readings (1080p) against the oracle: every 64th row
ANIM_SAMPLE = 256  # error of the animation batch: rays per frame (seeded), all 32 frames
MESH_SAMPLE = 3000  # error of the mesh normal mapping: vertices (seeded)
DECISION_MARGIN_BF16 = 5e-4  # value error of the BF16 path: decisions within it of eps are ambiguous


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_view(ws: int, rank: int):
    """The frame a rank renders in an N-GPU job (`--split frames`, weak scaling): view k = rank of an
    N-view orbit, camera eye 2.5 (sin a, 0, cos a) with a = 2 pi k / N, looking at the origin, up +y.
    View 0 is the headline camera (0, 0, 2.5).  Rays are independent (Alg. 1 per ray, Alg. 2 per
    point), so the ranks exchange nothing but the timing."""
    a = 2.0 * math.pi * rank / ws
    return rank, (2.5 * math.sin(a), 0.0, 2.5 * math.cos(a))


def row_band(height: int, ws: int, rank: int):
    """Rows [lo, hi) of one frame that a rank renders (`--split rows`, strong scaling): contiguous
    bands, the first height % ws ranks one row taller."""
    base, extra = divmod(height, ws)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_rays(wl, ws: int, rank: int, split: str):
    """(orig, dir) of this rank's share of the job and a description of the partition."""
    from paper_2201_09147_gb300 import inputs
    if split == "rows":
        lo, hi = row_band(wl.height, ws, rank)
        return (*inputs.camera_rays(wl.width, wl.height, rows=np.arange(lo, hi)),
                f"rows: rank r renders rows [r H/N, (r+1) H/N) of the {wl.width}x{wl.height} frame (strong)")
    _, eye = rank_view(ws, rank)
    return (*inputs.camera_rays(wl.width, wl.height, eye=eye),
            f"frames: rank r renders view r of an N-view orbit at {wl.width}x{wl.height} (weak; view 0 = the "
            "headline camera)")


def spawn_ranks(n: int) -> int:
    """Relaunches this command as n ranks on this node (torch.distributed.run, 127.0.0.1)."""
    port = 29400 + os.getpid() % 2000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}", "--master-addr",
           "127.0.0.1", "--master-port", str(port), str(Path(__file__).resolve()), *sys.argv[1:]]
    return subprocess.call(cmd)


def job_throughput(local_total_ms: float, units_per_rank: int, steps: int, ws: int, device="cpu"):
    """Whole-job throughput in millions of units per second: the units of all ranks over the
    slowest rank's timed region (max over ranks); returns (value, max_ms)."""
    t = float(local_total_ms)
    if ws > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return ws * units_per_rank * steps / (t / 1e3) / 1e6, t


def oracle_sample(wl, rows, threads=None):
    """Runs the FP64 oracle on the given image rows: trace + normal map at its hits."""
    import oracle
    orig, dirs = wl.rays(rows=rows)
    t0 = time.perf_counter()
    onets = [oracle.Net(b) for b in wl.level_bytes()]
    tp = oracle.TraceParams([oracle.SDF.of_net(n) for n in onets], wl.delta, wl.caps, wl.step_scale, wl.eps,
                            final_mode=wl.final_mode)
    res = tp.trace_batch(orig, dirs, threads=threads)
    fine = oracle.Net(wl.fine_bytes())
    nrm = fine.normal_map(res["pos"], res["hit"], threads=threads)
    dt = time.perf_counter() - t0
    return res, nrm, dt, orig.shape[1]


def _decisions(gh, oh, amb):
    una = ~amb
    return {"hit_agreement": float(np.mean(gh == oh)) if gh.size else None,
            "ambiguous_share": float(np.mean(amb)) if gh.size else None,
            "hit_agreement_unambiguous": float(np.mean(gh[una] == oh[una])) if una.any() else None}


def _q(x, q):
    return float(np.quantile(x, q)) if x.size else None


def _angles(gn, ref):
    """Angle in degrees between the columns of two (3, n) arrays (atan2 of |a x b| and a . b, which
    stays accurate near zero where arccos of the dot product does not)."""
    a, b = np.asarray(gn, np.float64), np.asarray(ref, np.float64)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(a.T, b.T), axis=1), np.sum(a * b, axis=0)))


def schedule_errors(samples):
    """Error of every timed schedule against the FP64 oracle on its sample: hit/miss agreement (all
    rays, and on the rays whose FP64 decision does not flip when eps moves by the BF16 value error),
    end-point distance on common hits, normal angle at the GPU's own end points."""
    import dataclasses

    import oracle
    out = {}
    for name in ("three_level_512", "silhouette_512", "normal_map_1080p_c64x2", "normal_map_1080p_zero"):
        if name not in samples:
            continue
        sm = samples[name]
        wl, orig, dirs = sm["wl"], *sm["orig"]
        lb = wl.level_bytes()

        def tr(eps):
            onets = [oracle.Net(b) for b in lb]
            tp = oracle.TraceParams([oracle.SDF.of_net(n) for n in onets], wl.delta, wl.caps, wl.step_scale, eps,
                                    final_mode=wl.final_mode)
            return tp.trace_batch(orig, dirs)

        o = tr(wl.eps)
        amb = tr(wl.eps - DECISION_MARGIN_BF16)["hit"] != tr(wl.eps + DECISION_MARGIN_BF16)["hit"]
        gh, oh = sm["hit"].astype(bool), o["hit"].astype(bool)
        both = gh & oh
        dp = np.linalg.norm(sm["pos"][:, both] - o["pos"][:, both], axis=0)
        ref = oracle.Net(wl.fine_bytes()).normal_map(sm["pos"].astype(np.float64), sm["hit"])
        ang = _angles(sm["normal"][:, gh], ref[:, gh])
        out[name] = {"rays": int(gh.size), "sample": sm.get("sample", f"every {SCHEDULE_ROW_STRIDE}th row"),
                     **_decisions(gh, oh, amb),
                     "hit_point_p999": _q(dp, 0.999), "hit_point_max": float(dp.max()) if dp.size else None,
                     "normal_deg_p999": _q(ang, 0.999), "normal_deg_max": float(ang.max()) if ang.size else None}
    for an in ("animation_32", "animation_32_pair", "animation_32_single"):
        if an not in samples:
            continue
        sm = samples[an]
        wa = sm["wl"]
        gh_all, oh_all, amb_all, dps, angs = [], [], [], [], []
        onets = [oracle.Net(b) for b in wa.level_bytes()]
        ofine = oracle.Net(wa.fine_bytes())
        from paper_2201_09147_gb300 import inputs as _inputs
        for fr in sm["frames"]:
            fw, fh = fr["size"]
            orig, dirs = _inputs.camera_rays(fw, fh)
            res = {}
            for key, eps in (("n", wa.eps), ("lo", wa.eps - DECISION_MARGIN_BF16), ("hi", wa.eps + DECISION_MARGIN_BF16)):
                tp = oracle.TraceParams([oracle.SDF.of_net(n, time=fr["time"]) for n in onets], wa.delta, wa.caps,
                                        wa.step_scale, eps, final_mode=wa.final_mode)
                res[key] = tp.trace_batch(orig, dirs, idx=fr["idx"])
            gh, oh = fr["hit"].astype(bool), res["n"]["hit"].astype(bool)
            both = gh & oh
            dps.append(np.linalg.norm(fr["pos"][:, both] - res["n"]["pos"][:, both], axis=0))
            ref = ofine.normal_map(fr["pos"].astype(np.float64), fr["hit"], time=fr["time"])
            angs.append(_angles(fr["normal"][:, gh], ref[:, gh]))
            gh_all.append(gh)
            oh_all.append(oh)
            amb_all.append(res["lo"]["hit"] != res["hi"]["hit"])
        gh, oh, amb = np.concatenate(gh_all), np.concatenate(oh_all), np.concatenate(amb_all)
        dp, ang = np.concatenate(dps), np.concatenate(angs)
        out[an] = {"rays": int(gh.size), "sample": f"{ANIM_SAMPLE} seeded rays of each of the 32 frames",
                               **_decisions(gh, oh, amb), "hit_point_p999": _q(dp, 0.999),
                               "hit_point_max": float(dp.max()) if dp.size else None,
                               "normal_deg_p999": _q(ang, 0.999), "normal_deg_max": float(ang.max()) if ang.size else None}
    if "mesh_normal_map" in samples:
        sm = samples["mesh_normal_map"]
        from paper_2201_09147_gb300 import workloads as _wl
        ref = oracle.Net(_wl.get("normal_map_1080p").fine_bytes()).normal_map(sm["pts"].astype(np.float64))
        ang = _angles(sm["normal"], ref)
        out["mesh_normal_map"] = {"vertices": int(ang.size), "sample": f"{MESH_SAMPLE} seeded vertices",
                                  "normal_deg_p999": _q(ang, 0.999), "normal_deg_median": _q(ang, 0.5),
                                  "normal_deg_max": float(ang.max()) if ang.size else None}
    return out


def reference_arm(args):
    """The FP64 oracle as the reference implementation, timed on the host cores."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    from paper_2201_09147_gb300 import workloads
    oracle.build()
    wl = workloads.get(WORKLOAD)
    rows = np.arange(0, wl.height, ORACLE_ROW_STRIDE * 2)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(wl, rows[:2])
    times, n = [], 0
    for _ in range(args.steps):
        _, _, dt, n = oracle_sample(wl, rows)
        times.append(dt)
    value = n * len(times) / sum(times) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_frame": wl.n_rays, "sample_rows_stride": ORACLE_ROW_STRIDE * 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
                             "sample": f"{n} rays per step (every {ORACLE_ROW_STRIDE * 2}th row of the 1080p frame)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def source_sha(path: Path) -> str:
    return hashlib.sha256(path.read_bytes()).hexdigest()[:16]


# the sources the inference kernels compile from: DRAM traffic measured by ncu is valid for these only
KERNEL_SOURCES = ["tc.cu", "grad_tc.cuh", "tc_common.cuh", "common.cuh", "rays.cuh", "internal.h"]


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update((ROOT / "paper_2201_09147_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def profile_train(points: int) -> int:
    """Lean run for ncu: two BF16 tensor-core fitting steps of the (256,3) network on `points` points."""
    import torch
    from paper_2201_09147_gb300 import build, inputs, sdfnn, workloads
    build.build()
    pts, tf, tg, near = (torch.from_numpy(x).cuda() for x in inputs.fit_batch(inputs.sphere_scene(1), 0, points))
    shape, theta = sdfnn.theta_from_sdfn((workloads.SCENES / "s8_256x3.sdfn").read_bytes())
    th = torch.from_numpy(theta).cuda()
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    ws = None
    for k in (1, 2):
        loss, ws = sdfnn.fit_step(shape, th, m, v, k, pts, tf, tg, near, lr=1e-5, workspace=ws,
                                  precision=sdfnn.SDF_BF16)
    sdfnn.sync_status()
    print(json.dumps({"profile_train": points, "objective": float(loss[3].item())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--split", default="frames", choices=["frames", "rows"],
                    help="N-GPU partition: each rank its own frame (weak) or a row band of one frame (strong)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="lean run for ncu: the timed steps only (no L2 flush buffer, no comparison legs)")
    ap.add_argument("--profile-normals", default="bf16", choices=["bf16", "fp16", "fp8"],
                    help="with --profile: operand type of the normal-mapping network")
    ap.add_argument("--profile-train", type=int, default=0, metavar="POINTS",
                    help="lean run for ncu: two BF16 fitting steps of the (256,3) on POINTS points, nothing else")
    args = ap.parse_args()
    if args.profile_train:
        return profile_train(args.profile_train)
    if args.profile:
        args.no_cpu_baseline = args.no_plain = True
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return spawn_ranks(args.gpus)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2201_09147_gb300 import build, sdfnn, workloads
    build.build()
    pk = peaks()

    wl = workloads.get(WORKLOAD)
    orig_h, dirs_h, partition = rank_rays(wl, ws, rank, args.split)
    n = orig_h.shape[1]
    orig = torch.from_numpy(orig_h).cuda()
    dirs = torch.from_numpy(dirs_h).cuda()
    coarse = [sdfnn.Net(b, sdfnn.SDF_BF16, local) for b in wl.level_bytes()]
    fine_prec = {"bf16": sdfnn.SDF_BF16, "fp16": sdfnn.SDF_FP16, "fp8": sdfnn.SDF_FP8}[args.profile_normals]
    if not args.profile:
        fine_prec = sdfnn.SDF_BF16
    fine = sdfnn.Net(wl.fine_bytes(), fine_prec, local)
    pos = torch.empty((3, n), device="cuda")
    tt = torch.empty(n, device="cuda")
    hit = torch.empty(n, dtype=torch.uint8, device="cuda")
    nrm = torch.empty((3, n), device="cuda")
    # writing 512 MB between timed steps evicts the 129 MB L2
    flush = torch.empty((1 if args.profile else 512 * 1024 * 1024 // 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        sdfnn.trace_multiscale(coarse, wl.delta, wl.caps, wl.eps, orig, dirs, step_scale=wl.step_scale,
                               final_mode=wl.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
        ev_mid = torch.cuda.Event(enable_timing=True)
        ev_mid.record(stream)
        sdfnn.normal_map(fine, pos, hit, out=nrm)
        return ev_mid

    for _ in range(args.warmup):
        step()
        flush.zero_()
    sdfnn.sync_status()

    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    evs = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        em = step()
        e1.record(stream)
        evs.append((e0, em, e1))
        flush.zero_()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    sdfnn.sync_status()
    step_ms = [a.elapsed_time(c) for a, _, c in evs]
    trace_ms = [a.elapsed_time(b) for a, b, _ in evs]
    nmap_ms = [b.elapsed_time(c) for _, b, c in evs]
    value, total_ms = job_throughput(sum(step_ms), n, args.steps, ws, "cuda")
    median_value, _ = job_throughput(statistics.median(step_ms) * args.steps, n, args.steps, ws, "cuda")
    n_hit = int(hit.sum().item())

    # roofline of the dominant kernel (algorithmic work / event-timed duration)
    W, KH = fine.width, fine.n_hidden
    normal_flops_per_point = 4 * KH * 2 * W * W          # forward + 3 tangents through the hidden layers
    nm_ms = statistics.mean(nmap_ms)
    tr_ms = statistics.mean(trace_ms)
    # iteration histogram for the trace's algorithmic work (one extra untimed run)
    _, _, _, iters = sdfnn.trace_multiscale(coarse, wl.delta, wl.caps, wl.eps, orig, dirs,
                                            step_scale=wl.step_scale, final_mode=wl.final_mode)
    torch.cuda.synchronize()
    total_evals = int(iters.to(torch.int64).sum().item())
    cw, ck = coarse[0].width, coarse[0].n_hidden
    sines_per_eval = (ck + 1) * cw
    # DRAM bytes per launch from the committed ncu launch list, valid only for the kernel source it was taken on
    traffic_path = ROOT / "profiles" / "traffic.json"
    traffic_tbl = {}
    if traffic_path.exists():
        tj = json.loads(traffic_path.read_text())
        if tj.get("source_sha") == kernel_sources_sha():
            traffic_tbl = tj.get("bytes_per_launch", {})
    # the normal-mapping kernel against the tensor roof (reported for both kernels; the
    # dominant one is `roofline`)
    nm_achieved = n_hit * normal_flops_per_point / (nm_ms / 1e3) / 1e12
    nm_peak = pk["bf16_tflops_sustained"]
    roofline_nm = {"kernel": "grad_tc_kernel<256> (neural normal mapping, (256,3))", "bound": "tensor",
                   "achieved": nm_achieved, "peak": nm_peak, "unit": "TFLOP/s", "frac": nm_achieved / nm_peak,
                   "traffic": traffic_tbl.get("grad_tc_kernel<256, 0, 0>"),
                   "peak_source": f"{pk['source']} bf16 sustained",
                   "work": f"{n_hit} points x {normal_flops_per_point} hidden-layer MMA flops"}
    if nm_ms >= tr_ms:
        roofline = roofline_nm
    else:
        # sine-bound: one hardware sine per unit per evaluation; the roof is the measured
        # rate of the same sine (independent chains on all SMs)
        sm_mhz = clk.get("sm_mhz") or 1900.0
        nominal_gsin = 152 * 16 * sm_mhz * 1e6 / 1e9
        peak_gsin = sdfnn.measure_sine_rate(local) / 1e9
        achieved = total_evals * sines_per_eval / (tr_ms / 1e3) / 1e9
        roofline = {"kernel": "trace_level_tc_kernel<64> (coarse (64,1) trace)", "bound": "alu", "achieved": achieved,
                    "peak": peak_gsin, "unit": "Gsin/s", "frac": achieved / peak_gsin,
                    "traffic": traffic_tbl.get("trace_level_tc_kernel<64, 0, 1>"),
                    "peak_source": "measured: sine microbenchmark (sdf_measure_sine_rate), "
                                   f"nominal 152 SMs x 16 per clock = {nominal_gsin:.0f} Gsin/s",
                    "work": f"{total_evals} evaluations x {sines_per_eval} sines"}

    # end to end from pinned host buffers through sdf_render_host
    e2e_value = None
    if not args.profile:
        ho = torch.from_numpy(orig_h).pin_memory()
        hd = torch.from_numpy(dirs_h).pin_memory()
        hp = torch.empty((3, n)).pin_memory()
        hh = torch.empty(n, dtype=torch.uint8).pin_memory()
        hn = torch.empty((3, n)).pin_memory()

        def e2e_step():
            sdfnn.render_host(coarse, wl.delta, wl.caps, wl.eps, fine, ho, hd, hp, hh, hn,
                              step_scale=wl.step_scale, final_mode=wl.final_mode)

        e2e_step()
        e2e_times = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            e2e_times.append(time.perf_counter() - t0)
        e2e_call_value, _ = job_throughput(1e3 * sum(e2e_times), n, len(e2e_times), ws, "cuda")
        # frames back to back through a frame queue (three frames in flight): each frame's rays are
        # copied in and its end points, hit flags and normals copied out while its neighbours'
        # kernels run; host wall clock from the first submission until the last frame's results
        # are in host memory
        q_depth = 3
        queue = sdfnn.FrameQueue(coarse, wl.delta, wl.caps, wl.eps, fine, n, depth=q_depth,
                                 step_scale=wl.step_scale, final_mode=wl.final_mode)
        qouts = [(torch.empty((3, n)).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory(),
                  torch.empty((3, n)).pin_memory()) for _ in range(q_depth)]
        for k in range(max(3, args.warmup)):
            queue.submit(ho, hd, *qouts[k % q_depth])
        queue.wait()
        q_frames = max(10, args.steps // 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(q_frames):
            queue.submit(ho, hd, *qouts[k % q_depth])
        queue.wait()
        q_dt = time.perf_counter() - t0
        queue.close()
        e2e_value, _ = job_throughput(1e3 * q_dt, n, q_frames, ws, "cuda")

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
              "ms_per_step_median": statistics.median(step_ms), "value_from_median_step": median_value,
              "higher_is_better": True,
              "scaling": "strong" if args.split == "rows" else "weak", "vs_baseline": None, "dtype": "bf16",
              "data": "synthetic",
              "config": {"workload": WORKLOAD, "rays_per_rank": n, "resolution": [wl.width, wl.height],
                         "coarse": "(64,1) BF16, final_mode 1, delta_0 0.04, cap 40",
                         "fine": "(256,3) BF16 normal mapping", "l2": "flushed between steps (512 MB write)",
                         "parallelism": f"{args.split} x{ws}", "partition": partition},
              "clocks": clk, "gpu_launches": 3 * args.steps,
              "e2e": ({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 3 * 4 * n,
                       "d2h_bytes_per_step": (3 + 3) * 4 * n + n,
                       "api": "sdf_frame_queue (three frames in flight, alternating two compute streams)",
                       "transfer": "pinned host buffers: every frame's rays copied in and its end points, hit "
                                   "flags and normals copied out by the queue's copy streams while the "
                                   "neighbouring frames' kernels run (no L2 flush: each frame's rays arrive "
                                   "by copy from host memory)",
                       "timer": f"host wall clock from the first of {q_frames} submissions until the last "
                                "frame's results are in host memory",
                       "per_call": {"value": e2e_call_value, "unit": UNIT, "api": "sdf_render_host",
                                    "transfer": "pinned host buffers: the trace kernel reads the rays and the "
                                                "normal-mapping kernel writes the hits' normals in host memory "
                                                "over NVLink-C2C; the copy engine clears the host normals during "
                                                "the trace and copies the end points and hit flags back during "
                                                "the normal mapping",
                                    "timer": "host wall clock around each sdf_render_host call (returns "
                                             "synchronised), L2 flushed before each"}}
                      if e2e_value is not None else None),
              "roofline": roofline,
              "roofline_normal_map": roofline_nm,
              "breakdown_ms": {"trace_coarse": tr_ms, "normal_map_fine": nm_ms, "hits": n_hit,
                               "mean_coarse_iters": total_evals / n},
              "wall_s_timed_region": t_wall}

    samples = {}  # sampled GPU outputs of the comparison legs, checked against the oracle at the end
    if not args.no_plain:
        # plain FP32 single-network (256,3) tracer with its own normals: the comparison path
        plain = workloads.get("plain_256x3_1080p")
        pn = [sdfnn.Net(b, sdfnn.SDF_FP32, local) for b in plain.level_bytes()]
        pf = sdfnn.Net(plain.fine_bytes(), sdfnn.SDF_FP32, local)

        def plain_step():
            sdfnn.trace_multiscale(pn, plain.delta, plain.caps, plain.eps, orig, dirs, step_scale=plain.step_scale,
                                   final_mode=plain.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            sdfnn.normal_map(pf, pos, hit, out=nrm)

        plain_step()
        torch.cuda.synchronize()
        pt = []
        for _ in range(2):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plain_step()
            b.record(stream)
            torch.cuda.synchronize()
            pt.append(a.elapsed_time(b))
        plain_value = n / (statistics.mean(pt) / 1e3) / 1e6
        # the same plain (256,3) tracer with BF16 hidden layers: the precision alone
        pb = [sdfnn.Net(b, sdfnn.SDF_BF16, local) for b in plain.level_bytes()]
        pbf = sdfnn.Net(plain.fine_bytes(), sdfnn.SDF_BF16, local)
        bt = []
        for _ in range(4):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sdfnn.trace_multiscale(pb, plain.delta, plain.caps, plain.eps, orig, dirs, step_scale=plain.step_scale,
                                   final_mode=plain.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            sdfnn.normal_map(pbf, pos, hit, out=nrm)
            b.record(stream)
            torch.cuda.synchronize()
            bt.append(a.elapsed_time(b))
        plain_bf16_value = n / (statistics.mean(bt[1:]) / 1e3) / 1e6
        # the plain (256,3) trace with E4M3 hidden layers (its normals E4M3 too)
        p8 = [sdfnn.Net(b, sdfnn.SDF_FP8, local) for b in plain.level_bytes()]
        p8f = sdfnn.Net(plain.fine_bytes(), sdfnn.SDF_FP8, local)
        et8 = []
        for _ in range(4):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sdfnn.trace_multiscale(p8, plain.delta, plain.caps, plain.eps, orig, dirs, step_scale=plain.step_scale,
                                   final_mode=plain.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            sdfnn.normal_map(p8f, pos, hit, out=nrm)
            b.record(stream)
            torch.cuda.synchronize()
            et8.append(a.elapsed_time(b))
        plain_fp8_value = n / (statistics.mean(et8[1:]) / 1e3) / 1e6
        # multiscale with FP32 hidden layers: isolates the algorithm from the precision
        c32 = [sdfnn.Net(b, sdfnn.SDF_FP32, local) for b in wl.level_bytes()]
        f32 = sdfnn.Net(wl.fine_bytes(), sdfnn.SDF_FP32, local)
        ft = []
        for _ in range(3):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sdfnn.trace_multiscale(c32, wl.delta, wl.caps, wl.eps, orig, dirs, step_scale=wl.step_scale,
                                   final_mode=wl.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            sdfnn.normal_map(f32, pos, hit, out=nrm)
            b.record(stream)
            torch.cuda.synchronize()
            ft.append(a.elapsed_time(b))
        ms_fp32_value = n / (statistics.mean(ft[1:]) / 1e3) / 1e6
        # the same frame with FP16 tensor-core operands
        c16 = [sdfnn.Net(b, sdfnn.SDF_FP16, local) for b in wl.level_bytes()]
        f16 = sdfnn.Net(wl.fine_bytes(), sdfnn.SDF_FP16, local)
        ht = []
        for _ in range(args.warmup + args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sdfnn.trace_multiscale(c16, wl.delta, wl.caps, wl.eps, orig, dirs, step_scale=wl.step_scale,
                                   final_mode=wl.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            sdfnn.normal_map(f16, pos, hit, out=nrm)
            b.record(stream)
            ht.append((a, b))
        torch.cuda.synchronize()
        fp16_value = n / (statistics.mean([a.elapsed_time(b) for a, b in ht[args.warmup:]]) / 1e3) / 1e6
        # BF16 coarse trace with E4M3 normal mapping (kind::f8f6f4 gradient kernel)
        f8 = sdfnn.Net(wl.fine_bytes(), sdfnn.SDF_FP8, local)
        et = []
        for _ in range(args.warmup + args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            m = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sdfnn.trace_multiscale(coarse, wl.delta, wl.caps, wl.eps, orig, dirs, step_scale=wl.step_scale,
                                   final_mode=wl.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            m.record(stream)
            sdfnn.normal_map(f8, pos, hit, out=nrm)
            b.record(stream)
            et.append((a, m, b))
        torch.cuda.synchronize()
        fp8_value = n / (statistics.mean([a.elapsed_time(b) for a, _, b in et[args.warmup:]]) / 1e3) / 1e6
        fp8_nm_ms = statistics.mean([m.elapsed_time(b) for _, m, b in et[args.warmup:]])
        result["comparisons"] = {"fp16_Mrays_s": fp16_value,
                                 "fp8_normal_map_Mrays_s": fp8_value,
                                 "fp8_normal_map_ms": fp8_nm_ms,
                                 "plain_fp32_256x3_Mrays_s": plain_value,
                                 "plain_bf16_256x3_Mrays_s": plain_bf16_value,
                                 "plain_fp8_256x3_Mrays_s": plain_fp8_value,
                                 "speedup_precision_only_plain": plain_bf16_value / plain_value,
                                 "speedup_vs_plain_fp32": value / ws / plain_value,
                                 "multiscale_fp32_Mrays_s": ms_fp32_value,
                                 "speedup_algorithm_only": ms_fp32_value / plain_value,
                                 "speedup_precision_only_multiscale": value / ws / ms_fp32_value}
        sdfnn.sync_status()

        def timed_ms(fn, reps=5):
            fn()
            out = []
            for _ in range(reps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                out.append(a.elapsed_time(b))
            return statistics.median(out)

        # three-level normal mapping (the last row of Tab. 3) and its silhouette variant, 512 x 512, BF16
        for name in ("three_level_512", "silhouette_512"):
            w3 = workloads.get(name)
            o3, d3 = (torch.from_numpy(x).cuda() for x in w3.rays())
            n3 = [sdfnn.Net(b, sdfnn.SDF_BF16, local) for b in w3.level_bytes()]
            f3 = sdfnn.Net(w3.fine_bytes(), sdfnn.SDF_BF16, local)
            plan3 = sdfnn.Plan(n3, w3.delta, w3.caps, w3.eps, o3, d3, fine=f3, step_scale=w3.step_scale,
                               final_mode=w3.final_mode, autotune=True, want_iters=False)
            ms3 = timed_ms(plan3.launch, 20)
            result["comparisons"][f"{name}_Mrays_s"] = w3.n_rays / (ms3 / 1e3) / 1e6
            result["comparisons"][f"{name}_hits"] = int(plan3.hit.sum().item())
            rows3 = np.arange(0, w3.height, SCHEDULE_ROW_STRIDE)
            i3 = (rows3[:, None] * w3.width + np.arange(w3.width)[None, :]).ravel()
            samples[name] = {"wl": w3, "idx": i3, "pos": plan3.pos.cpu().numpy()[:, i3],
                             "hit": plan3.hit.cpu().numpy()[i3], "normal": plan3.normal.cpu().numpy()[:, i3],
                             "orig": w3.rays(rows=rows3)}
            plan3.close()

        # config 3's other readings of "coarse 64-wide net" and of the end condition: the (64,2) of the
        # nested sequence as the coarse net, and the (64,1) traced to its zero set; (256,3) normals, BF16
        for name in ("normal_map_1080p_c64x2", "normal_map_1080p_zero"):
            wv = workloads.get(name)
            cv = [sdfnn.Net(b, sdfnn.SDF_BF16, local) for b in wv.level_bytes()]

            def vstep(wv=wv, cv=cv):
                sdfnn.trace_multiscale(cv, wv.delta, wv.caps, wv.eps, orig, dirs, step_scale=wv.step_scale,
                                       final_mode=wv.final_mode, out_pos=pos, out_t=tt, out_hit=hit,
                                       want_iters=False)
                sdfnn.normal_map(fine, pos, hit, out=nrm)

            msv = timed_ms(vstep, 10)
            vstep()
            sdfnn.sync_status()
            result["comparisons"][f"{name}_Mrays_s"] = n / (msv / 1e3) / 1e6
            result["comparisons"][f"{name}_hits"] = int(hit.sum().item())
            if args.split == "frames":
                rows_v = np.arange(0, wl.height, VARIANT_ROW_STRIDE)
                iv = (rows_v[:, None] * wl.width + np.arange(wl.width)[None, :]).ravel()
                samples[name] = {"wl": wv, "idx": iv, "pos": pos.cpu().numpy()[:, iv], "hit": hit.cpu().numpy()[iv],
                                 "normal": nrm.cpu().numpy()[:, iv],
                                 "orig": (np.ascontiguousarray(orig_h[:, iv]), np.ascontiguousarray(dirs_h[:, iv])),
                                 "sample": f"every {VARIANT_ROW_STRIDE}th row of the 1080p frame"}

        # neural normal mapping onto the full-size mesh (displaced icosphere, subdivision 7), BF16
        mesh_h, _ = workloads.mesh_points(7)
        mesh = torch.from_numpy(mesh_h).cuda()
        mesh_out = torch.empty_like(mesh)
        ms_mesh = timed_ms(lambda: sdfnn.normal_map(fine, mesh, out=mesh_out), 20)
        result["comparisons"]["mesh_normal_map"] = {"vertices": int(mesh.shape[1]), "ms": ms_mesh,
                                                    "Mvertices_s": mesh.shape[1] / (ms_mesh / 1e3) / 1e6,
                                                    "net": "(256,3) BF16"}
        from paper_2201_09147_gb300 import inputs as _inputs
        im = np.sort(np.unique((_inputs.uniform01(77, MESH_SAMPLE) * mesh_h.shape[1]).astype(np.int64)))
        samples["mesh_normal_map"] = {"pts": mesh_h[:, im], "normal": mesh_out.cpu().numpy()[:, im]}
        del mesh, mesh_out

        # 32 animated frames of mixed sizes (8 x 256^2, 16 x 1280x720, 8 x 1920x1080): one autotuned
        # plan (CUDA graph) per schedule; the first against per-frame calls
        from paper_2201_09147_gb300 import inputs as _inputs
        for an in ("animation_32", "animation_32_pair", "animation_32_single"):
            wa = workloads.get(an)
            if not all((workloads.SCENES / f).exists() for f in wa.levels + [wa.fine]):
                continue
            oa_h, da_h, ta_h, off = workloads.batch_rays(wa.frames)
            oa, da, ta = (torch.from_numpy(x).cuda() for x in (oa_h, da_h, ta_h))
            del oa_h, da_h
            na = [sdfnn.Net(b, sdfnn.SDF_BF16, local) for b in wa.level_bytes()]
            fa = sdfnn.Net(wa.fine_bytes(), sdfnn.SDF_BF16, local)
            plan_a = sdfnn.Plan(na, wa.delta, wa.caps, wa.eps, oa, da, fine=fa, ray_time=ta,
                                step_scale=wa.step_scale, final_mode=wa.final_mode, autotune=True, want_iters=False)
            ms_plan = timed_ms(plan_a.launch, 5)
            tiles, nodes = plan_a.info()
            n_hits_a = int(plan_a.hit.sum().item())
            # ANIM_SAMPLE rays of every frame (seeded), for the error against the oracle
            a_pos, a_hit, a_nrm = plan_a.pos.cpu().numpy(), plan_a.hit.cpu().numpy(), plan_a.normal.cpu().numpy()
            a_frames = []
            for k, (fw, fh, tk) in enumerate(wa.frames):
                lo_ = int(off[k])
                fi = np.sort(np.unique((_inputs.uniform01(500 + k, ANIM_SAMPLE) * fw * fh).astype(np.int64)))
                a_frames.append({"size": (fw, fh), "time": float(tk), "idx": fi, "pos": a_pos[:, lo_ + fi],
                                 "hit": a_hit[lo_ + fi], "normal": a_nrm[:, lo_ + fi]})
            samples[an] = {"wl": wa, "frames": a_frames}
            del a_pos, a_hit, a_nrm
            plan_a.close()
            entry = {"rays": wa.n_rays, "frames": "8 x 256^2, 16 x 1280x720, 8 x 1920x1080, t_k = k/31",
                     "levels": [f"{x} (delta {d}, cap {c})" for x, d, c in zip(wa.levels, wa.delta, wa.caps)],
                     "normals": wa.fine, "final_mode": wa.final_mode,
                     "plan_Mrays_s": wa.n_rays / (ms_plan / 1e3) / 1e6, "plan_ms": ms_plan,
                     "autotuned_tiles": tiles, "graph_nodes": nodes, "hits": n_hits_a}
            if an == "animation_32":
                frames = []
                for k, (fw, fh, tk) in enumerate(wa.frames):
                    lo, hi = int(off[k]), int(off[k + 1])
                    frames.append((oa[:, lo:hi].contiguous(), da[:, lo:hi].contiguous(), float(tk)))

                def per_frame():
                    for fo, fd, tk in frames:
                        p_, _, h_, _ = sdfnn.trace_multiscale(na, wa.delta, wa.caps, wa.eps, fo, fd,
                                                              step_scale=wa.step_scale, final_mode=wa.final_mode,
                                                              time=tk, want_iters=False)
                        fa.set_time(tk)
                        sdfnn.normal_map(fa, p_, h_)

                ms_frames = timed_ms(per_frame, 3)
                entry["per_frame_calls_Mrays_s"] = wa.n_rays / (ms_frames / 1e3) / 1e6
                entry["per_frame_calls_ms"] = ms_frames
                del frames
            result["comparisons"][an] = entry
            del oa, da, ta
            sdfnn.sync_status()

        # native fitting steps on 2^20 points (forward with tangents, objective, backward, Adam):
        # the 3-net nested sequence with BF16 tensor-core contractions (config 5), and the (256,3)
        # with BF16 and with FP32 CUDA-core contractions
        fp, ftf, ftg, fnear = (torch.from_numpy(x).cuda()
                               for x in _inputs.fit_batch(_inputs.sphere_scene(1), 0, 1 << 20))

        def fit_ms_of(name, prec):
            shape, theta_h = sdfnn.theta_from_sdfn((workloads.SCENES / f"{name}.sdfn").read_bytes())
            th = torch.from_numpy(theta_h).cuda()
            m_, v_ = torch.zeros_like(th), torch.zeros_like(th)
            loss_, ws_ = sdfnn.fit_step(shape, th, m_, v_, 1, fp, ftf, ftg, fnear, lr=1e-5, precision=prec)
            torch.cuda.synchronize()
            out = []
            for k in range(2, 6):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                loss_, ws_ = sdfnn.fit_step(shape, th, m_, v_, k, fp, ftf, ftg, fnear, lr=1e-5, workspace=ws_,
                                            precision=prec)
                b.record(stream)
                torch.cuda.synchronize()
                out.append(a.elapsed_time(b))
            sdfnn.sync_status()
            ws_gb = ws_.numel() / 1e9
            del ws_
            torch.cuda.empty_cache()
            return statistics.median(out), float(loss_[3].item()), ws_gb

        seq = {}
        for name in ("s8_64x2", "s8_128x2", "s8_256x2"):
            ms_, obj_, gb_ = fit_ms_of(name, sdfnn.SDF_BF16)
            seq[name] = {"ms_per_step": ms_, "objective": obj_, "workspace_GB": gb_}
        bf_ms, bf_obj, bf_gb = fit_ms_of("s8_256x3", sdfnn.SDF_BF16)
        f32_ms, f32_obj, f32_gb = fit_ms_of("s8_256x3", sdfnn.SDF_FP32)
        seq_ms = sum(v["ms_per_step"] for v in seq.values())
        result["comparisons"]["fit_step_nested_sequence_2^20"] = {
            "nets": seq, "ms_per_step": seq_ms, "points_per_s": (1 << 20) / (seq_ms / 1e3),
            "kernels": "BF16 tcgen05: forward + tangents, backward-data, weight gradients; FP32 objective and Adam"}
        result["comparisons"]["fit_step_256x3_2^20"] = {
            "bf16_tensor_core": {"ms_per_step": bf_ms, "objective": bf_obj, "workspace_GB": bf_gb},
            "fp32_cuda_core": {"ms_per_step": f32_ms, "objective": f32_obj, "workspace_GB": f32_gb},
            "speedup": f32_ms / bf_ms}
        del fp, ftf, ftg, fnear
        sdfnn.sync_status()

    if rank == 0 and not args.no_cpu_baseline:
        # FP64 oracle on a bounded sample of the same frame: speed, and the error of this run
        rows = np.arange(0, wl.height, ORACLE_ROW_STRIDE)
        res, onrm, dt, ns = oracle_sample(wl, rows)
        import oracle
        # one core, on a 16x smaller sample
        _, _, dt1, ns1 = oracle_sample(wl, rows[::16], threads=1)
        result["cpu_baseline"] = {"value": ns / dt / 1e6, "unit": UNIT, "cores": oracle.default_threads(),
                                  "kind": "oracle",
                                  "sample": f"{ns} rays: every {ORACLE_ROW_STRIDE}th row of the 1080p frame, "
                                            f"trace + normal map in FP64",
                                  "one_core": {"value": ns1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                                               "sample": f"{ns1} rays: every {16 * ORACLE_ROW_STRIDE}th row"}}
        idx = (rows[:, None] * wl.width + np.arange(wl.width)[None, :]).ravel()
        fine_oracle = oracle.Net(wl.fine_bytes())

        def error_of(cnets, fnet, qfmt=None):
            sdfnn.trace_multiscale(cnets, wl.delta, wl.caps, wl.eps, orig, dirs, step_scale=wl.step_scale,
                                   final_mode=wl.final_mode, out_pos=pos, out_t=tt, out_hit=hit, want_iters=False)
            sdfnn.normal_map(fnet, pos, hit, out=nrm)
            sdfnn.sync_status()
            gp = pos.cpu().numpy()[:, idx]
            gh = hit.cpu().numpy()[idx].astype(bool)
            gn = nrm.cpu().numpy()[:, idx]
            oh = res["hit"].astype(bool)
            both = gh & oh
            dp = np.linalg.norm(gp[:, both] - res["pos"][:, both], axis=0)
            ref = fine_oracle.normal_map(gp.astype(np.float64), gh.astype(np.uint8))
            ang = _angles(gn[:, gh], ref[:, gh])
            out = {"rays": int(idx.size), "hits": int(gh.sum()), "hit_agreement": float(np.mean(gh == oh)),
                   "hit_point_p999": float(np.quantile(dp, 0.999)) if dp.size else None,
                   "hit_point_max": float(dp.max()) if dp.size else None,
                   "normal_deg_p999": float(np.quantile(ang, 0.999)) if ang.size else None,
                   "normal_deg_max": float(ang.max()) if ang.size else None,
                   # hits where |grad f| < 1e-12 get (0, 0, 0): counted, and part of the angles above
                   "zero_normals": int((np.linalg.norm(gn[:, gh], axis=0) == 0.0).sum())}
            # FP64 residual of the GPU's end points against the level set the last level traces
            d_last = wl.delta[-1] if wl.final_mode == 1 else 0.0
            lvl = np.abs(oracle.eval_batch(wl.level_bytes()[-1], gp[:, gh].astype(np.float64)) - d_last)
            out["end_residual_p999"] = _q(lvl, 0.999)
            out["end_residual_max"] = float(lvl.max()) if lvl.size else None
            # end to end: the GPU normal at its end point against the FP64 normal at the oracle's
            ang_e2e = _angles(gn[:, both], onrm[:, both])
            out["normal_deg_end_to_end_p999"] = _q(ang_e2e, 0.999)
            out["normal_deg_end_to_end_max"] = float(ang_e2e.max()) if ang_e2e.size else None
            if qfmt:
                # the oracle on the 16-bit hidden weights the kernel multiplies with: the angle from
                # the exact FP64 normals is the weight rounding alone, the angle to the GPU's the
                # arithmetic (16-bit activations and tangents, FP32 accumulation, hardware sine)
                qref = oracle.Net(oracle.quantised_image(wl.fine_bytes(), qfmt)).normal_map(
                    gp.astype(np.float64), gh.astype(np.uint8))
                aq, ag = _angles(qref[:, gh], ref[:, gh]), _angles(gn[:, gh], qref[:, gh])
                out["split_vs_oracle_on_16bit_weights"] = {
                    "weights": qfmt, "weight_rounding_deg_p999": _q(aq, 0.999), "weight_rounding_deg_median": _q(aq, 0.5),
                    "arithmetic_deg_p999": _q(ag, 0.999), "arithmetic_deg_median": _q(ag, 0.5)}
            return out

        if args.split == "frames":  # rank 0 renders the headline frame itself
            result["error_vs_oracle"] = error_of(coarse, fine, "bf16")
            if not args.no_plain:
                result["error_vs_oracle_fp16"] = error_of(c16, f16, "f16")
                result["error_vs_oracle_fp8_normal_map"] = error_of(coarse, f8)
        if not args.no_plain:
            result["error_vs_oracle_schedules"] = schedule_errors(samples)
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
