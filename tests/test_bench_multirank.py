"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1).

Each rank renders its own share of the job (its own view of an N-view orbit,
or a row band of one frame); the job value is all ranks' units over the
slowest rank's time, and every rank agrees on it.  The shares cover the job
exactly once.  The reference arm runs on rank 0 only."""
import io
import json
import os
import sys
from contextlib import redirect_stdout
from pathlib import Path

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import bench
    import numpy as np

    from paper_2201_09147_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        value, max_ms = bench.job_throughput(local_ms, 2_000_000, 10, ws)
        # the shares of a small frame, gathered: views (weak) and row bands (strong)
        wl = workloads.get("normal_map_1080p", 48, 27)
        shares = {}
        for split in ("frames", "rows"):
            o, d, _ = bench.rank_rays(wl, ws, rank, split)
            got = [None] * ws
            dist.all_gather_object(got, (rank, o.tobytes(), d.tobytes(), o.shape[1]))
            shares[split] = got
        out.put((rank, value, max_ms, bench.dist_info(), shares))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, m0, d0, s0), (r1, v1, m1, d1, s1) = res
    assert m0 == m1 == 150.0                      # max over ranks
    assert v0 == v1 == pytest.approx(2 * 2_000_000 * 10 / 0.150 / 1e6)
    assert d0 == (2, 0, 0) and d1 == (2, 1, 1)
    import numpy as np

    from paper_2201_09147_gb300 import inputs
    w, h = 48, 27
    # frames: rank 0 renders the single-GPU frame itself, rank 1 another view; both full frames
    full_o, full_d = inputs.camera_rays(w, h)
    f = s0["frames"]
    assert f == s1["frames"] and [x[0] for x in f] == [0, 1]
    assert f[0][1] == full_o.tobytes() and f[0][2] == full_d.tobytes()
    assert f[1][3] == f[0][3] == w * h and f[1][2] != f[0][2]
    # rows: the two bands, in rank order, are the frame's rays exactly once
    r = s0["rows"]
    assert r == s1["rows"] and sum(x[3] for x in r) == w * h
    cat_d = np.concatenate([np.frombuffer(x[2], np.float32).reshape(3, -1) for x in r], axis=1)
    assert cat_d.tobytes() == full_d.tobytes()


def test_row_bands_cover_every_row_once():
    sys.path.insert(0, str(ROOT))
    import bench
    for height in (1, 7, 27, 1080):
        for ws in (1, 2, 3, 8):
            bands = [bench.row_band(height, ws, r) for r in range(ws)]
            assert bands[0][0] == 0 and bands[-1][1] == height
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            assert max(b[1] - b[0] for b in bands) - min(b[1] - b[0] for b in bands) <= 1
    assert bench.rank_view(1, 0) == (0, (0.0, 0.0, 2.5))


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.reference_arm(type("A", (), {"steps": 1, "warmup": 0})())
    assert rc == 0 and buf.getvalue() == ""
