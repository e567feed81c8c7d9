"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1).

Each rank times its own replica; the job value is all ranks' units over the
slowest rank's time, and every rank agrees on it.  The reference arm runs on
rank 0 only."""
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
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        value, max_ms = bench.job_throughput(local_ms, 2_000_000, 10, ws)
        out.put((rank, value, max_ms, bench.dist_info()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, m0, d0), (r1, v1, m1, d1) = res
    assert m0 == m1 == 150.0                      # max over ranks
    assert v0 == v1 == pytest.approx(2 * 2_000_000 * 10 / 0.150 / 1e6)
    assert d0 == (2, 0, 0) and d1 == (2, 1, 1)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.reference_arm(type("A", (), {"steps": 1, "warmup": 0})())
    assert rc == 0 and buf.getvalue() == ""
