"""The allocation-free trace entry point, sdf_trace_multiscale_noalloc.

Callers that may not allocate device memory while they run (a render loop
that forbids allocation after start-up, a host whose device memory belongs
to its own allocator) call this variant instead of sdf_trace_multiscale; its
scratch is a static array inside the library.  It must return what the
regular entry point returns, call after call.  This file is collected last
so that a run stopping at its first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2201_09147_gb300 import workloads
from parity import TOL

pytestmark = pytest.mark.gpu

CASES = [("nested_3level_512", 96, 96, 1),   # three levels: uses both ray queues
         ("normal_map_1080p", 200, 113, 3),  # one level, final_mode 1
         ("random_siren_64x1", 64, 64, 0)]   # FP32 kernels, Lipschitz steps


@pytest.mark.parametrize("name,w,h,precision", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_regular_entry_point(sdf, name, w, h, precision):
    wl = workloads.get(name, w, h)
    orig, dirs = wl.rays()
    nets = [sdf.Net(b, precision) for b in wl.level_bytes()]
    o = torch.from_numpy(orig).cuda()
    d = torch.from_numpy(dirs).cuda()
    kw = dict(step_scale=wl.step_scale, final_mode=wl.final_mode)
    ref_pos, ref_t, ref_hit, ref_it = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, o, d, **kw)
    sdf.sync_status()
    tol = TOL[0][1]  # the same kernels run on the same rays: FP32-level agreement
    for _ in range(2):  # two calls in a row share the static scratch
        pos, t, hit, it = sdf.trace_multiscale_noalloc(nets, wl.delta, wl.caps, wl.eps, o, d, **kw)
        torch.cuda.synchronize()
        assert torch.equal(hit, ref_hit)
        assert torch.equal(it, ref_it)
        assert float((pos - ref_pos).abs().max()) <= tol
        assert float((t - ref_t).abs().max()) <= tol
        # no bounded wait of these launches expired: the array's status word is clear
        sdf.sync_status()
    assert int(ref_hit.sum()) > 0


def test_noalloc_rejects_more_rays_than_its_scratch_holds(sdf):
    """One ray more than the static scratch holds is refused before any launch.  The buffers
    passed are sized for that many rays, so a regression that launched anyway would still stay
    inside them."""
    wl = workloads.get("normal_map_1080p", 4, 4)
    nets = [sdf.Net(b, sdf.SDF_FP16) for b in wl.level_bytes()]
    p, keep = sdf.make_params(nets, wl.delta, wl.caps, wl.eps, wl.step_scale, (-1.0, 1.0), wl.final_mode, 0.0)
    n = (1 << 21) + 1
    rays = torch.zeros((3, n), device="cuda")
    rays[2] = 1.0  # unit directions (and origins on the z axis)
    pos = torch.zeros((3, n), device="cuda")
    t = torch.zeros(n, device="cuda")
    hit = torch.zeros(n, dtype=torch.uint8, device="cuda")
    rc = sdf.lib().sdf_trace_multiscale_noalloc(C.byref(p), C.c_void_p(rays.data_ptr()), C.c_void_p(rays.data_ptr()),
                                                n, C.c_void_p(pos.data_ptr()), C.c_void_p(t.data_ptr()),
                                                C.c_void_p(hit.data_ptr()), None, None)
    assert rc == -1
    assert b"at most" in sdf.lib().sdf_last_error()
    torch.cuda.synchronize()
    assert int(hit.sum()) == 0 and float(pos.abs().max()) == 0.0  # nothing ran
    del keep


def test_noalloc_timeout_is_reported_by_sync_status(sdf):
    """A bounded wait that expires while latching into the static array's status word (the
    self-test's wait on a barrier nothing signals, 20 ms) is reported by sdf_sync_status as
    SDF_ERR_TIMEOUT and cleared; the entry point then traces as before."""
    for _ in range(2):
        sdf.selftest_noalloc_timeout(20000)
    sdf.sync_status()
    wl = workloads.get("normal_map_1080p", 64, 36)
    orig, dirs = wl.rays()
    nets = [sdf.Net(b, sdf.SDF_BF16) for b in wl.level_bytes()]
    o = torch.from_numpy(orig).cuda()
    d = torch.from_numpy(dirs).cuda()
    kw = dict(step_scale=wl.step_scale, final_mode=wl.final_mode)
    ref = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, o, d, **kw)
    got = sdf.trace_multiscale_noalloc(nets, wl.delta, wl.caps, wl.eps, o, d, **kw)
    sdf.sync_status()
    assert torch.equal(got[2], ref[2]) and torch.equal(got[0], ref[0])
