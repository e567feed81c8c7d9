"""Device-side failure detection, exercised without a GPU fault: a bounded wait on a
barrier that nothing signals expires, the kernel returns, the host reads the latched
status, and the device keeps working."""
import numpy as np
import pytest
import torch

from paper_2201_09147_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_expiry_is_reported_and_the_device_stays_usable(sdf):
    for _ in range(2):
        sdf.selftest_wait_timeout(20000)   # 20 ms budget, reported as SDF_ERR_TIMEOUT and cleared
    sdf.sync_status()                      # nothing pending afterwards
    wl = workloads.get("normal_map_1080p", 64, 36)
    orig, dirs = wl.rays()
    nets = [sdf.Net(b, sdf.SDF_BF16) for b in wl.level_bytes()]
    pos, _, hit, _ = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, torch.from_numpy(orig).cuda(),
                                          torch.from_numpy(dirs).cuda(), step_scale=wl.step_scale,
                                          final_mode=wl.final_mode)
    sdf.sync_status()
    assert int(hit.sum().item()) > 0 and torch.isfinite(pos).all()


def test_selftest_rejects_bad_budget(sdf):
    with pytest.raises(sdf.SdfError) as e:
        sdf.selftest_wait_timeout(0)
    assert e.value.code == -1
