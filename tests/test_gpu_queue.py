"""Frame queues (sdf_frame_queue_*): host frames rendered back to back with
their copies overlapping the kernels of neighbouring frames give the bytes of
the device calls (sdf_trace_multiscale + sdf_normal_map) frame by frame."""
import numpy as np
import pytest
import torch

from paper_2201_09147_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu


def _device_frame(sdf, wl, nets, fine, orig, dirs):
    o = torch.from_numpy(np.ascontiguousarray(orig)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(dirs)).cuda()
    pos, _, hit, _ = sdf.trace_multiscale(nets, wl.delta, wl.caps, wl.eps, o, d, step_scale=wl.step_scale,
                                          final_mode=wl.final_mode, want_iters=False)
    nrm = sdf.normal_map(fine, pos, hit)
    sdf.sync_status()
    return pos.cpu(), hit.cpu(), nrm.cpu()


def _frames(orig, dirs, count, seed):
    """`count` frames: the rays in a different seeded order each time."""
    n = orig.shape[1]
    out = []
    for k in range(count):
        perm = np.argsort(inputs.uniform01(seed + k, n), kind="stable")
        out.append((perm, np.ascontiguousarray(orig[:, perm]), np.ascontiguousarray(dirs[:, perm])))
    return out


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_frame_queue_matches_device_calls(sdf, depth, memory):
    wl = workloads.get("normal_map_1080p", 320, 180)
    orig, dirs = wl.rays()
    n = orig.shape[1]
    nets = [sdf.Net(b, sdf.SDF_BF16) for b in wl.level_bytes()]
    fine = sdf.Net(wl.fine_bytes(), sdf.SDF_BF16)
    ref_pos, ref_hit, ref_nrm = _device_frame(sdf, wl, nets, fine, orig, dirs)
    pin = (lambda t: t.pin_memory()) if memory == "pinned" else (lambda t: t)
    q = sdf.FrameQueue(nets, wl.delta, wl.caps, wl.eps, fine, n, depth=depth, step_scale=wl.step_scale,
                       final_mode=wl.final_mode)
    outs = []
    for k, (perm, o, d) in enumerate(_frames(orig, dirs, 5, 40)):
        bufs = (pin(torch.from_numpy(o)), pin(torch.from_numpy(d)), pin(torch.full((3, n), float("nan"))),
                pin(torch.full((n,), 7, dtype=torch.uint8)), pin(torch.full((3, n), float("nan"))))
        assert q.submit(*bufs) == k
        outs.append((perm, bufs))
    q.wait()
    for perm, (_, _, pos, hit, nrm) in outs:
        p = torch.from_numpy(perm)
        assert torch.equal(hit, ref_hit[p])
        assert torch.equal(pos, ref_pos[:, p])
        assert torch.equal(nrm, ref_nrm[:, p])
    q.close()


def test_frame_queue_three_levels_and_tickets(sdf):
    """Three levels (the plan's level queues inside each slot), waits on single tickets, an unissued ticket,
    and freeing a queue with frames in flight."""
    wl = workloads.get("three_level_512")
    orig, dirs = wl.rays()
    n = orig.shape[1]
    nets = [sdf.Net(b, sdf.SDF_BF16) for b in wl.level_bytes()]
    fine = sdf.Net(wl.fine_bytes(), sdf.SDF_BF16)
    ref_pos, ref_hit, ref_nrm = _device_frame(sdf, wl, nets, fine, orig, dirs)
    q = sdf.FrameQueue(nets, wl.delta, wl.caps, wl.eps, fine, n, depth=2, step_scale=wl.step_scale,
                       final_mode=wl.final_mode)
    with pytest.raises(sdf.SdfError) as e:
        q.wait(0)  # nothing submitted yet
    assert e.value.code == -1
    q.wait()  # no frame: returns at once
    frames = _frames(orig, dirs, 4, 90)
    for k, (perm, o, d) in enumerate(frames):
        bufs = (torch.from_numpy(o).pin_memory(), torch.from_numpy(d).pin_memory(), torch.empty((3, n)).pin_memory(),
                torch.empty(n, dtype=torch.uint8).pin_memory(), torch.empty((3, n)).pin_memory())
        t = q.submit(*bufs)
        q.wait(t)  # this frame (and every earlier one) is in host memory now
        p = torch.from_numpy(perm)
        assert torch.equal(bufs[3], ref_hit[p]) and torch.equal(bufs[2], ref_pos[:, p])
        assert torch.equal(bufs[4], ref_nrm[:, p])
    with pytest.raises(sdf.SdfError):
        q.wait(len(frames))
    o = torch.from_numpy(np.ascontiguousarray(orig)).pin_memory()
    d = torch.from_numpy(np.ascontiguousarray(dirs)).pin_memory()
    keep = [torch.empty((3, n)).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory(),
            torch.empty((3, n)).pin_memory()]
    q.submit(o, d, *keep)
    q.close()  # waits for the frame in flight before freeing
    sdf.sync_status()


def test_frame_queue_rejects_bad_arguments(sdf):
    wl = workloads.get("normal_map_1080p", 64, 36)
    nets = [sdf.Net(b, sdf.SDF_BF16) for b in wl.level_bytes()]
    fine = sdf.Net(wl.fine_bytes(), sdf.SDF_BF16)
    for n, depth in ((0, 2), (wl.n_rays, 0), (wl.n_rays, 5)):
        with pytest.raises(sdf.SdfError) as e:
            sdf.FrameQueue(nets, wl.delta, wl.caps, wl.eps, fine, n, depth=depth, step_scale=wl.step_scale,
                           final_mode=wl.final_mode)
        assert e.value.code == -1
    q = sdf.FrameQueue(nets, wl.delta, wl.caps, wl.eps, fine, wl.n_rays, step_scale=wl.step_scale,
                       final_mode=wl.final_mode)
    with pytest.raises(ValueError):
        q.submit(torch.zeros((3, wl.n_rays - 1)), torch.zeros((3, wl.n_rays)), torch.zeros((3, wl.n_rays)),
                 torch.zeros(wl.n_rays, dtype=torch.uint8), torch.zeros((3, wl.n_rays)))
    q.close()
