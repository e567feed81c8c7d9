"""Thin Python binding of libsdfnn (argument marshalling only).

Every computation runs in the CUDA library; this module converts torch
tensors into device pointers and the current CUDA stream into a
cudaStream_t.  Importing it does not need a GPU; calling it does, and it
fails loudly (SdfError / RuntimeError) when the library is not built.
The C entry points are declared in include/sdfnn.h.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import torch

from .build import lib_path

SDF_FP32, SDF_BF16, SDF_FP8, SDF_FP16 = 0, 1, 2, 3
SDF_OK = 0
ERRORS = {-1: "SDF_ERR_ARG", -2: "SDF_ERR_FILE", -3: "SDF_ERR_FORMAT", -4: "SDF_ERR_CUDA",
          -5: "SDF_ERR_NONFINITE", -6: "SDF_ERR_TIMEOUT", -7: "SDF_ERR_UNSUPPORTED"}

EXPORTS = ["sdf_net_load", "sdf_net_load_mem", "sdf_net_info", "sdf_net_set_time", "sdf_net_free",
           "sdf_trace_multiscale", "sdf_normals", "sdf_normal_map", "sdf_render_host", "sdf_sync_status",
           "sdf_last_error", "sdf_trace_multiscale_noalloc", "sdf_normal_map_timed", "sdf_plan_create",
           "sdf_plan_launch", "sdf_plan_info", "sdf_plan_free", "sdf_train_shape_info", "sdf_train_forward",
           "sdf_train_backward", "sdf_fit_loss", "sdf_adam_step", "sdf_selftest_wait_timeout",
           "sdf_measure_sine_rate", "sdf_frame_queue_create", "sdf_frame_queue_submit", "sdf_frame_queue_wait",
           "sdf_frame_queue_free", "sdf_selftest_noalloc_timeout", "sdf_theta_from_image",
           "sdf_eval_sine"]


class SdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class TraceParamsC(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("nets", C.POINTER(C.c_void_p)), ("delta", C.POINTER(C.c_float)),
                ("max_iters", C.POINTER(C.c_int)), ("eps", C.c_float), ("step_scale", C.POINTER(C.c_float)),
                ("box_min", C.c_float), ("box_max", C.c_float), ("final_mode", C.c_int), ("time", C.c_float),
                ("ray_time", C.c_void_p)]


class FrameBatchC(C.Structure):
    _fields_ = [("orig", C.c_void_p), ("dir", C.c_void_p), ("ray_time", C.c_void_p), ("n", C.c_int64),
                ("out_pos", C.c_void_p), ("out_t", C.c_void_p), ("out_hit", C.c_void_p), ("out_iters", C.c_void_p),
                ("out_normal", C.c_void_p)]


_lib = None


def lib():
    """The loaded libsdfnn (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = lib_path()
        if not p.exists():
            raise RuntimeError(f"libsdfnn is not built ({p}); run paper_2201_09147_gb300.build.build()")
        L = C.CDLL(str(p))
        vp = C.c_void_p
        L.sdf_net_load.argtypes = [C.c_char_p, C.c_int, C.c_int, C.POINTER(vp)]
        L.sdf_net_load_mem.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.c_int, C.POINTER(vp)]
        L.sdf_net_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]
        L.sdf_net_set_time.argtypes = [vp, C.c_float]
        L.sdf_net_free.argtypes = [vp]
        L.sdf_net_free.restype = None
        L.sdf_trace_multiscale.argtypes = [C.POINTER(TraceParamsC), vp, vp, C.c_int64, vp, vp, vp, vp, vp]
        L.sdf_trace_multiscale_noalloc.argtypes = [C.POINTER(TraceParamsC), vp, vp, C.c_int64, vp, vp, vp, vp, vp]
        L.sdf_normals.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.sdf_normal_map.argtypes = [vp, vp, vp, C.c_int64, vp, vp]
        L.sdf_normal_map_timed.argtypes = [vp, vp, vp, vp, C.c_int64, vp, vp]
        L.sdf_plan_create.argtypes = [C.POINTER(TraceParamsC), vp, C.POINTER(FrameBatchC), C.c_int, vp, C.POINTER(vp)]
        L.sdf_plan_launch.argtypes = [vp, vp]
        L.sdf_plan_info.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int64)]
        L.sdf_plan_free.argtypes = [vp]
        L.sdf_plan_free.restype = None
        L.sdf_render_host.argtypes = [C.POINTER(TraceParamsC), vp, vp, vp, C.c_int64, vp, vp, vp, vp]
        L.sdf_frame_queue_create.argtypes = [C.POINTER(TraceParamsC), vp, C.c_int64, C.c_int, C.POINTER(vp)]
        L.sdf_frame_queue_submit.argtypes = [vp, vp, vp, vp, vp, vp, C.POINTER(C.c_int64)]
        L.sdf_frame_queue_wait.argtypes = [vp, C.c_int64]
        L.sdf_frame_queue_free.argtypes = [vp]
        L.sdf_frame_queue_free.restype = None
        i64p = C.POINTER(C.c_int64)
        L.sdf_train_shape_info.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, i64p, i64p]
        L.sdf_train_forward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_int64, vp, vp, vp, vp]
        L.sdf_train_backward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_int64, vp, vp, vp, vp,
                                         vp]
        L.sdf_fit_loss.argtypes = [vp, vp, vp, vp, vp, C.c_int64, C.c_float, C.c_float, vp, vp, vp, vp]
        L.sdf_adam_step.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                                    vp]
        L.sdf_selftest_wait_timeout.argtypes = [C.c_int, C.c_int64, vp]
        L.sdf_selftest_noalloc_timeout.argtypes = [C.c_int, C.c_int64, vp]
        L.sdf_theta_from_image.argtypes = [C.c_char_p, C.c_size_t, vp, C.c_int64, i64p, C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.sdf_measure_sine_rate.argtypes = [C.c_int, C.POINTER(C.c_double), vp]
        L.sdf_eval_sine.argtypes = [C.c_int, vp, C.c_int64, vp, vp, vp]
        L.sdf_sync_status.argtypes = [vp]
        L.sdf_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != SDF_OK:
        raise SdfError(rc, lib().sdf_last_error().decode(errors="replace"))


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None):
    """Device (or host) address of a tensor's data.  The C calls read SoA arrays at plain offsets,
    so a tensor with other strides (a transposed or sliced view, e.g. one made from a numpy array
    in Fortran order) is refused rather than read in the wrong order."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError(f"tensor of shape {tuple(t.shape)} and strides {t.stride()} is not contiguous; "
                         "pass .contiguous()")
    return C.c_void_p(t.data_ptr())


class Net:
    """A network loaded into the library (sdf_net_load / sdf_net_load_mem)."""

    def __init__(self, source, precision: int = SDF_BF16, device: int = 0):
        h = C.c_void_p()
        if isinstance(source, (bytes, bytearray)):
            _check(lib().sdf_net_load_mem(bytes(source), len(source), precision, device, C.byref(h)))
        else:
            _check(lib().sdf_net_load(str(Path(source)).encode(), precision, device, C.byref(h)))
        self.handle = h
        self.precision = precision
        self.device = device
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(lib().sdf_net_info(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        self.in_dim, self.width, self.n_hidden, self.lipschitz = a.value, b.value, c.value, d.value

    def set_time(self, t: float):
        _check(lib().sdf_net_set_time(self.handle, float(t)))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().sdf_net_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(nets, delta, max_iters, eps, step_scale=None, box=(-1.0, 1.0), final_mode=0, time=0.0,
                ray_time=None):
    """Builds sdf_trace_params; returns (struct, keep-alive tuple)."""
    m = len(nets)
    hs = (C.c_void_p * m)(*[n.handle.value for n in nets])
    d = (C.c_float * m)(*[float(x) for x in delta])
    it = (C.c_int * m)(*[int(x) for x in max_iters])
    ss = None if step_scale is None else (C.c_float * m)(*[float(x) for x in step_scale])
    p = TraceParamsC(m, C.cast(hs, C.POINTER(C.c_void_p)), C.cast(d, C.POINTER(C.c_float)),
                     C.cast(it, C.POINTER(C.c_int)), float(eps),
                     None if ss is None else C.cast(ss, C.POINTER(C.c_float)), float(box[0]), float(box[1]),
                     int(final_mode), float(time), None if ray_time is None else _ptr(ray_time).value)
    return p, (hs, d, it, ss, nets, ray_time)


def trace_multiscale(nets, delta, max_iters, eps, orig, dirs, *, step_scale=None, box=(-1.0, 1.0), final_mode=0,
                     time=0.0, ray_time=None, out_pos=None, out_t=None, out_hit=None, out_iters=None,
                     want_iters=True, stream=None):
    """Alg. 1 on device rays orig/dirs (float32, shape (3, n)); returns (pos, t, hit, iters).
    ray_time: optional device (n,) float32, the 4th input of each ray (4-D networks)."""
    n = orig.shape[1]
    dev = orig.device
    out_pos = torch.empty((3, n), dtype=torch.float32, device=dev) if out_pos is None else out_pos
    out_t = torch.empty(n, dtype=torch.float32, device=dev) if out_t is None else out_t
    out_hit = torch.empty(n, dtype=torch.uint8, device=dev) if out_hit is None else out_hit
    if out_iters is None and want_iters:
        out_iters = torch.empty(n, dtype=torch.uint16, device=dev)
    p, keep = make_params(nets, delta, max_iters, eps, step_scale, box, final_mode, time, ray_time)
    _check(lib().sdf_trace_multiscale(C.byref(p), _ptr(orig), _ptr(dirs), n, _ptr(out_pos), _ptr(out_t),
                                      _ptr(out_hit), _ptr(out_iters), C.c_void_p(_stream(stream))))
    del keep
    return out_pos, out_t, out_hit, out_iters


def trace_multiscale_noalloc(nets, delta, max_iters, eps, orig, dirs, *, step_scale=None, box=(-1.0, 1.0),
                             final_mode=0, time=0.0, ray_time=None, out_pos=None, out_t=None, out_hit=None, out_iters=None,
                             want_iters=True, stream=None):
    """Alg. 1 through sdf_trace_multiscale_noalloc: the library allocates no
    device memory for the call (its scratch is a static device array, at most
    2,097,152 rays per call; calls must not overlap on the GPU).  The output
    tensors, if not given, are still created here by torch."""
    n = orig.shape[1]
    dev = orig.device
    out_pos = torch.empty((3, n), dtype=torch.float32, device=dev) if out_pos is None else out_pos
    out_t = torch.empty(n, dtype=torch.float32, device=dev) if out_t is None else out_t
    out_hit = torch.empty(n, dtype=torch.uint8, device=dev) if out_hit is None else out_hit
    if out_iters is None and want_iters:
        out_iters = torch.empty(n, dtype=torch.uint16, device=dev)
    p, keep = make_params(nets, delta, max_iters, eps, step_scale, box, final_mode, time, ray_time)
    _check(lib().sdf_trace_multiscale_noalloc(C.byref(p), _ptr(orig), _ptr(dirs), n, _ptr(out_pos), _ptr(out_t),
                                              _ptr(out_hit), _ptr(out_iters), C.c_void_p(_stream(stream))))
    del keep
    return out_pos, out_t, out_hit, out_iters


def normals(net: Net, pts, out=None, stream=None):
    """Unnormalised analytic gradients (Alg. 2) at device points (3, n)."""
    n = pts.shape[1]
    out = torch.empty((3, n), dtype=torch.float32, device=pts.device) if out is None else out
    _check(lib().sdf_normals(net.handle, _ptr(pts), n, _ptr(out), C.c_void_p(_stream(stream))))
    return out


def normal_map(net: Net, pts, mask=None, out=None, stream=None):
    """Unit normals of `net` at device points (3, n) where mask != 0 (Sec. 5)."""
    n = pts.shape[1]
    out = torch.empty((3, n), dtype=torch.float32, device=pts.device) if out is None else out
    _check(lib().sdf_normal_map(net.handle, _ptr(pts), _ptr(mask), n, _ptr(out), C.c_void_p(_stream(stream))))
    return out


def normal_map_timed(net: Net, pts, pt_time, mask=None, out=None, stream=None):
    """normal_map of a 4-D network with a time per point (device (n,) float32)."""
    n = pts.shape[1]
    out = torch.empty((3, n), dtype=torch.float32, device=pts.device) if out is None else out
    _check(lib().sdf_normal_map_timed(net.handle, _ptr(pts), _ptr(pt_time), _ptr(mask), n, _ptr(out),
                                      C.c_void_p(_stream(stream))))
    return out


class Plan:
    """A frame-batch plan (sdf_plan_create): the whole trace and the normal
    mapping of a fixed set of device buffers, captured as one CUDA graph.

    The output tensors are allocated here (torch) unless given and are
    attributes of the plan: pos (3, n), t (n), hit (n), iters (n) or None,
    normal (3, n) or None (no fine network)."""

    def __init__(self, nets, delta, max_iters, eps, orig, dirs, *, fine: Net | None = None, ray_time=None,
                 step_scale=None, box=(-1.0, 1.0), final_mode=0, time=0.0, autotune=False, want_iters=True,
                 stream=None):
        n = orig.shape[1]
        dev = orig.device
        self.orig, self.dirs, self.ray_time = orig, dirs, ray_time
        self.pos = torch.empty((3, n), dtype=torch.float32, device=dev)
        self.t = torch.empty(n, dtype=torch.float32, device=dev)
        self.hit = torch.empty(n, dtype=torch.uint8, device=dev)
        self.iters = torch.empty(n, dtype=torch.uint16, device=dev) if want_iters else None
        self.normal = torch.empty((3, n), dtype=torch.float32, device=dev) if fine is not None else None
        self.nets, self.fine, self.n_levels = list(nets), fine, len(nets)
        p, keep = make_params(nets, delta, max_iters, eps, step_scale, box, final_mode, time)
        b = FrameBatchC(_ptr(orig).value, _ptr(dirs).value, None if ray_time is None else _ptr(ray_time).value, n,
                        self.pos.data_ptr(), self.t.data_ptr(), self.hit.data_ptr(),
                        None if self.iters is None else self.iters.data_ptr(),
                        None if self.normal is None else self.normal.data_ptr())
        h = C.c_void_p()
        _check(lib().sdf_plan_create(C.byref(p), None if fine is None else fine.handle, C.byref(b),
                                     1 if autotune else 0, C.c_void_p(_stream(stream)), C.byref(h)))
        del keep
        self.handle = h

    def launch(self, stream=None):
        _check(lib().sdf_plan_launch(self.handle, C.c_void_p(_stream(stream))))

    def info(self):
        """(tile count per level, number of CUDA graph nodes)."""
        tiles = (C.c_int * self.n_levels)()
        nodes = C.c_int64()
        _check(lib().sdf_plan_info(self.handle, tiles, self.n_levels, C.byref(nodes)))
        return list(tiles), nodes.value

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().sdf_plan_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render_host(nets, delta, max_iters, eps, fine: Net, orig, dirs, out_pos, out_hit, out_normal, *,
                step_scale=None, box=(-1.0, 1.0), final_mode=0, time=0.0, stream=None):
    """One frame from host (CPU, ideally pinned) tensors through sdf_render_host."""
    n = orig.shape[1]
    p, keep = make_params(nets, delta, max_iters, eps, step_scale, box, final_mode, time)
    _check(lib().sdf_render_host(C.byref(p), fine.handle, _ptr(orig), _ptr(dirs), n, _ptr(out_pos), _ptr(out_hit),
                                 _ptr(out_normal), C.c_void_p(_stream(stream))))
    del keep


class FrameQueue:
    """Host frames rendered back to back (sdf_frame_queue_*): up to `depth`
    frames in flight, the copies of one frame overlapping the kernels of
    another.  submit() takes host (CPU, ideally pinned) tensors that must stay
    alive and untouched until wait() covers the frame; it returns the
    frame's ticket."""

    def __init__(self, nets, delta, max_iters, eps, fine: Net, n: int, *, depth=2, step_scale=None,
                 box=(-1.0, 1.0), final_mode=0, time=0.0):
        p, keep = make_params(nets, delta, max_iters, eps, step_scale, box, final_mode, time)
        h = C.c_void_p()
        _check(lib().sdf_frame_queue_create(C.byref(p), fine.handle, int(n), int(depth), C.byref(h)))
        del keep
        self.handle, self.n, self.nets, self.fine = h, int(n), list(nets), fine
        self._pending = {}  # ticket -> the frame's host tensors, kept alive until waited for

    def submit(self, orig, dirs, out_pos, out_hit, out_normal) -> int:
        for t, shape in ((orig, (3, self.n)), (dirs, (3, self.n)), (out_pos, (3, self.n)), (out_hit, (self.n,)),
                         (out_normal, (3, self.n))):
            if t.device.type != "cpu" or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"frame buffers are contiguous host tensors of shape {shape}")
        ticket = C.c_int64()
        _check(lib().sdf_frame_queue_submit(self.handle, _ptr(orig), _ptr(dirs), _ptr(out_pos), _ptr(out_hit),
                                            _ptr(out_normal), C.byref(ticket)))
        self._pending[ticket.value] = (orig, dirs, out_pos, out_hit, out_normal)
        return ticket.value

    def wait(self, ticket: int = -1):
        _check(lib().sdf_frame_queue_wait(self.handle, int(ticket)))
        last = max(self._pending) if ticket < 0 and self._pending else ticket
        for k in [k for k in self._pending if k <= last]:
            del self._pending[k]

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib().sdf_frame_queue_free(self.handle)
            self.handle = C.c_void_p()
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_wait_timeout(budget_us: int = 20000, device: int = 0, stream=None):
    """Runs the device-side timeout self-test (raises if the expiry is not reported)."""
    _check(lib().sdf_selftest_wait_timeout(device, int(budget_us), C.c_void_p(_stream(stream))))


def selftest_noalloc_timeout(budget_us: int = 20000, device: int = 0, stream=None):
    """Timeout self-test of the allocation-free entry point's status word (raises if not reported)."""
    _check(lib().sdf_selftest_noalloc_timeout(device, int(budget_us), C.c_void_p(_stream(stream))))


def measure_sine_rate(device: int = 0, stream=None) -> float:
    """Sines per second of the kernels' hardware sine on all SMs."""
    r = C.c_double()
    _check(lib().sdf_measure_sine_rate(device, C.byref(r), C.c_void_p(_stream(stream))))
    return r.value


def eval_sine(x, variant: int, stream=None):
    """(sin, cos) of device float32 x as the kernels compute them: variant 0 = the FP32 path,
    1 = the tensor-core paths."""
    s_, c_ = torch.empty_like(x), torch.empty_like(x)
    _check(lib().sdf_eval_sine(int(variant), _ptr(x), x.numel(), _ptr(s_), _ptr(c_), C.c_void_p(_stream(stream))))
    return s_, c_


def sync_status(stream=None):
    """Synchronises the stream and raises on a device-side error (SDF_ERR_TIMEOUT)."""
    _check(lib().sdf_sync_status(C.c_void_p(_stream(stream))))


# ---------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------

def train_shape_info(in_dim: int, width: int, n_hidden: int, n: int = 0, precision: int = SDF_FP32):
    """(length of theta, workspace bytes for n points at that precision)."""
    pc, wb = C.c_int64(), C.c_int64()
    _check(lib().sdf_train_shape_info(precision, in_dim, width, n_hidden, n, C.byref(pc), C.byref(wb)))
    return pc.value, wb.value


def theta_from_sdfn(data: bytes):
    """(shape, theta) of an SDFN image: the folded parameters as a float32 numpy
    vector, folded by the library (sdf_theta_from_image, host only)."""
    import numpy as np
    data = bytes(data)
    count, a, b, c = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
    _check(lib().sdf_theta_from_image(data, len(data), None, 0, C.byref(count), C.byref(a), C.byref(b), C.byref(c)))
    theta = np.empty(count.value, np.float32)
    _check(lib().sdf_theta_from_image(data, len(data), C.c_void_p(theta.ctypes.data), theta.size, None, None, None,
                                      None))
    return (a.value, b.value, c.value), theta


def sdfn_from_theta(shape, theta) -> bytes:
    """SDFN image (folded, flags bit 0) of a parameter vector."""
    import numpy as np
    in_dim, width, n_hidden = shape
    hdr = np.array([0, 1, in_dim, width, n_hidden, 0, 0, 1], dtype="<u4")
    hdr[5:7] = np.array([1.0, 1.0], dtype="<f4").view("<u4")
    return b"SDFN" + hdr[1:].tobytes() + np.asarray(theta, dtype="<f4").tobytes()


def train_forward(shape, theta, pts, pt_time=None, workspace=None, stream=None, precision: int = SDF_FP32):
    """f (n) and grad f (3, n) at device points (3, n); returns (f, grad, workspace).  A given
    workspace is used if it is large enough, else a new one is made."""
    in_dim, width, n_hidden = shape
    n = pts.shape[1]
    _, wb = train_shape_info(in_dim, width, n_hidden, n, precision)
    if workspace is None or workspace.numel() < wb:
        workspace = torch.empty(wb, dtype=torch.uint8, device=pts.device)
    f = torch.empty(n, dtype=torch.float32, device=pts.device)
    g = torch.empty((3, n), dtype=torch.float32, device=pts.device)
    _check(lib().sdf_train_forward(precision, in_dim, width, n_hidden, _ptr(theta), _ptr(pts), _ptr(pt_time), n,
                                   _ptr(f), _ptr(g), _ptr(workspace), C.c_void_p(_stream(stream))))
    return f, g, workspace


def train_backward(shape, theta, pts, d_f, d_grad, workspace, d_theta=None, pt_time=None, stream=None,
                   precision: int = SDF_FP32):
    """Adds dL/dtheta to d_theta (allocated zero if None) and returns it."""
    in_dim, width, n_hidden = shape
    n = pts.shape[1]
    if d_theta is None:
        d_theta = torch.zeros_like(theta)
    _check(lib().sdf_train_backward(precision, in_dim, width, n_hidden, _ptr(theta), _ptr(pts), _ptr(pt_time), n,
                                    _ptr(d_f), _ptr(d_grad), _ptr(workspace), _ptr(d_theta),
                                    C.c_void_p(_stream(stream))))
    return d_theta


def fit_loss(f, grad, target_f, target_grad, near, lam_n: float, lam_e: float, stream=None):
    """(d_f, d_grad, loss) of the fitting objective; loss = device float64 (l_val, l_dir, l_eik, L)."""
    n = f.shape[0]
    d_f = torch.empty_like(f)
    d_g = torch.empty_like(grad)
    loss = torch.zeros(4, dtype=torch.float64, device=f.device)
    _check(lib().sdf_fit_loss(_ptr(f), _ptr(grad), _ptr(target_f), _ptr(target_grad), _ptr(near), n, float(lam_n),
                              float(lam_e), _ptr(d_f), _ptr(d_g), _ptr(loss), C.c_void_p(_stream(stream))))
    return d_f, d_g, loss


def adam_step(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().sdf_adam_step(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(), float(lr), float(beta1),
                               float(beta2), float(eps), int(step), C.c_void_p(_stream(stream))))


class SineMLP(torch.autograd.Function):
    """(f, grad f) = SineMLP.apply(theta, pts, shape[, pt_time[, precision]]) through the
    library's training kernels; backward gives dL/dtheta (the points get no gradient)."""

    @staticmethod
    def forward(ctx, theta, pts, shape, pt_time=None, precision=SDF_FP32):
        f, g, ws = train_forward(shape, theta.detach(), pts, pt_time, precision=precision)
        ctx.save_for_backward(theta.detach(), pts, ws)
        ctx.shape, ctx.pt_time, ctx.precision = shape, pt_time, precision
        return f, g

    @staticmethod
    def backward(ctx, d_f, d_grad):
        theta, pts, ws = ctx.saved_tensors
        d_f = torch.zeros(pts.shape[1], device=pts.device) if d_f is None else d_f.contiguous()
        d_grad = torch.zeros_like(pts) if d_grad is None else d_grad.contiguous()
        d_theta = train_backward(ctx.shape, theta, pts, d_f, d_grad, ws, pt_time=ctx.pt_time,
                                 precision=ctx.precision)
        return d_theta, None, None, None, None


def fit_step(shape, theta, m, v, step, pts, target_f, target_grad, near, *, lam_n=0.1, lam_e=0.05, lr=1e-4,
             workspace=None, stream=None, precision: int = SDF_FP32, pt_time=None, sine_lr_scale: float = 1.0):
    """One native fitting step: forward, objective, backward, Adam.  Returns (loss, workspace);
    loss is the device float64 vector (l_val, l_dir, l_eik, L) before the update.
    sine_lr_scale multiplies the learning rate of the sine layers' (folded) parameters: with the
    frequency omega it gives the steps Adam takes on the unfolded SIREN parameters."""
    f, g, workspace = train_forward(shape, theta, pts, pt_time=pt_time, workspace=workspace, stream=stream,
                                    precision=precision)
    d_f, d_g, loss = fit_loss(f, g, target_f, target_grad, near, lam_n, lam_e, stream=stream)
    d_theta = train_backward(shape, theta, pts, d_f, d_g, workspace, pt_time=pt_time, stream=stream,
                             precision=precision)
    if sine_lr_scale == 1.0:
        adam_step(theta, d_theta, m, v, step, lr, stream=stream)
    else:
        in_dim, width, n_hidden = shape
        k = width * in_dim + width + n_hidden * (width * width + width)  # the sine layers come first
        adam_step(theta[:k], d_theta[:k], m[:k], v[:k], step, lr * sine_lr_scale, stream=stream)
        adam_step(theta[k:], d_theta[k:], m[k:], v[k:], step, lr, stream=stream)
    return loss, workspace
