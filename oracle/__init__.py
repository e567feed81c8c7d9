"""Python binding of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does.

The C library ``sdf_oracle.c`` restates the paper plainly in double
precision: Eq. 2 (network), Alg. 2 with Eqs. 3-4 (analytic normals), Alg. 1
(multiscale sphere tracing), the neural normal mapping of Sec. 5 and the
threshold recurrences of Props. 1-2 (Sec. 3.3).

``quantised_image`` writes the network with its hidden weights rounded to
16 bits as the tensor-core paths store them; the oracle then evaluates it in
FP64 (a reported mode that separates weight rounding from arithmetic error).

``fit_loss`` and ``adam_step`` (FP64, numpy on top of the C network) define
the fitting objective and the optimiser step of the training path.  The
paper trains each network of a sequence with an external framework it only
cites (Sec. 2, Sec. 3.3); the objective restated here is the one that
framework's SDF fitting uses: an L1 term on the values, a (1 - cos) term on
the gradient directions at points near the surface and an Eikonal term.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sdf_oracle.c"
_BUILD = _HERE / "_build"

SDF_KIND_NET, SDF_KIND_SPHERE, SDF_KIND_TORUS = 0, 1, 2


def lib_path() -> Path:
    return _BUILD / f"liboracle_{platform.machine()}.so"


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (IEEE double, no contraction into FMA)."""
    out = lib_path()
    if out.exists() and not force and out.stat().st_mtime >= _SRC.stat().st_mtime:
        return out
    _BUILD.mkdir(exist_ok=True)
    tmp = out.with_suffix(f".tmp{os.getpid()}.so")
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-o", str(tmp), str(_SRC), "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _SDF(C.Structure):
    _fields_ = [("kind", C.c_int), ("net", C.c_void_p), ("c", C.c_double * 3), ("r", C.c_double),
                ("R", C.c_double), ("time", C.c_double)]


class _TraceParams(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("levels", C.POINTER(_SDF)), ("delta", C.POINTER(C.c_double)),
                ("cap", C.POINTER(C.c_int)), ("scale", C.POINTER(C.c_double)), ("eps", C.c_double),
                ("box_lo", C.c_double), ("box_hi", C.c_double), ("final_mode", C.c_int)]


class _RayResult(C.Structure):
    _fields_ = [("hit", C.c_int), ("iters", C.c_int), ("p", C.c_double * 3), ("tau", C.c_double)]


_lib = None
_POOL = None  # threads of eval_batch


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(build()))
        vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)
        L.oracle_net_from_bytes.restype = vp
        L.oracle_net_from_bytes.argtypes = [C.c_char_p, C.c_size_t]
        L.oracle_net_free.argtypes = [vp]
        L.oracle_net_shape.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.oracle_net_eval.restype = C.c_double
        L.oracle_net_eval.argtypes = [vp, dp]
        L.oracle_net_grad.argtypes = [vp, dp, dp]
        L.oracle_lipschitz.restype = C.c_double
        L.oracle_lipschitz.argtypes = [vp]
        L.oracle_sdf_value.restype = C.c_double
        L.oracle_sdf_value.argtypes = [C.POINTER(_SDF), dp]
        L.oracle_trace_ray.argtypes = [C.POINTER(_TraceParams), dp, dp, C.POINTER(_RayResult), dp,
                                       C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
        L.oracle_trace_batch.argtypes = [C.POINTER(_TraceParams), fp, fp, C.c_int64, C.POINTER(C.c_int64),
                                         C.c_int64, fp, dp, fp, C.POINTER(C.c_uint8), C.POINTER(C.c_int32),
                                         C.c_int]
        L.oracle_first_root.restype = C.c_int
        L.oracle_first_root.argtypes = [C.POINTER(_SDF), dp, dp, C.c_double, C.c_double, C.c_double,
                                        C.c_double, dp]
        L.oracle_grad_batch.argtypes = [vp, dp, C.c_int64, C.c_double, dp, dp, C.c_int]
        L.oracle_normal_map.argtypes = [vp, dp, C.POINTER(C.c_uint8), C.c_int64, C.c_double, dp, C.c_int]
        L.oracle_thresholds_prop1.argtypes = [dp, C.c_int, dp]
        L.oracle_thresholds_prop2.argtypes = [dp, C.c_int, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Net:
    """An SDFN network loaded by the oracle (folded, float64)."""

    def __init__(self, data: bytes):
        self._h = lib().oracle_net_from_bytes(data, len(data))
        if not self._h:
            raise ValueError("oracle could not parse the SDFN image")
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        lib().oracle_net_shape(self._h, C.byref(a), C.byref(b), C.byref(c))
        self.in_dim, self.width, self.n_hidden = a.value, b.value, c.value

    @classmethod
    def from_file(cls, path, **kw):
        return cls(Path(path).read_bytes(), **kw)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_net_free(self._h)
            self._h = None

    def eval(self, p) -> float:
        q = np.zeros(4)
        q[:len(p)] = p
        return lib().oracle_net_eval(self._h, _dp(q))

    def grad(self, p) -> np.ndarray:
        q = np.zeros(4)
        q[:len(p)] = p
        g = np.zeros(4)
        lib().oracle_net_grad(self._h, _dp(q), _dp(g))
        return g[:self.in_dim].copy()

    def lipschitz(self) -> float:
        return lib().oracle_lipschitz(self._h)

    def grad_batch(self, pts, time: float = 0.0, with_value: bool = False, threads: int | None = None):
        """Alg. 2 at SoA points (3, n) -> gradients (3, n) float64 (and values)."""
        pts = np.ascontiguousarray(pts, np.float64)
        n = pts.shape[1]
        g = np.zeros((3, n))
        v = np.zeros(n) if with_value else None
        lib().oracle_grad_batch(self._h, _dp(pts), n, time, _dp(g), _dp(v) if with_value else None,
                                threads or default_threads())
        return (g, v) if with_value else g

    def normal_map(self, pts, mask=None, time: float = 0.0, threads: int | None = None) -> np.ndarray:
        pts = np.ascontiguousarray(pts, np.float64)
        n = pts.shape[1]
        out = np.zeros((3, n))
        m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
        lib().oracle_normal_map(self._h, _dp(pts), None if m is None else m.ctypes.data_as(C.POINTER(C.c_uint8)),
                                n, time, _dp(out), threads or default_threads())
        return out


class SDF:
    """One level of a traced sequence: a network or an analytic shape."""

    def __init__(self, kind, net: Net | None = None, centre=(0, 0, 0), r=0.0, R=0.0, time=0.0):
        self.net = net  # keeps the network alive
        self.s = _SDF(kind, net._h if net is not None else None, (C.c_double * 3)(*centre), r, R, time)

    @classmethod
    def of_net(cls, net: Net, time: float = 0.0):
        return cls(SDF_KIND_NET, net=net, time=time)

    @classmethod
    def sphere(cls, centre, r):
        return cls(SDF_KIND_SPHERE, centre=centre, r=r)

    @classmethod
    def torus(cls, centre, R, r):
        return cls(SDF_KIND_TORUS, centre=centre, R=R, r=r)

    def value(self, p) -> float:
        q = np.ascontiguousarray(p, np.float64)
        return lib().oracle_sdf_value(C.byref(self.s), _dp(q))


class TraceParams:
    """Alg. 1 parameters for a nested sequence f_1 |> ... |> f_m."""

    def __init__(self, levels, delta, caps, scales, eps, box=(-1.0, 1.0), final_mode=0):
        m = len(levels)
        self.levels = list(levels)
        self._lv = (_SDF * m)(*[lv.s for lv in levels])
        self._delta = np.ascontiguousarray(np.broadcast_to(np.asarray(delta, np.float64), (m,)))
        self._cap = (C.c_int * m)(*[int(c) for c in caps])
        self._scale = np.ascontiguousarray(np.broadcast_to(np.asarray(scales, np.float64), (m,)))
        self.p = _TraceParams(m, self._lv, _dp(self._delta), self._cap, _dp(self._scale), float(eps),
                              float(box[0]), float(box[1]), int(final_mode))

    def trace_ray(self, o, v, traj_cap: int = 0):
        o = np.ascontiguousarray(o, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        r = _RayResult()
        if traj_cap:
            traj = np.zeros((traj_cap, 3))
            lvl = (C.c_int * traj_cap)()
            tl = C.c_int()
            lib().oracle_trace_ray(C.byref(self.p), _dp(o), _dp(v), C.byref(r), _dp(traj), lvl, traj_cap,
                                   C.byref(tl))
            return r, traj[:tl.value].copy(), np.array(lvl[:tl.value])
        lib().oracle_trace_ray(C.byref(self.p), _dp(o), _dp(v), C.byref(r), None, None, 0, None)
        return r

    def trace_batch(self, orig, dirs, idx=None, threads: int | None = None):
        """Trace SoA float32 rays (3, N); `idx` selects a subset.  Returns a dict."""
        orig = np.ascontiguousarray(orig, np.float32)
        dirs = np.ascontiguousarray(dirs, np.float32)
        N = orig.shape[1]
        ii = None if idx is None else np.ascontiguousarray(idx, np.int64)
        n = N if ii is None else ii.size
        pos = np.zeros((3, n), np.float32)
        pos64 = np.zeros((3, n))
        tau = np.zeros(n, np.float32)
        hit = np.zeros(n, np.uint8)
        iters = np.zeros(n, np.int32)
        lib().oracle_trace_batch(C.byref(self.p), _fp(orig), _fp(dirs), N,
                                 None if ii is None else ii.ctypes.data_as(C.POINTER(C.c_int64)), n,
                                 _fp(pos), _dp(pos64), _fp(tau), hit.ctypes.data_as(C.POINTER(C.c_uint8)),
                                 iters.ctypes.data_as(C.POINTER(C.c_int32)), threads or default_threads())
        return {"pos": pos64, "tau": tau, "hit": hit, "iters": iters}


def first_root(sdf: SDF, o, v, t0, t1, h=1e-4, tol=1e-13):
    o = np.ascontiguousarray(o, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    t = C.c_double()
    ok = lib().oracle_first_root(C.byref(sdf.s), _dp(o), _dp(v), t0, t1, h, tol, C.byref(t))
    return t.value if ok else None


def _parse_sdfn(data: bytes):
    """(in_dim, width, n_hidden, folded sine-layer weights [(W, b)], w_out, b_out) of an SDFN image,
    FP64; the frequencies multiplied in as in Eq. 2 written with plain sin(W x + b): layer 0 by
    omega0, the hidden layers by omega, the linear output row unchanged."""
    hdr = np.frombuffer(data[4:32], dtype="<u4")
    in_dim, width, n_hidden, flags = int(hdr[1]), int(hdr[2]), int(hdr[3]), int(hdr[6])
    omega0, omega = (float(x) for x in np.frombuffer(data[20:28], dtype="<f4"))
    q = np.frombuffer(data[32:], dtype="<f4").astype(np.float64)
    layers, o = [], 0
    for li in range(n_hidden + 1):
        fan_in = in_dim if li == 0 else width
        s = 1.0 if flags & 1 else (omega0 if li == 0 else omega)
        W = q[o:o + width * fan_in].reshape(width, fan_in) * s
        o += width * fan_in
        b = q[o:o + width] * s
        o += width
        layers.append((W, b))
    w_out = q[o:o + width]
    b_out = float(q[o + width])
    return in_dim, width, n_hidden, layers, w_out, b_out


def round_bf16(x) -> np.ndarray:
    """Each float32 of x rounded to the nearest bfloat16 (ties to even), returned as float32: the top
    16 bits of the float32 pattern after adding half of the dropped range (0x7FFF plus the lowest
    kept bit, so that an exact half rounds to the even neighbour).  Finite inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def quantised_image(net_bytes: bytes, fmt: str = "bf16") -> bytes:
    """The SDFN image of the network whose hidden weights are those the 16-bit tensor-core paths
    multiply with, stored folded (flag 1): every hidden W' = omega W formed in FP64, rounded to
    float32, then to bfloat16 ("bf16") or IEEE half ("f16"), round to nearest even; layer 0, the
    biases and the output row as the float32 rounding of their folded FP64 values.  Evaluated by
    this oracle in FP64, it separates the error of storing the weights in 16 bits from the error of
    the 16-bit arithmetic on the activations (the reference-only mode of Sec. 5.1's normals)."""
    in_dim, width, n_hidden, layers, w_out, b_out = _parse_sdfn(net_bytes)
    hdr = bytearray(net_bytes[:32])
    flags = int(np.frombuffer(bytes(hdr[28:32]), dtype="<u4")[0]) | 1
    hdr[28:32] = np.array([flags], dtype="<u4").tobytes()
    parts = []
    for li, (W, b) in enumerate(layers):
        w32 = W.astype(np.float32)
        if li > 0:
            w32 = round_bf16(w32) if fmt == "bf16" else w32.astype(np.float16).astype(np.float32)
        parts += [w32.ravel(), b.astype(np.float32)]
    parts += [w_out.astype(np.float32), np.array([b_out], np.float32)]
    return bytes(hdr) + np.concatenate(parts).astype("<f4").tobytes()


def eval_batch(net_bytes: bytes, pts, threads: int | None = None) -> np.ndarray:
    """Eq. 2 at many points in FP64 with numpy: rows of `pts` (in_dim, n) are x, y, z (and t for
    4-D networks); f_0 = sin(W_0 p + b_0), f_i = sin(W_i f_{i-1} + b_i), f = w_out . f_k + b_out.
    The matrix products are library calls; chunks of points run on `threads` threads.  The
    per-point loops of oracle_net_eval compute the same values (pinned against them)."""
    import concurrent.futures as cf
    global _POOL
    in_dim, width, n_hidden, layers, w_out, b_out = _parse_sdfn(net_bytes)
    P = np.ascontiguousarray(np.asarray(pts, np.float64)[:in_dim])
    n = P.shape[1]
    out = np.empty(n)

    def run(lo, hi):
        x = P[:, lo:hi]
        for W, b in layers:
            x = np.sin(W @ x + b[:, None])
        out[lo:hi] = w_out @ x + b_out

    nt = threads or default_threads()
    chunk = max(256, min(16384, -(-n // nt)))
    if n <= chunk:
        run(0, n)
        return out
    if _POOL is None or _POOL._max_workers != nt:
        _POOL = cf.ThreadPoolExecutor(max_workers=nt)
    list(_POOL.map(lambda lo: run(lo, min(n, lo + chunk)), range(0, n, chunk)))
    return out


def max_preactivation(net_bytes: bytes, pts) -> list:
    """Largest |W_l x + b_l| per sine layer of Eq. 2 (frequencies folded) over the points."""
    _, _, _, layers, _, _ = _parse_sdfn(net_bytes)
    x = np.asarray(pts, np.float64)[:layers[0][0].shape[1]]
    out = []
    for W, b in layers:
        z = W @ x + b[:, None]
        out.append(float(np.abs(z).max()))
        x = np.sin(z)
    return out


def first_roots_batch(net_bytes: bytes, offset: float, orig, dirs, t0, t1, h: float = 1e-3, time=None,
                      bisections: int = 60):
    """The plain definition of the first hit, for many rays at once: the first root of f - offset
    along o + t v for t in [t0, t1], found as oracle_first_root does (march with step h until the
    sign changes or f - offset == 0, then bisect), all rays in lockstep with eval_batch.

    orig, dirs: (3, n); t0, t1: (n,).  Returns (t_root (nan where no root), the smallest
    f - offset seen on the march) per ray."""
    o = np.asarray(orig, np.float64)
    v = np.asarray(dirs, np.float64)
    t0 = np.asarray(t0, np.float64)
    t1 = np.asarray(t1, np.float64)
    n = o.shape[1]

    def f(idx, t):
        p = o[:, idx] + t * v[:, idx]
        if time is not None:
            p = np.vstack([p, np.full((1, idx.size), float(time))])
        return eval_batch(net_bytes, p) - offset

    t_root = np.full(n, np.nan)
    fmin = np.full(n, np.inf)
    lo = np.full(n, np.nan)
    hi = np.full(n, np.nan)
    t = t0.copy()
    fa = np.full(n, np.nan)
    idx = np.nonzero(t1 >= t0)[0]
    fa[idx] = f(idx, t[idx])
    fmin[idx] = fa[idx]
    at_root = idx[fa[idx] == 0.0]
    t_root[at_root] = t[at_root]
    idx = idx[fa[idx] != 0.0]
    while idx.size:
        tb = np.minimum(t[idx] + h, t1[idx])
        fb = f(idx, tb)
        fmin[idx] = np.minimum(fmin[idx], fb)
        zero = fb == 0.0
        t_root[idx[zero]] = tb[zero]
        cross = ~zero & ((fa[idx] > 0.0) != (fb > 0.0))
        lo[idx[cross]] = t[idx[cross]]
        hi[idx[cross]] = tb[cross]
        done = zero | cross | (tb >= t1[idx])
        t[idx] = tb
        fa[idx] = fb
        idx = idx[~done]
    b = np.nonzero(~np.isnan(lo))[0]
    if b.size:
        L, H = lo[b].copy(), hi[b].copy()
        fL = f(b, L)
        for _ in range(bisections):
            M = 0.5 * (L + H)
            same = (f(b, M) > 0.0) == (fL > 0.0)
            L = np.where(same, M, L)
            H = np.where(same, H, M)
        t_root[b] = 0.5 * (L + H)
    return t_root, fmin


def nesting_violations(coarse: np.ndarray, delta_c: float, fine: np.ndarray, delta_f: float):
    """Eq. 1 on samples: the points in [|f_fine| <= delta_f] that are outside [|f_coarse| <= delta_c].
    Returns (number of samples in the fine neighbourhood, number of violations, the largest
    |f_coarse| over the fine neighbourhood)."""
    inner = np.abs(fine) <= delta_f
    worst = float(np.abs(coarse[inner]).max()) if inner.any() else 0.0
    return int(inner.sum()), int(np.sum(np.abs(coarse[inner]) > delta_c)), worst


def thresholds_prop1(eps):
    e = np.ascontiguousarray(eps, np.float64)
    d = np.zeros_like(e)
    lib().oracle_thresholds_prop1(_dp(e), e.size, _dp(d))
    return d


def thresholds_prop2(eps):
    e = np.ascontiguousarray(eps, np.float64)
    d = np.zeros_like(e)
    lib().oracle_thresholds_prop2(_dp(e), e.size, _dp(d))
    return d


def fit_loss(net_bytes: bytes, pts, target_f, target_grad, near, lam_n: float, lam_e: float, time: float = 0.0):
    """Fitting objective of one network at SoA points (3, n), in FP64:

        L = mean_i |f(p_i) - g_i|
          + lam_n * mean_{i near} (1 - <grad f(p_i), grad g_i> / (|grad f(p_i)| |grad g_i|))
          + lam_e * mean_i | |grad f(p_i)| - 1 |

    with f and grad f from Eq. 2 and Alg. 2; `near` marks the points that
    enter the direction term (a mean over an empty set is 0).  Returns
    (L, (l_val, l_dir, l_eik)).
    """
    gf, f = Net(net_bytes).grad_batch(pts, time=time, with_value=True)
    tf = np.asarray(target_f, np.float64)
    tg = np.asarray(target_grad, np.float64)
    near = np.asarray(near).astype(bool)
    l_val = float(np.mean(np.abs(f - tf)))
    na = np.linalg.norm(gf, axis=0)
    nb = np.linalg.norm(tg, axis=0)
    cos = np.sum(gf * tg, axis=0) / (na * nb)
    l_dir = float(np.mean(1.0 - cos[near])) if near.any() else 0.0
    l_eik = float(np.mean(np.abs(na - 1.0)))
    return l_val + lam_n * l_dir + lam_e * l_eik, (l_val, l_dir, l_eik)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba) in FP64: returns (theta, m, v) after step `step` (1-based)."""
    theta, grad = np.asarray(theta, np.float64), np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
