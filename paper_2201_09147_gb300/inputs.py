"""Seeded synthetic inputs: network files, cameras, scenes and meshes.

This module is the only code shared by the GPU path's tests and the FP64
oracle's tests.  It draws random numbers and lays out bytes; it holds none of
the method's arithmetic (no network evaluation, no sphere tracing, no
gradients).  Everything is reproducible bit for bit from integer seeds:

* random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014), mapped to
  doubles in [0, 1) by keeping the top 53 bits;
* network weights follow the SIREN initialisation the paper trains with
  (Sec. 2: sine networks initialised as in Sitzmann et al.), drawn layer by
  layer, each weight matrix row-major and then its bias vector;
* the network file layout ("SDFN") stores the sine MLP of Eq. 2 as FP32
  little-endian arrays in the order W_0, b_0, W_1, b_1, ..., W_n, b_n.

Net notation (w, k) follows Sec. 6: k square w x w matrices, i.e. k + 1 sine
layers of width w after the input, then a linear output.
"""
from __future__ import annotations

import dataclasses
import math
import struct
from pathlib import Path

import numpy as np

SDFN_MAGIC = b"SDFN"
SDFN_VERSION = 1
SDFN_HEADER_BYTES = 32
FLAG_FOLDED = 1  # weights already carry the sine frequencies

_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start+1 .. start+n of the SplitMix64 stream seeded with `seed`."""
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * _GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class _Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        u = uniform01(self.seed, n, self.pos)
        self.pos += n
        return lo + (hi - lo) * u


# --------------------------------------------------------------------------
# network files
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SineNet:
    """A sine MLP as stored on disk (Eq. 2), unfolded unless `folded`.

    weights[i] has shape (out, in); layer 0 maps in_dim -> width, layers
    1..n_hidden map width -> width, and the last entry is the 1 x width
    output row.  biases[i] has shape (out,).
    """

    in_dim: int
    width: int
    n_hidden: int
    omega0: float
    omega: float
    weights: list
    biases: list
    folded: bool = False

    def n_params(self) -> int:
        return sum(w.size for w in self.weights) + sum(b.size for b in self.biases)


def param_count(in_dim: int, width: int, n_hidden: int) -> int:
    """Number of FP32 parameters of a (width, n_hidden) sine MLP with in_dim inputs."""
    return width * in_dim + width + n_hidden * (width * width + width) + width + 1


def siren_init(seed: int, width: int, n_hidden: int, in_dim: int = 3,
               omega0: float = 30.0, omega: float = 30.0,
               out_scale: float = 1.0, out_shift: float = 0.0) -> SineNet:
    """SIREN initialisation drawn from SplitMix64(seed).

    Layer 0: W ~ U(-1/in_dim, 1/in_dim).  Hidden layers: W ~ U(-c, c) with
    c = sqrt(6/width)/omega.  Output row: U(-c, c) * out_scale.  Every bias:
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)); `out_shift` is added to the output
    bias afterwards.  Draw order: layer by layer, W row-major, then b.
    """
    rng = _Stream(seed)
    weights, biases = [], []
    fan_in = in_dim
    bound_w = 1.0 / in_dim
    w = rng.uniform(width * in_dim, -bound_w, bound_w).reshape(width, in_dim)
    b = rng.uniform(width, -1.0 / math.sqrt(fan_in), 1.0 / math.sqrt(fan_in))
    weights.append(w)
    biases.append(b)
    c = math.sqrt(6.0 / width) / omega
    for _ in range(n_hidden):
        weights.append(rng.uniform(width * width, -c, c).reshape(width, width))
        biases.append(rng.uniform(width, -1.0 / math.sqrt(width), 1.0 / math.sqrt(width)))
    wo = rng.uniform(width, -c, c).reshape(1, width) * out_scale
    bo = rng.uniform(1, -1.0 / math.sqrt(width), 1.0 / math.sqrt(width)) + out_shift
    weights.append(wo)
    biases.append(bo)
    return _as_f32(SineNet(in_dim, width, n_hidden, omega0, omega, weights, biases, folded=False))


def random_plain_net(seed: int, width: int, n_hidden: int, in_dim: int = 3,
                     scale: float = 1.0, omega0: float = 1.0, omega: float = 1.0) -> SineNet:
    """Weights and biases all U(-scale, scale): a generic net for algebraic pins."""
    rng = _Stream(seed)
    dims = [in_dim] + [width] * (n_hidden + 1)
    weights, biases = [], []
    for i in range(n_hidden + 1):
        weights.append(rng.uniform(dims[i + 1] * dims[i], -scale, scale).reshape(dims[i + 1], dims[i]))
        biases.append(rng.uniform(dims[i + 1], -scale, scale))
    weights.append(rng.uniform(width, -scale, scale).reshape(1, width))
    biases.append(rng.uniform(1, -scale, scale))
    return _as_f32(SineNet(in_dim, width, n_hidden, omega0, omega, weights, biases, folded=False))


def _as_f32(net: SineNet) -> SineNet:
    """Rounds every parameter to float32, the precision the file stores."""
    net.weights = [np.ascontiguousarray(w, np.float32) for w in net.weights]
    net.biases = [np.ascontiguousarray(b, np.float32) for b in net.biases]
    net.omega0 = float(np.float32(net.omega0))
    net.omega = float(np.float32(net.omega))
    return net


def net_to_bytes(net: SineNet) -> bytes:
    flags = FLAG_FOLDED if net.folded else 0
    hdr = SDFN_MAGIC + struct.pack("<IIIIffI", SDFN_VERSION, net.in_dim, net.width, net.n_hidden,
                                   float(net.omega0), float(net.omega), flags)
    assert len(hdr) == SDFN_HEADER_BYTES
    parts = []
    for w, b in zip(net.weights, net.biases):
        parts.append(np.ascontiguousarray(w, dtype="<f4").ravel())
        parts.append(np.ascontiguousarray(b, dtype="<f4").ravel())
    body = np.concatenate(parts)
    assert body.size == param_count(net.in_dim, net.width, net.n_hidden)
    return hdr + body.tobytes()


def net_from_bytes(data: bytes) -> SineNet:
    if len(data) < SDFN_HEADER_BYTES or data[:4] != SDFN_MAGIC:
        raise ValueError("not an SDFN file")
    version, in_dim, width, n_hidden, omega0, omega, flags = struct.unpack("<IIIIffI", data[4:32])
    if version != SDFN_VERSION:
        raise ValueError(f"unsupported SDFN version {version}")
    count = param_count(in_dim, width, n_hidden)
    if len(data) != SDFN_HEADER_BYTES + 4 * count:
        raise ValueError("SDFN size mismatch")
    body = np.frombuffer(data, dtype="<f4", offset=SDFN_HEADER_BYTES).astype(np.float32)
    dims = [in_dim] + [width] * (n_hidden + 1) + [1]
    weights, biases, o = [], [], 0
    for i in range(n_hidden + 2):
        n_out, n_in = dims[i + 1], dims[i]
        weights.append(body[o:o + n_out * n_in].reshape(n_out, n_in).copy())
        o += n_out * n_in
        biases.append(body[o:o + n_out].copy())
        o += n_out
    return SineNet(in_dim, width, n_hidden, omega0, omega, weights, biases, folded=bool(flags & FLAG_FOLDED))


def write_net(path, net: SineNet) -> None:
    Path(path).write_bytes(net_to_bytes(net))


def read_net(path) -> SineNet:
    return net_from_bytes(Path(path).read_bytes())


# --------------------------------------------------------------------------
# cameras and rays
# --------------------------------------------------------------------------

def camera_rays(width: int, height: int, eye=(0.0, 0.0, 2.5), target=(0.0, 0.0, 0.0),
                up=(0.0, 1.0, 0.0), fov_y_deg: float = 45.0, rows=None):
    """Pinhole camera rays, SoA float32 arrays orig (3, n) and dir (3, n).

    Pixel (i, j) (column i, row j, row 0 at the top) shoots through the pixel
    centre (i + 0.5, j + 0.5).  Directions are normalised in float64 and then
    rounded to float32.  `rows` selects a subset of image rows (default all).
    """
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    tan_half = math.tan(math.radians(fov_y_deg) * 0.5)
    aspect = width / height
    rows = np.arange(height) if rows is None else np.asarray(rows)
    jj, ii = np.meshgrid(rows.astype(np.float64), np.arange(width, dtype=np.float64), indexing="ij")
    x = (2.0 * (ii + 0.5) / width - 1.0) * tan_half * aspect
    y = (1.0 - 2.0 * (jj + 0.5) / height) * tan_half
    d = fwd[None, None, :] + x[..., None] * right[None, None, :] + y[..., None] * upv[None, None, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    d = d.reshape(-1, 3)
    o = np.broadcast_to(eye, d.shape)
    return (np.ascontiguousarray(o.T, dtype=np.float32), np.ascontiguousarray(d.T, dtype=np.float32))


def random_rays(seed: int, n: int, box: float = 1.0, radius: float = 2.5):
    """Rays from random points on a sphere of `radius` towards random points in the box."""
    rng = _Stream(seed)
    z = rng.uniform(n, -1.0, 1.0)
    phi = rng.uniform(n, 0.0, 2.0 * math.pi)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    o = radius * np.stack([s * np.cos(phi), s * np.sin(phi), z])
    tgt = np.stack([rng.uniform(n, -box, box) * 0.8 for _ in range(3)])
    d = tgt - o
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    return np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)


def random_points(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n points uniform in the cube [lo, hi]^3, SoA float32 (3, n)."""
    rng = _Stream(seed)
    return np.ascontiguousarray(np.stack([rng.uniform(n, lo, hi) for _ in range(3)]), np.float32)


# --------------------------------------------------------------------------
# the analytic scene the nested sequences are fitted to
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SphereScene:
    """Union of spheres with a small sine displacement.

    g(p) = min_i(|p - c_i| - r_i) + amp * sin(freq x) sin(freq y) sin(freq z).
    g is not an exact SDF: its Lipschitz constant is at most 1 + amp*freq*sqrt(3).
    """

    centres: np.ndarray  # (m, 3)
    radii: np.ndarray  # (m,)
    amp: float = 0.01
    freq: float = 20.0

    def g(self, p: np.ndarray) -> np.ndarray:
        """Field value at points p of shape (n, 3), float64."""
        p = np.asarray(p, np.float64)
        d = np.linalg.norm(p[:, None, :] - self.centres[None], axis=-1) - self.radii[None]
        disp = self.amp * np.sin(self.freq * p[:, 0]) * np.sin(self.freq * p[:, 1]) * np.sin(self.freq * p[:, 2])
        return d.min(axis=1) + disp

    def lipschitz(self) -> float:
        return 1.0 + self.amp * self.freq * math.sqrt(3.0)

    def value_and_grad(self, p: np.ndarray):
        """g and its gradient at points p of shape (n, 3), float64 (the gradient of the
        nearest sphere's distance plus that of the displacement)."""
        p = np.asarray(p, np.float64)
        diff = p[:, None, :] - self.centres[None]
        dist = np.linalg.norm(diff, axis=-1)
        k = np.argmin(dist - self.radii[None], axis=1)
        rows = np.arange(p.shape[0])
        nrm = diff[rows, k] / np.maximum(dist[rows, k], 1e-300)[:, None]
        a, fr = self.amp, self.freq
        sx, sy, sz = np.sin(fr * p[:, 0]), np.sin(fr * p[:, 1]), np.sin(fr * p[:, 2])
        cx, cy, cz = np.cos(fr * p[:, 0]), np.cos(fr * p[:, 1]), np.cos(fr * p[:, 2])
        val = dist[rows, k] - self.radii[k] + a * sx * sy * sz
        grad = nrm + a * fr * np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz], axis=1)
        return val, grad


def sphere_scene(seed: int = 1, m: int = 8, time: float | None = None) -> SphereScene:
    """m spheres, centre U[-0.6, 0.6]^3 then radius U[0.15, 0.3], from SplitMix64(seed).

    With `time` set, every centre moves on a circle of radius 0.15 in the xy
    plane with a seeded phase (drawn after all centres and radii).
    """
    rng = _Stream(seed)
    centres, radii = [], []
    for _ in range(m):
        centres.append(rng.uniform(3, -0.6, 0.6))
        radii.append(rng.uniform(1, 0.15, 0.3)[0])
    centres = np.array(centres)
    if time is not None:
        phase = rng.uniform(m, 0.0, 2.0 * math.pi)
        ang = 2.0 * math.pi * time + phase
        centres = centres + 0.15 * np.stack([np.cos(ang), np.sin(ang), np.zeros(m)], axis=1)
    return SphereScene(centres, np.array(radii))


def fit_batch(scene: SphereScene, seed: int, n: int):
    """Training points of the fitting objective and their targets, from SplitMix64(seed):
    the first n // 2 near the surface (a sphere picked uniformly, a uniform direction,
    the radius plus N(0, 0.02^2) normal jitter), the rest uniform in [-1, 1]^3.
    Returns pts (3, n), target value (n), target gradient (3, n) as float32 and the
    near-surface flags (n) as uint8."""
    rng = _Stream(seed)
    half = n // 2
    m = len(scene.radii)
    k = np.minimum((rng.uniform(half, 0.0, 1.0) * m).astype(np.int64), m - 1)
    z = rng.uniform(half, -1.0, 1.0)
    phi = rng.uniform(half, 0.0, 2.0 * math.pi)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    u = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    # Box-Muller normal jitter of the radius
    u1 = np.maximum(rng.uniform(half, 0.0, 1.0), 1e-300)
    u2 = rng.uniform(half, 0.0, 1.0)
    jit = 0.02 * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    near = scene.centres[k] + (scene.radii[k] + jit)[:, None] * u
    unif = np.stack([rng.uniform(n - half, -1.0, 1.0) for _ in range(3)], axis=1)
    p = np.clip(np.concatenate([near, unif]), -1.0, 1.0)
    p32 = p.astype(np.float32)
    val, grad = scene.value_and_grad(p32.astype(np.float64))
    flags = np.zeros(n, np.uint8)
    flags[:half] = 1
    return (np.ascontiguousarray(p32.T), val.astype(np.float32), np.ascontiguousarray(grad.T, dtype=np.float32),
            flags)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def icosphere(subdivisions: int) -> np.ndarray:
    """Unit icosphere vertices (float64, (V, 3)), V = 10 * 4^s + 2.

    Each subdivision splits every triangle into four through its edge
    midpoints (shared between neighbours) projected onto the unit sphere.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
                      (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], np.float64)
    faces = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
                      (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
                      (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], np.int64)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    for _ in range(subdivisions):
        nv = verts.shape[0]
        edges = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
        key = np.minimum(edges[:, 0], edges[:, 1]) * nv + np.maximum(edges[:, 0], edges[:, 1])
        uniq, inv = np.unique(key, return_inverse=True)
        a, b = uniq // nv, uniq % nv
        mids = verts[a] + verts[b]
        mids /= np.linalg.norm(mids, axis=1, keepdims=True)
        mid = (nv + inv).reshape(3, -1)  # midpoint index of edges (v0v1, v1v2, v2v0) per face
        ab, bc, ca = mid[0], mid[1], mid[2]
        f0, f1, f2 = faces[:, 0], faces[:, 1], faces[:, 2]
        faces = np.concatenate([np.stack([f0, ab, ca], 1), np.stack([f1, bc, ab], 1), np.stack([f2, ca, bc], 1),
                                np.stack([ab, bc, ca], 1)])
        verts = np.concatenate([verts, mids])
    return verts


def displaced_icosphere(scene: SphereScene, subdivisions: int = 7, r_start: float = 1.8,
                        step: float = 1e-3, r_end: float = 0.0) -> tuple[np.ndarray, float]:
    """Icosphere vertices moved radially onto the scene's zero set.

    For each unit vertex u, g(r u) is sampled from r_start inwards with step
    `step`; the first sign change is refined by bisection in float64.  Where
    no sign change exists the vertex stays at r = 1.  Returns SoA float32
    (3, V) and the fraction of vertices that found a root.  Samples beyond the
    scene's bounding radius (max |c_i| + r_i + amp) are skipped: g > 0 there.
    """
    u = icosphere(subdivisions)
    n = u.shape[0]
    r_hit = np.full(n, np.nan)
    bound = float(np.max(np.linalg.norm(scene.centres, axis=1) + scene.radii)) + scene.amp
    k0 = max(0, int(np.floor((r_start - bound) / step)) - 1)
    radii = r_start - step * np.arange(k0, int(np.ceil((r_start - r_end) / step)) + 1)
    # g(r u) along each radial line: |r u - c_i|^2 = r^2 - 2 r (u . c_i) + |c_i|^2
    uc = u @ scene.centres.T
    cc = np.sum(scene.centres ** 2, axis=1)

    def g_radial(sel, r):
        """Sign-exact g(r u): the displacement (|.| <= amp) is added only where it can flip the sign."""
        d = (np.sqrt(np.maximum(r * r - 2.0 * r * uc[sel] + cc[None, :], 0.0)) - scene.radii[None, :]).min(axis=1)
        near = d <= scene.amp
        if near.any():
            us = u[sel[near]]
            d[near] += scene.amp * np.sin(scene.freq * r * us[:, 0]) * np.sin(scene.freq * r * us[:, 1]) * \
                np.sin(scene.freq * r * us[:, 2])
        return d

    active = np.arange(n)
    prev = g_radial(active, radii[0])
    for r in radii[1:]:
        cur = g_radial(active, r)
        newly = (cur <= 0) & (prev > 0)
        if newly.any():
            idx = active[newly]
            lo = np.full(idx.size, r)          # g(lo) <= 0
            hi = np.full(idx.size, r + step)   # g(hi) > 0
            for _ in range(60):
                m = 0.5 * (lo + hi)
                gm = scene.g(u[idx] * m[:, None])
                inside = gm <= 0
                lo = np.where(inside, m, lo)
                hi = np.where(inside, hi, m)
            r_hit[idx] = 0.5 * (lo + hi)
            keep = ~newly
            active, prev = active[keep], cur[keep]
        else:
            prev = cur
        if active.size == 0:
            break
    found = ~np.isnan(r_hit)
    r_hit[~found] = 1.0
    pts = u * r_hit[:, None]
    return np.ascontiguousarray(pts.T, np.float32), float(found.mean())
