"""Named synthetic workloads (input recipes shared by tests and the benchmark).

Each workload fixes the networks, Alg. 1 parameters and rays; nothing here
evaluates a network.  The fitted sequences live in ``scenes/`` (written by
``fit.py`` from the seeded sphere scene of ``inputs.sphere_scene``).

* ``random_siren_64x1`` - one random SIREN (64, 1), seed 0, traced with the
  Lipschitz step 1/L at 128 x 128, 32 steps, eps 1e-3, normals at the hits.
  SIREN's output initialisation keeps |f| below 0.1, so the printed +0.3
  shift alone leaves f > 0 everywhere; the output row is drawn at the
  fan-in scale U(+-sqrt(6/w)) (the linear output layer carries no omega)
  and 0.3 is added to its bias, which gives a non-empty zero set.
* ``nested_3level_512`` - (64,2) |> (128,2) |> (256,2) fitted to the scene,
  delta = 0.04 / 0.015 / 0.005, caps 48 / 32 / 16, 512 x 512 rays, normals
  of the finest net at the hits.
* ``normal_map_1080p`` - trace the coarse (64,1) until f <= delta_0 + eps
  (final_mode 1, delta_0 = 0.04, cap 40) at 1920 x 1080, then map the
  normals of the fine (256,3) onto the end points (Sec. 5).  Its plain
  comparison is the (256,3) alone, 40 steps, with its own normals.
* ``normal_map_1080p_c64x2`` - the same frame with the (64,2) of the nested
  sequence as the coarse net (the other reading of config 3's "coarse
  64-wide net"), delta_0 = 0.04, cap 40.
* ``normal_map_1080p_zero`` - the coarse (64,1) traced to its own zero set
  (final_mode 0, cap 40), then the (256,3) normals mapped onto those end
  points: the zero-set reading of Sec. 5.
* ``three_level_512`` - the schedule of the last row of Tab. 3: the (64,1)
  for 20 steps to its delta shell (0.04), the (256,1) for 5 steps to its
  own shell (0.02) against the (256,3), whose normals are then mapped onto
  the end points; 512 x 512 rays.
* ``silhouette_512`` - the same with (256,2) as the middle level (shell
  0.01), the variant whose silhouettes Sec. 6 compares.
* ``animation_32`` - 32 frames of the animated scene (sphere centres moving
  on circles, ``inputs.sphere_scene(time=t)``), t_k = k / 31: 8 frames at
  256 x 256, 16 at 1280 x 720, 8 at 1920 x 1080 (31,858,688 rays), traced as
  one batch with a time per ray through the 4-D (64,1) to its delta shell
  and normal-mapped with the 4-D (256,3) (Sec. 3.2, Sec. 5).
* ``animation_32_pair`` - the same 32 frames with the paper's animated pair
  (Sec. 6: coarse (64,1), baseline (128,2)): the 4-D (64,1) to its delta
  shell, normals of the 4-D (128,2).
* ``animation_32_single`` - the same 32 frames traced on the 4-D (256,3)
  itself (its zero set, 40 steps) with its own normals: the single-network
  reading of the batched animation.
* ``mesh_normals`` - vertices of a subdivision-7 icosphere moved onto the
  scene's zero set, normal-mapped with the fine (256,3).
"""
from __future__ import annotations

import dataclasses
from pathlib import Path

import numpy as np

from . import inputs

SCENES = Path(__file__).resolve().parent / "scenes"


@dataclasses.dataclass
class Workload:
    name: str
    levels: list          # network file names (scenes/) or SineNet objects
    delta: list
    caps: list
    eps: float
    step_scale: list | None  # None: 1/L per level
    final_mode: int
    width: int
    height: int
    fine: object          # network used for the normals / normal mapping
    frames: list | None = None  # [(width, height, time)] of a frame batch (4-D networks)

    def level_bytes(self):
        return [_net_bytes(x) for x in self.levels]

    def fine_bytes(self):
        return _net_bytes(self.fine)

    def rays(self, rows=None):
        return inputs.camera_rays(self.width, self.height, rows=rows)

    @property
    def n_rays(self) -> int:
        if self.frames is not None:
            return sum(w * h for w, h, _ in self.frames)
        return self.width * self.height


def _net_bytes(x) -> bytes:
    if isinstance(x, inputs.SineNet):
        return inputs.net_to_bytes(x)
    return (SCENES / x).read_bytes()


def random_siren_64x1() -> inputs.SineNet:
    return inputs.siren_init(0, 64, 1, out_scale=30.0, out_shift=0.3)


# delta of the 4-D (64,1) against the 4-D (256,3): the largest |f_c - f_f| found near the
# surface (|f_f| < 0.05) over 20,000 points at five times was 0.057
ANIM_DELTA = 0.06
# delta of the 4-D (64,1) against the 4-D (128,2) of the animated pair: the same 0.06 (Eq. 1 holds
# on 10^6 samples at eight times, tests/test_oracle_nesting.py)
ANIM_PAIR_DELTA = 0.06


def animation_frames(counts=((8, 256, 256), (16, 1280, 720), (8, 1920, 1080))):
    """[(width, height, time)]: frames in the order of `counts`, t_k = k / (K - 1)."""
    sizes = [(w, h) for c, w, h in counts for _ in range(c)]
    k = len(sizes)
    return [(w, h, (i / (k - 1)) if k > 1 else 0.0) for i, (w, h) in enumerate(sizes)]


def batch_rays(frames):
    """Rays of a frame batch: orig (3, N), dir (3, N) float32, time (N,) float32 and the
    start offset of each frame (len(frames) + 1)."""
    os_, ds, ts, off = [], [], [], [0]
    for w, h, t in frames:
        o, d = inputs.camera_rays(w, h)
        os_.append(o)
        ds.append(d)
        ts.append(np.full(w * h, t, np.float32))
        off.append(off[-1] + w * h)
    return (np.ascontiguousarray(np.concatenate(os_, axis=1)), np.ascontiguousarray(np.concatenate(ds, axis=1)),
            np.concatenate(ts), np.array(off, np.int64))


def get(name: str, width: int | None = None, height: int | None = None, frames=None) -> Workload:
    if name == "random_siren_64x1":
        net = random_siren_64x1()
        w = Workload(name, [net], [0.0], [32], 1e-3, None, 0, 128, 128, net)
    elif name == "nested_3level_512":
        w = Workload(name, ["s8_64x2.sdfn", "s8_128x2.sdfn", "s8_256x2.sdfn"], [0.04, 0.015, 0.005], [48, 32, 16],
                     1e-3, [1.0, 1.0, 1.0], 0, 512, 512, "s8_256x2.sdfn")
    elif name == "normal_map_1080p":
        w = Workload(name, ["s8_64x1.sdfn"], [0.04], [40], 1e-3, [1.0], 1, 1920, 1080, "s8_256x3.sdfn")
    elif name == "normal_map_1080p_c64x2":
        w = Workload(name, ["s8_64x2.sdfn"], [0.04], [40], 1e-3, [1.0], 1, 1920, 1080, "s8_256x3.sdfn")
    elif name == "normal_map_1080p_zero":
        w = Workload(name, ["s8_64x1.sdfn"], [0.0], [40], 1e-3, [1.0], 0, 1920, 1080, "s8_256x3.sdfn")
    elif name == "three_level_512":
        w = Workload(name, ["s8_64x1.sdfn", "s8_256x1.sdfn"], [0.04, 0.02], [20, 5], 1e-3, [1.0, 1.0], 1, 512, 512,
                     "s8_256x3.sdfn")
    elif name == "silhouette_512":
        w = Workload(name, ["s8_64x1.sdfn", "s8_256x2.sdfn"], [0.04, 0.01], [20, 5], 1e-3, [1.0, 1.0], 1, 512, 512,
                     "s8_256x3.sdfn")
    elif name == "animation_32":
        w = Workload(name, ["a8_64x1_t.sdfn"], [ANIM_DELTA], [40], 1e-3, [1.0], 1, 0, 0, "a8_256x3_t.sdfn")
        w.frames = animation_frames() if frames is None else frames
    elif name == "animation_32_pair":
        w = Workload(name, ["a8_64x1_t.sdfn"], [ANIM_PAIR_DELTA], [40], 1e-3, [1.0], 1, 0, 0, "a8_128x2_t.sdfn")
        w.frames = animation_frames() if frames is None else frames
    elif name == "animation_32_single":
        w = Workload(name, ["a8_256x3_t.sdfn"], [0.0], [40], 1e-3, [1.0], 0, 0, 0, "a8_256x3_t.sdfn")
        w.frames = animation_frames() if frames is None else frames
    elif name == "plain_256x3_1080p":
        w = Workload(name, ["s8_256x3.sdfn"], [0.0], [40], 1e-3, [1.0], 0, 1920, 1080, "s8_256x3.sdfn")
    else:
        raise KeyError(name)
    if width:
        w.width = width
    if height:
        w.height = height
    return w


def mesh_points(subdivisions: int = 7):
    """Displaced icosphere vertices (3, V) float32 and the fraction placed on the zero set."""
    return inputs.displaced_icosphere(inputs.sphere_scene(seed=1), subdivisions=subdivisions)
