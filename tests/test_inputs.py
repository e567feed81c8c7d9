"""Seeded input generators: published test vectors and geometric invariants."""
import numpy as np

from paper_2201_09147_gb300 import inputs, workloads


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea and Flood 2014; Vigna's reference code)
    assert [int(x) for x in inputs.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = inputs.uniform01(0, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def test_stream_offsets_are_consistent():
    assert np.array_equal(inputs.splitmix64(7, 10)[5:], inputs.splitmix64(7, 5, start=5))


def test_siren_init_bounds_and_determinism():
    a = inputs.siren_init(0, 64, 1)
    b = inputs.siren_init(0, 64, 1)
    assert all(np.array_equal(x, y) for x, y in zip(a.weights, b.weights))
    assert np.abs(a.weights[0]).max() <= 1 / 3
    c = np.sqrt(6 / 64) / 30
    assert np.abs(a.weights[1]).max() <= c and np.abs(a.weights[2]).max() <= c
    assert a.n_params() == inputs.param_count(3, 64, 1) == 4481


def test_camera_rays_unit_and_centred():
    o, d = inputs.camera_rays(64, 48)
    assert o.shape == (3, 64 * 48) and o.dtype == np.float32
    assert np.allclose(np.linalg.norm(d.astype(np.float64), axis=0), 1.0, atol=1e-6)
    assert np.allclose(o[:, 0], [0, 0, 2.5])
    # symmetric image: the mean direction points down -z
    m = d.astype(np.float64).mean(axis=1)
    assert abs(m[0]) < 1e-6 and abs(m[1]) < 1e-6 and m[2] < -0.9
    # row 0 is the top of the image, column 0 the left
    assert d[1, 0] > 0 and d[0, 0] < 0
    # half the vertical field of view is 22.5 degrees at the image edge
    top = np.degrees(np.arctan2(d[1, :64], -d[2, :64]))
    assert np.allclose(top, np.degrees(np.arctan(np.tan(np.radians(22.5)) * 47 / 48)), atol=1e-4)


def test_icosphere_counts_and_radius():
    for s in range(4):
        v = inputs.icosphere(s)
        assert v.shape[0] == 10 * 4 ** s + 2
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    assert 10 * 4 ** 7 + 2 == 163842


def test_scene_draws_and_field():
    sc = inputs.sphere_scene(1)
    assert sc.centres.shape == (8, 3) and np.all(np.abs(sc.centres) <= 0.6)
    assert np.all((sc.radii >= 0.15) & (sc.radii <= 0.3))
    # the field is negative at a centre, positive far away
    assert sc.g(sc.centres[:1])[0] < 0
    assert sc.g(np.array([[3.0, 3.0, 3.0]]))[0] > 0


def test_displaced_icosphere_on_zero_set():
    sc = inputs.sphere_scene(1)
    pts, frac = inputs.displaced_icosphere(sc, subdivisions=2)
    assert pts.shape == (3, 162)
    assert frac > 0.5
    g = sc.g(pts.T.astype(np.float64))
    on = np.abs(g) < 1e-5
    assert on.mean() >= frac - 1e-9


def test_workloads_resolve():
    for name in ("random_siren_64x1", "nested_3level_512", "normal_map_1080p", "plain_256x3_1080p"):
        w = workloads.get(name)
        assert len(w.level_bytes()) == len(w.delta) == len(w.caps)
        w.fine_bytes()
    assert workloads.get("normal_map_1080p").n_rays == 2073600


def test_scene_gradient_and_fit_batch():
    """The analytic scene gradient is the derivative of g (central differences); the fit
    batch is half near-surface, half uniform, with targets equal to g there."""
    sc = inputs.sphere_scene(1)
    p, tf, tg, near = inputs.fit_batch(sc, 0, 2000)
    assert p.shape == (3, 2000) and near.sum() == 1000 and p.dtype == np.float32
    P = p.T.astype(np.float64)[::97]
    v, g = sc.value_and_grad(P)
    h = 1e-6
    fd = np.stack([(sc.g(P + h * np.eye(3)[c]) - sc.g(P - h * np.eye(3)[c])) / (2 * h) for c in range(3)], axis=1)
    assert np.abs(fd - g).max() < 1e-6
    assert np.array_equal(v, sc.g(P))
    assert np.abs(tf[:1000]).mean() < 0.05 < np.abs(tf[1000:]).mean()
