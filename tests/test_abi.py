"""The C ABI: the library builds, loads and exports every declared symbol.

No compute call is made here (no GPU); host-side validation that runs before
any device work is exercised through the loader.
"""
import ctypes as C
import re
from pathlib import Path

import pytest

from paper_2201_09147_gb300 import build, inputs

HEADER = Path(__file__).resolve().parents[1] / "include" / "sdfnn.h"


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(sdf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return C.CDLL(str(build.build()))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2201_09147_gb300 import sdfnn
    assert sorted(sdfnn.EXPORTS) == declared_functions()


def test_loader_rejects_malformed_images_without_a_gpu(lib):
    lib.sdf_net_load_mem.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
    lib.sdf_last_error.restype = C.c_char_p
    h = C.c_void_p(1)
    good = inputs.net_to_bytes(inputs.siren_init(0, 64, 1))
    assert lib.sdf_net_load_mem(b"nope", 4, 1, 0, C.byref(h)) == -3 and h.value is None
    assert lib.sdf_net_load_mem(good[:-4], len(good) - 4, 1, 0, C.byref(h)) == -3
    assert lib.sdf_net_load_mem(good, len(good), 2, 0, C.byref(h)) == -7   # E4M3 needs width >= 128
    w256 = inputs.net_to_bytes(inputs.siren_init(0, 256, 2))
    # E4M3 quantisation and calibration run on the host; without a GPU the device check then fails
    assert lib.sdf_net_load_mem(w256, len(w256), 2, 0, C.byref(h)) == -1 and h.value is None
    assert lib.sdf_net_load_mem(good, len(good), 9, 0, C.byref(h)) == -1   # unknown precision
    assert lib.sdf_net_load_mem(None, 0, 1, 0, C.byref(h)) == -1
    bad = bytearray(good)
    bad[36:40] = bytes([0, 0, 0xC0, 0x7F])  # NaN in W_0
    assert lib.sdf_net_load_mem(bytes(bad), len(bad), 1, 0, C.byref(h)) == -5
    wide = inputs.net_to_bytes(inputs.siren_init(0, 96, 1))
    assert lib.sdf_net_load_mem(wide, len(wide), 0, 0, C.byref(h)) == -7
    lib.sdf_net_load.argtypes = [C.c_char_p, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
    assert lib.sdf_net_load(b"/nonexistent/file.sdfn", 1, 0, C.byref(h)) == -2
    assert len(lib.sdf_last_error()) > 0


def test_null_arguments_are_rejected(lib):
    lib.sdf_trace_multiscale.argtypes = [C.c_void_p] * 4 + [C.c_void_p] * 5
    lib.sdf_trace_multiscale.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.sdf_trace_multiscale(None, None, None, 0, None, None, None, None, None) == -1
    lib.sdf_normals.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    assert lib.sdf_normals(None, None, 0, None, None) == -1
    lib.sdf_net_free.argtypes = [C.c_void_p]
    lib.sdf_net_free(None)
    lib.sdf_normal_map_timed.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_void_p, C.c_void_p]
    assert lib.sdf_normal_map_timed(None, None, None, None, 0, None, None) == -1
    # plans: NULL handles and arguments fail before any device work
    h = C.c_void_p(1)
    lib.sdf_plan_create.argtypes = [C.c_void_p] * 3 + [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
    assert lib.sdf_plan_create(None, None, None, 0, None, C.byref(h)) == -1 and h.value is None
    assert lib.sdf_plan_create(None, None, None, 0, None, None) == -1
    lib.sdf_plan_launch.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.sdf_plan_launch(None, None) == -1
    lib.sdf_plan_info.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    assert lib.sdf_plan_info(None, None, 0, None) == -1
    lib.sdf_plan_free.argtypes = [C.c_void_p]
    lib.sdf_plan_free(None)
    # frame queues likewise
    lib.sdf_frame_queue_create.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_void_p)]
    assert lib.sdf_frame_queue_create(None, None, 16, 2, C.byref(h)) == -1 and h.value is None
    assert lib.sdf_frame_queue_create(None, None, 16, 2, None) == -1
    lib.sdf_frame_queue_submit.argtypes = [C.c_void_p] * 6 + [C.c_void_p]
    assert lib.sdf_frame_queue_submit(None, None, None, None, None, None, None) == -1
    lib.sdf_frame_queue_wait.argtypes = [C.c_void_p, C.c_int64]
    assert lib.sdf_frame_queue_wait(None, -1) == -1
    lib.sdf_frame_queue_free.argtypes = [C.c_void_p]
    lib.sdf_frame_queue_free(None)


def test_training_shapes_and_null_arguments(lib):
    from paper_2201_09147_gb300 import sdfnn
    for in_dim, w, k in ((3, 64, 1), (4, 128, 2), (3, 256, 3)):
        count, ws = sdfnn.train_shape_info(in_dim, w, k, 1000)
        assert count == inputs.param_count(in_dim, w, k)
        # transposed weights, A_0, and two (k, n, 4, w) float blocks
        assert ws >= 4 * (k * w * w + 1000 * w + 2 * k * 1000 * 4 * w)
    with pytest.raises(sdfnn.SdfError) as e:
        sdfnn.train_shape_info(3, 96, 1)
    assert e.value.code == -7
    lib.sdf_train_forward.argtypes = [C.c_int] * 4 + [C.c_void_p] * 3 + [C.c_int64] + [C.c_void_p] * 4
    assert lib.sdf_train_forward(0, 3, 64, 1, None, None, None, 0, None, None, None, None) == -1
    assert lib.sdf_train_forward(1, 3, 64, 1, None, None, None, 0, None, None, None, None) == -1
    assert lib.sdf_train_forward(2, 3, 64, 1, None, None, None, 0, None, None, None, None) == -7  # no E4M3 training
    # the 16-bit workspace: (1 + 5k) w floats per point plus two 16-bit weight images (2 x 384 KB)
    _, ws16 = sdfnn.train_shape_info(3, 256, 3, 1 << 20, sdfnn.SDF_BF16)
    _, ws32 = sdfnn.train_shape_info(3, 256, 3, 1 << 20, sdfnn.SDF_FP32)
    per_point = 4 * (1 << 20) * 256 * (1 + 5 * 3)
    assert per_point <= ws16 < per_point + 2 * 384 * 1024 + 4096 and ws16 < 0.8 * ws32
    lib.sdf_adam_step.argtypes = [C.c_void_p] * 4 + [C.c_int64] + [C.c_float] * 4 + [C.c_int, C.c_void_p]
    assert lib.sdf_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == -1  # step from 1


def test_theta_roundtrip_through_sdfn():
    """The folded parameter vector and its SDFN image describe the same network."""
    import numpy as np
    import oracle
    from paper_2201_09147_gb300 import sdfnn
    net = inputs.siren_init(9, 64, 2)
    b = inputs.net_to_bytes(net)
    shape, theta = sdfnn.theta_from_sdfn(b)
    assert shape == (3, 64, 2) and theta.size == inputs.param_count(3, 64, 2)
    b2 = sdfnn.sdfn_from_theta(shape, theta)
    assert sdfnn.theta_from_sdfn(b2)[1].tobytes() == theta.tobytes()
    pts = inputs.random_points(2, 50).astype(np.float64)
    g1, v1 = oracle.Net(b).grad_batch(pts, with_value=True)
    g2, v2 = oracle.Net(b2).grad_batch(pts, with_value=True)
    assert np.allclose(v1, v2, rtol=1e-5, atol=1e-5) and np.allclose(g1, g2, rtol=1e-4, atol=1e-3)


def test_selftest_argument_check_without_a_gpu(lib):
    lib.sdf_selftest_wait_timeout.argtypes = [C.c_int, C.c_int64, C.c_void_p]
    assert lib.sdf_selftest_wait_timeout(0, 0, None) == -1
    assert lib.sdf_selftest_wait_timeout(0, 10 ** 8, None) == -1
    lib.sdf_selftest_noalloc_timeout.argtypes = [C.c_int, C.c_int64, C.c_void_p]
    assert lib.sdf_selftest_noalloc_timeout(0, 0, None) == -1


def test_theta_from_image_folds_the_frequencies():
    """sdf_theta_from_image (host only) multiplies omega0 into layer 0 and omega into the hidden
    layers (Eq. 2 as plain sin(W x + b)) and leaves the output row; a folded image passes through."""
    import numpy as np
    from paper_2201_09147_gb300 import sdfnn
    net = inputs.siren_init(4, 64, 2)
    b = inputs.net_to_bytes(net)
    shape, theta = sdfnn.theta_from_sdfn(b)
    raw = np.frombuffer(b[32:], "<f4").astype(np.float64)
    w, k = 64, 2
    n0 = w * 3 + w
    per = w * w + w
    expect = raw.copy()
    expect[:n0] *= 30.0
    expect[n0:n0 + k * per] *= 30.0
    assert shape == (3, 64, 2)
    assert np.array_equal(theta, expect.astype(np.float32))
    assert np.array_equal(sdfnn.theta_from_sdfn(sdfnn.sdfn_from_theta(shape, theta))[1], theta)
    with pytest.raises(sdfnn.SdfError) as e:
        sdfnn.theta_from_sdfn(b[:-4])
    assert e.value.code == -3
    small = np.empty(10, np.float32)
    assert sdfnn.lib().sdf_theta_from_image(b, len(b), C.c_void_p(small.ctypes.data), 10, None, None, None,
                                            None) == -1
