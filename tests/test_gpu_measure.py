"""Measurement helpers: the sine-rate microbenchmark the trace kernel's roofline uses."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_sine_rate_is_near_the_nominal_sfu_rate(sdf):
    r = sdf.measure_sine_rate(0)
    props = torch.cuda.get_device_properties(0)
    # 16 hardware sines per clock per SM at 1.0-2.2 GHz
    lo, hi = props.multi_processor_count * 16 * 1.0e9, props.multi_processor_count * 16 * 2.2e9
    print("Gsin/s", r / 1e9)
    assert 0.5 * lo <= r <= 1.2 * hi


# Absolute error bounds of the kernels' sine and cosine against FP64 at FP32 arguments (the paper is
# silent on sine accuracy).  FP32 path: the hardware approximation on [-pi, pi] after reduction by
# 2 pi; the reduced argument carries one rounding (<= 1.2e-7 at |r| <= pi), the approximation's
# own error is below 4e-7: bound 5e-7 over |x| <= 256.  Tensor-core paths: the hardware
# approximation applied to x directly; its error grows with |x| (it scales x by 1/(2 pi) in
# reduced precision): bounds 8.7e-6 over |x| <= 64 and 3.5e-5 over |x| <= 256.  Both stay far
# below the 16-bit operand roundings (4e-3 BF16, 5e-4 FP16) the tensor-core paths store sines in.
SINE_BOUNDS = {0: ((256.0, 5e-7),), 1: ((64.0, 8.7e-6), (256.0, 3.5e-5))}


@pytest.mark.parametrize("variant", [0, 1], ids=["fp32_path", "tensor_core_paths"])
def test_sine_cosine_accuracy_sweep(sdf, variant):
    """A dense sweep of |x| <= 256 (2^24 evenly spaced floats, the float neighbours of multiples
    of pi / 2 and 2^20 seeded uniform arguments) against numpy's FP64 sin / cos."""
    import numpy as np

    from paper_2201_09147_gb300 import inputs
    grid = np.linspace(-256.0, 256.0, 1 << 24, dtype=np.float32)
    k = np.arange(-163, 164, dtype=np.float64) * (np.pi / 2)
    near_k = np.concatenate([np.nextafter(k.astype(np.float32), s) for s in (-np.inf, np.inf)] + [k.astype(np.float32)])
    rnd = (inputs.uniform01(5, 1 << 20) * 512.0 - 256.0).astype(np.float32)
    x = np.concatenate([grid, near_k, rnd, np.array([0.0, -0.0, 256.0, -256.0], np.float32)])
    s, c = sdf.eval_sine(torch.from_numpy(x).cuda(), variant)
    s, c = s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)
    assert not np.isnan(s).any()  # the trace kernels' sine is the value returned here
    xd = x.astype(np.float64)
    es, ec = np.abs(s - np.sin(xd)), np.abs(c - np.cos(xd))
    for lim, bound in SINE_BOUNDS[variant]:
        sel = np.abs(xd) <= lim
        print(f"variant {variant} |x| <= {lim}: max |sin err| {es[sel].max():.3g}, max |cos err| {ec[sel].max():.3g}")
        assert es[sel].max() <= bound and ec[sel].max() <= bound
