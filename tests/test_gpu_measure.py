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
