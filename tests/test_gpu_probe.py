"""The multiply-add rate probe the ALU roofline is read against."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04374_gb300 import api  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def test_fma_probe_is_near_the_pipes_nominal_rates():
    """GB300: 152 SMs x 128 FP32 lanes x 2 flops x <= 2.07 GHz = 80.5 TFLOP/s;
    FP64 is far slower (nominal 1.25 TFLOP/s).  The probe must land within a
    factor of two of those (clocks vary with load and power)."""
    f32 = api.probe_fma_tflops("fp32")
    f64 = api.probe_fma_tflops("fp64")
    assert 40.0 < f32 < 85.0, f32
    assert 0.3 < f64 < 5.0, f64
    assert f32 > 10 * f64
