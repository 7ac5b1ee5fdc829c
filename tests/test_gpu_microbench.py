"""The device's FMA throughput measurement (rism3d_fma_rate) behind the FP64 form's
arithmetic roofline: finite, positive, FP32 above FP64, and refused for other precisions."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()


def test_fma_rates():
    r32, r64 = capi.fma_rate(32), capi.fma_rate(64)
    assert 1e12 < r32 < 1e15 and 1e10 < r64 < 1e15 and r32 > r64, (r32, r64)
    with pytest.raises(capi.RismError):
        capi.fma_rate(16)
