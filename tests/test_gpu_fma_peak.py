"""The FP32 FMA throughput probe reports a rate within the physical range of
the device: above a tenth of, and below 1.25x, the FP32 lanes x 2 flops x the
SM clock limit (paired instructions may count twice the lanes)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_08289_gb300 as L

    L.load_library()
    p = torch.cuda.get_device_properties(0)
    clock_ghz = 2.2   # above any sm_10x boost clock
    nominal = p.multi_processor_count * 128 * 2 * clock_ghz / 1e3   # TFLOP/s
    plain = L.lsfft_fma_peak(False, 2)
    paired = L.lsfft_fma_peak(True, 2)
    assert 0.1 * nominal < plain < 1.25 * nominal
    assert 0.1 * nominal < paired < 2.5 * nominal
