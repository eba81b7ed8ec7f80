"""sr_measure_alu_peaks: the measured instruction-throughput roofs of the
blend loops (FP32 FMA, packed FP32x2 FMA, FP32 min/max, ex2, rcp) are
positive, finite and ordered as the hardware's units are (the multi-function
unit is slower than the FMA pipe), and the FMA rate lies within the range
that 128 FP32 lanes per SM at the GPU's clock range allow."""
import pytest
import torch

from paper_2605_18334_gb300 import native as N

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_measured_alu_peaks_are_plausible():
    sink = torch.zeros(32, dtype=torch.float32, device="cuda")
    p = N.sr_measure_alu_peaks(sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print("alu peaks (per SM per clock at 2070 MHz): " +
          " ".join(f"{k}={v / (sms * 2.07e9):.2f}" for k, v in p.items() if k != "seconds") +
          f" seconds={p['seconds']:.3f}")
    for k, v in p.items():
        assert v > 0 and v < float("inf"), k
    lanes_at_max_clock = sms * 128 * 2.07e9
    assert 0.3 * lanes_at_max_clock < p["fma_lane_ops_per_s"] < 1.05 * lanes_at_max_clock
    assert p["ex2_per_s"] < p["fma_lane_ops_per_s"] and p["rcp_per_s"] < p["fma_lane_ops_per_s"]
    assert float(sink.abs().sum()) == 0.0  # the sink is never written
