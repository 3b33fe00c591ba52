"""FP64 and FP32 FMA throughput of the GPU, measured by the library's probe
(gw_fma_rate): the per-clock rates behind the roofline fractions of the point
kernels.  Prints the measured rates; asserts only what the hardware allows
(at most 128 FP32 lanes per SM, each doing up to two FMAs per clock with packed
FP32x2 instructions; FP64 at a small fraction of FP32 on this part) and that the SM clock seen by the cycle counter over the CUDA
events' time is a plausible one."""
import pytest
import torch

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def test_fma_rates():
    r64 = gw.gw_fma_rate(True)
    r32 = gw.gw_fma_rate(False)
    sms = r32["sms"]
    print(f"\nSMs {sms}; FP64 {r64['fma_per_clk_sm']:.2f} FMA/clk/SM "
          f"({2 * r64['fma_per_s'] / 1e12:.3f} TFLOP/s at {r64['sm_mhz']:.0f} MHz); "
          f"FP32 {r32['fma_per_clk_sm']:.1f} FMA/clk/SM "
          f"({2 * r32['fma_per_s'] / 1e12:.2f} TFLOP/s at {r32['sm_mhz']:.0f} MHz)")
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    assert 32.0 <= r32["fma_per_clk_sm"] <= 256.0 * 1.02
    assert 0.5 <= r64["fma_per_clk_sm"] <= r32["fma_per_clk_sm"]
    for r in (r32, r64):
        assert 300.0 <= r["sm_mhz"] <= 3000.0
