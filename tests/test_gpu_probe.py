"""The pipe-throughput probe (lisa_probe_pipes) that the bench line reports beside the
derived FP64 / FP32 peaks: rates of the right order for the device and the FP32:FP64
ratio of a part whose FP64 pipe is a small fraction of its FP32 pipe."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2005_01827_gb300 import build

    build.build()
    from paper_2005_01827_gb300 import lisalike

    r = lisalike.probe_pipes(0)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    clk = r["sm_clock_hz"]
    assert 5e8 < clk < 4e9
    fp64_per_sm_clk = r["fp64_fma_per_s"] / (nsm * clk)
    fp32_per_sm_clk = r["fp32_fma_per_s"] / (nsm * clk)
    print("per SM per clock: FP64 FMA %.2f, FP32 FMA %.1f, MUFU %.1f"
          % (fp64_per_sm_clk, fp32_per_sm_clk, r["mufu_per_s"] / (nsm * clk)))
    assert 0.5 < fp64_per_sm_clk < 80
    assert 30 < fp32_per_sm_clk < 160
    assert 4 < r["mufu_per_s"] / (nsm * clk) < 40
