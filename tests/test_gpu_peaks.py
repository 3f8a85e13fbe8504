"""The library's microbenchmarks of on-chip peaks (wake_measure_peaks):
each rate must be positive and within what the GPU's unit counts allow at
the clock it reports (a microbenchmark that timed nothing, or that the
compiler emptied, would read far above)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_physical():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2603_16623_gb300 import wake
    p = wake.measure_peaks()
    sms, f = p["sms"], p["sm_clock_mhz"] * 1e6
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    assert 500e6 < f < 3e9, p
    # per SM and clock: 128 FP32 lanes (2 flop per FMA), 16 MUFU, 128 B of
    # shared memory; a little above for clock drift between kernels
    assert 0.3 < p["fp32_tflops"] * 1e12 / (sms * f * 256) < 1.1, p
    assert 0 < p["fp64_tflops"] < p["fp32_tflops"], p
    assert 0.2 < p["mufu_lg2_tops"] * 1e12 / (sms * f * 16) < 1.1, p
    assert 0.2 < p["smem_tbs"] * 1e12 / (sms * f * 128) < 1.1, p
    assert 2 <= p["fma_latency_cycles"] < 20, p
    assert 5 < p["syncthreads_cycles"] < 2000, p
    assert p["syncthreads_cycles"] < p["cluster_barrier_cycles"] < 20000, p
