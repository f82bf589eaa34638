"""The FP32 probe (lbm_probe_fp32) that gives the instruction side of the roofline.

Its FMA kernels must run at a rate the GB300's arithmetic units allow: 152 SMs x 128 FP32
lanes x 2 flops per FMA at an SM clock between 0.8 and 2.1 GHz (31-82 TFLOP/s for scalar
FFMA), at most one warp instruction per cycle per SM sub-partition, and the paired form
(two FMAs per instruction) no slower than the scalar one."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_probe_measures_a_plausible_rate(lbm_lib):
    import torch
    r = lbm_lib.lbm_probe_fp32(torch.cuda.current_stream().cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lanes_flops_per_cycle = sms * 128 * 2
    assert 0.8e9 * lanes_flops_per_cycle * 0.9 / 1e12 < r["ffma_tflops"] < 2.1e9 * lanes_flops_per_cycle / 1e12
    assert r["warp_ffma_per_s_per_smsp"] < 2.1e9
    assert r["ffma2_tflops"] > 0.9 * r["ffma_tflops"]
    assert r["ms"] > 1.0
