"""Per-pass CUDA-event profiling (dqj_set_profiling / dqj_pass_ms) and the FMA
throughput microbenchmark (dqj_fma_peak) on the GPU: the figures the
benchmark's roofline is built from."""
import pytest

from paper_2303_14827_gb300 import binding, scenes

pytestmark = pytest.mark.gpu


def test_pass_times_ring():
    import torch
    ctx = binding.dqj_create(0)
    try:
        s = scenes.default_scene()
        o = binding.alloc_outputs(s["width"], s["height"])
        stream = torch.cuda.current_stream().cuda_stream
        binding.dqj_set_profiling(ctx, 4)
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_pass_ms(ctx, 1)
        assert ei.value.status == binding.DQJ_ERR_NOT_FOUND
        for _ in range(6):  # the ring of 4 wraps; the 4 latest renders remain
            binding.dqj_render(ctx, s, binding.outputs_of(o), stream)
        ms = binding.dqj_pass_ms(ctx, 4)
        assert len(ms) == 4
        for march, bisect, recheck, fixup in ms:
            assert 0.0 < march < 50.0 and 0.0 <= bisect < 50.0
            assert 0.0 <= recheck < 0.05 and 0.0 <= fixup < 0.05  # FP32: no recheck passes
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_pass_ms(ctx, 5)
        assert ei.value.status == binding.DQJ_ERR_INVALID
        binding.dqj_render(ctx, dict(s, precision=scenes.PRECISION_FP32_RECHECK), binding.outputs_of(o), stream)
        (march, bisect, recheck, fixup), = binding.dqj_pass_ms(ctx, 1)
        assert march > 0.0 and recheck > 0.0 and fixup >= 0.0
        binding.dqj_set_profiling(ctx, 0)
        with pytest.raises(binding.DqjError):
            binding.dqj_pass_ms(ctx, 1)
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_set_profiling(ctx, 4097)
        assert ei.value.status == binding.DQJ_ERR_INVALID
    finally:
        binding.dqj_destroy(ctx)


def test_fma_peak_microbenchmark():
    fp32_paired = binding.dqj_fma_peak(0, 1, 2)
    fp64 = binding.dqj_fma_peak(0, 4, 2)
    assert 20e12 < fp32_paired < 200e12, fp32_paired
    assert 0.2e12 < fp64 < 20e12, fp64
    assert fp32_paired > 10 * fp64
