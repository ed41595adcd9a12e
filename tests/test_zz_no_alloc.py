"""dqj_render_noalloc, the render entry point that allocates nothing, checked
through the C ABI against dqj_render on the same scenes.  It serves callers that
must not allocate device memory: a host application that has reserved the
device's memory for its own pool, or a frame loop that must not block on the
allocator; its scratch is a fixed array inside the library.  Both run the same kernels, so their outputs must
agree exactly; two different scenes are rendered back to back through the fixed
scratch array to show that each call starts from cleared counters.  This file
sorts last so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

from paper_2303_14827_gb300 import binding, scenes
from parity import to_numpy

pytestmark = pytest.mark.gpu


def _both(rdr, s):
    import torch
    ref = rdr.render(s)
    out = binding.alloc_outputs(s["width"], s["height"])
    stream = torch.cuda.current_stream()
    binding.dqj_render_noalloc(s, binding.outputs_of(out), stream.cuda_stream)
    stream.synchronize()
    return ref, out


def test_noalloc_matches_render_twice():
    import torch
    assert torch.cuda.is_available()
    with binding.Renderer(0) as rdr:
        cases = [scenes.default_scene(width=200, height=144),
                 scenes.default_scene(c=list(scenes.PAPER_C_VALUES["highres"]), width=512, height=512, max_iter=15)]
        for s in cases:  # two calls in a row through the shared scratch
            ref, out = _both(rdr, s)
            a, b = to_numpy(ref, s["width"], s["height"]), to_numpy(out, s["width"], s["height"])
            for k in ("iter", "depth", "normal", "rgba"):
                assert np.array_equal(a[k], b[k]), k
            assert binding.stats_dict(ref["stats"]) == binding.stats_dict(out["stats"])
            assert binding.stats_dict(out["stats"])["hits"] > 0


def test_noalloc_fp64_and_limits():
    import torch
    with binding.Renderer(0) as rdr:
        s = scenes.default_scene(width=96, height=64, precision=scenes.PRECISION_FP64)
        ref, out = _both(rdr, s)
        a, b = to_numpy(ref, 96, 64), to_numpy(out, 96, 64)
        for k in ("iter", "depth", "normal", "rgba"):
            assert np.array_equal(a[k], b[k]), k
    big = scenes.default_scene(width=1024, height=1024)
    no_planes = binding.make_outputs(pitch_px=1024)
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_render_noalloc(big, no_planes, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == binding.DQJ_ERR_INVALID and "DQJ_NOALLOC_MAX_PIXELS" in str(ei.value)
    with pytest.raises(binding.DqjError) as ei:
        binding.dqj_render_noalloc(scenes.default_scene(precision=scenes.PRECISION_FP32_RECHECK),
                                   binding.make_outputs(pitch_px=256), 0)
    assert ei.value.status == binding.DQJ_ERR_INVALID and "DQJ_FP64 only" in str(ei.value)


def test_noalloc_distance_estimate_traversal_and_no_allocation():
    """The sphere-tracing traversal through the fixed array equals dqj_render, and
    a call after a warm-up of the same kind changes neither the device's free
    memory nor torch's allocations: the entry point allocates nothing.  (The
    warm-up comes first because under lazy module loading the first launch of a
    kernel loads its code.)"""
    import torch
    with binding.Renderer(0) as rdr:
        s = scenes.default_scene(width=160, height=120, traversal=scenes.TRAVERSAL_DE)
        ref, out = _both(rdr, s)
        a, b = to_numpy(ref, 160, 120), to_numpy(out, 160, 120)
        for k in ("iter", "depth", "normal", "rgba"):
            assert np.array_equal(a[k], b[k]), k
        assert binding.stats_dict(ref["stats"]) == binding.stats_dict(out["stats"])
        march = scenes.default_scene(width=200, height=144)
        o2 = binding.alloc_outputs(200, 144)
        stream = torch.cuda.current_stream()
        for sc, o in ((s, out), (march, o2)):  # warm-up of both kinds
            binding.dqj_render_noalloc(sc, binding.outputs_of(o), stream.cuda_stream)
        torch.cuda.synchronize()
        free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        for sc, o in ((s, out), (march, o2)):
            binding.dqj_render_noalloc(sc, binding.outputs_of(o), stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == torch0
