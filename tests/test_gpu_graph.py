"""dqj_render captured in a CUDA graph (torch.cuda.CUDAGraph): after a warm-up
render sizes the context's scratch, a sequence of renders is captured and
replayed; every replay's images and counters equal the plain renders'.  The
recheck mode is included (under capture it clears its per-pixel tags per
frame), and a capture on a context whose scratch is too small is refused
before any CUDA work."""
import numpy as np
import pytest

from paper_2303_14827_gb300 import binding, scenes
from parity import to_numpy

pytestmark = pytest.mark.gpu


def scenes_for(prec):
    return [scenes.default_scene(width=160, height=120, precision=prec),
            scenes.default_scene(c=list(scenes.PAPER_C_VALUES["highres"]), width=160, height=120, max_iter=15,
                                 precision=prec),
            scenes.default_scene(width=96, height=64, max_iter=9, precision=prec)]


@pytest.mark.parametrize("prec", [scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK])
def test_captured_renders_replay_equal(prec):
    import torch
    frames = scenes_for(prec)
    with binding.Renderer(0) as plain:
        ref = [to_numpy(plain.render(s), s["width"], s["height"]) for s in frames]
        ref_stats = [binding.stats_dict(plain.render(s)["stats"]) for s in frames]
    ctx = binding.dqj_create(0)
    try:
        outs = [binding.alloc_outputs(s["width"], s["height"]) for s in frames]
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            binding.dqj_render(ctx, frames[0], binding.outputs_of(outs[0]), st.cuda_stream)  # sizes the scratch
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for s, o in zip(frames, outs):
                binding.dqj_render(ctx, s, binding.outputs_of(o), st.cuda_stream)
        for rep in range(2):
            for o in outs:
                o["iter"].fill_(-5)
                o["stats"].fill_(-5)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            for s, o, r, rs in zip(frames, outs, ref, ref_stats):
                got = to_numpy(o, s["width"], s["height"])
                for k in ("iter", "depth", "normal", "rgba"):
                    assert np.array_equal(got[k], r[k]), (rep, k)
                assert binding.stats_dict(o["stats"]) == rs
        del g  # a graph holding renders goes before its context
        torch.cuda.synchronize()
        # ordinary renders on the same context after the capture
        for s, o, r in zip(frames, outs, ref):
            binding.dqj_render(ctx, s, binding.outputs_of(o), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = to_numpy(o, s["width"], s["height"])
            assert all(np.array_equal(got[k], r[k]) for k in ("iter", "depth", "normal", "rgba"))
    finally:
        binding.dqj_destroy(ctx)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # the refused render adds no work to the graph
def test_capture_refused_without_scratch():
    import torch
    ctx = binding.dqj_create(0)
    try:
        s = scenes.default_scene(width=64, height=48)
        o = binding.alloc_outputs(64, 48)
        torch.cuda.synchronize()
        st = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            with pytest.raises(binding.DqjError) as ei:
                binding.dqj_render(ctx, s, binding.outputs_of(o), st.cuda_stream)
            assert ei.value.status == binding.DQJ_ERR_INVALID and "capture" in binding.last_error()
        del g
        torch.cuda.synchronize()
    finally:
        binding.dqj_destroy(ctx)
