"""dqj_render_batch pipelines frames over two scratch sets and two streams (a
frame's bisection and FP64 passes run beside the next frame's march); every
frame must equal its dqj_render alone, planes and stats, whatever mix of
precisions, traversals, slices and sizes the batch holds, and the context's
later renders must stay ordered after it.  dqj_render_host_batch takes the
same pipeline for n > 1."""
import numpy as np
import pytest
import torch

from paper_2303_14827_gb300 import binding, scenes

pytestmark = pytest.mark.gpu

PLANES = ("iter", "depth", "normal", "rgba", "stats")


def mixed_batch():
    rng = np.random.default_rng(5)
    return [
        scenes.full_hd_scene(3, precision=scenes.PRECISION_FP32_RECHECK),
        scenes.default_scene(),  # small frame: split march, four lanes per hit
        scenes.default_scene(width=333, height=211, precision=scenes.PRECISION_FP32_RECHECK),
        scenes.default_scene(width=200, height=150, precision=scenes.PRECISION_FP64),
        scenes.default_scene(width=160, height=120, traversal=scenes.TRAVERSAL_DE,
                             precision=scenes.PRECISION_FP32_RECHECK),
        scenes.default_scene(width=301, height=177, slice_basis=scenes.random_slice_frame(rng)),
        scenes.full_hd_scene(0, precision=scenes.PRECISION_FP32_RECHECK),
    ]


def host(o, w):
    return {k: (o[k] if k == "stats" else o[k][:, :w]).cpu().numpy() for k in PLANES}


def test_batch_equals_single_renders():
    frames = mixed_batch()
    ctx = binding.dqj_create(0)
    try:
        st = torch.cuda.current_stream()
        ref = []
        for s in frames:
            o = binding.alloc_outputs(s["width"], s["height"])
            binding.dqj_render(ctx, s, binding.outputs_of(o), st.cuda_stream)
            st.synchronize()
            ref.append(host(o, s["width"]))
        for rep in range(2):  # the second batch reuses the grown scratch sets
            outs = [binding.alloc_outputs(s["width"], s["height"]) for s in frames]
            for o in outs:
                for k in ("iter", "normal", "rgba"):
                    o[k].fill_(3)
                o["depth"].fill_(3.0)
            binding.dqj_render_batch(ctx, frames, [binding.outputs_of(o) for o in outs], st.cuda_stream)
            st.synchronize()
            for i, (s, o) in enumerate(zip(frames, outs)):
                got = host(o, s["width"])
                for k in PLANES:
                    assert np.array_equal(got[k], ref[i][k], equal_nan=True), (rep, i, k)
    finally:
        binding.dqj_destroy(ctx)


def test_later_render_is_ordered_after_the_batch():
    """A dqj_render on another stream right after a batch shares the batch's
    scratch; it must run after the batch, so its own result is exact."""
    frames = [scenes.full_hd_scene(k, precision=scenes.PRECISION_FP32_RECHECK) for k in range(3)]
    other = scenes.default_scene(width=640, height=480, precision=scenes.PRECISION_FP32_RECHECK)
    ctx = binding.dqj_create(0)
    try:
        st = torch.cuda.current_stream()
        alone = binding.alloc_outputs(640, 480)
        binding.dqj_render(ctx, other, binding.outputs_of(alone), st.cuda_stream)
        st.synchronize()
        want = host(alone, 640)
        outs = [binding.alloc_outputs(1920, 1080) for _ in frames]
        side = torch.cuda.Stream()
        o2 = binding.alloc_outputs(640, 480)
        binding.dqj_render_batch(ctx, frames, [binding.outputs_of(o) for o in outs], st.cuda_stream)
        binding.dqj_render(ctx, other, binding.outputs_of(o2), side.cuda_stream)
        torch.cuda.synchronize()
        got = host(o2, 640)
        for k in PLANES:
            assert np.array_equal(got[k], want[k], equal_nan=True), k
    finally:
        binding.dqj_destroy(ctx)


def test_host_batch_equals_device_renders():
    frames = mixed_batch()[:5]
    ctx = binding.dqj_create(0)
    try:
        st = torch.cuda.current_stream()
        ref = []
        for s in frames:
            o = binding.alloc_outputs(s["width"], s["height"])
            binding.dqj_render(ctx, s, binding.outputs_of(o), st.cuda_stream)
            st.synchronize()
            ref.append(host(o, s["width"]))
        hosts = [binding.alloc_outputs(s["width"], s["height"], device="cpu") for s in frames]
        for h in hosts:
            for k in PLANES:
                h[k] = h[k].pin_memory()
        binding.dqj_render_host_batch(ctx, frames, [binding.outputs_of(h) for h in hosts])
        for i, (s, h) in enumerate(zip(frames, hosts)):
            got = host(h, s["width"])
            for k in PLANES:
                assert np.array_equal(got[k], ref[i][k], equal_nan=True), (i, k)
    finally:
        binding.dqj_destroy(ctx)
