"""Tile-shape autotuner: it records one 64-ray shape per (size class, iteration
bucket), writes a cache that a new context on the same device reads back, and
renders with the tuned shapes are identical to renders with the default shape
(every pixel's arithmetic is independent of the tiling)."""
import json

import numpy as np
import pytest

from paper_2303_14827_gb300 import binding, scenes
from parity import to_numpy

pytestmark = pytest.mark.gpu


def test_autotune_cache_roundtrip_and_results(tmp_path):
    cache = str(tmp_path / "tiles.json")
    probe = [scenes.default_scene(width=200, height=200, max_iter=mi, march_steps=512, bisect_steps=10)
             for mi in (10, 16, 24, 32)]
    with binding.Renderer(0) as plain:
        ref = [to_numpy(plain.render(s), s["width"], s["height"]) for s in probe]
    ctx = binding.dqj_create(0, autotune_cache=cache)
    try:
        binding.dqj_autotune(ctx, 2)
        data = json.load(open(cache))
        assert data["sms"] > 0 and len(data["entries"]) == 8
        for v, sc, b, tw, th in data["entries"]:
            assert v == 1 and tw * th == 64 and 0 <= sc < 2 and 0 <= b < 4
        shapes = [binding.dqj_tile_shape(ctx, s) for s in probe]
    finally:
        binding.dqj_destroy(ctx)
    ctx2 = binding.dqj_create(0, autotune_cache=cache)
    try:
        assert [binding.dqj_tile_shape(ctx2, s) for s in probe] == shapes
        import torch
        for s, r in zip(probe, ref):
            out = binding.alloc_outputs(s["width"], s["height"])
            binding.dqj_render(ctx2, s, binding.outputs_of(out), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            g = to_numpy(out, s["width"], s["height"])
            for k in ("iter", "depth", "normal", "rgba"):
                assert np.array_equal(g[k], r[k]), k
    finally:
        binding.dqj_destroy(ctx2)
