"""FP32 + FP64 recheck on frames with long orbits: the dual-number modulus
(whose escape test ignores the dual half, so orbits near the real half's Julia
set run many steps), large constants and max_iter 16-24, plus 8-component
frames up to max_iter 32.  An FP32 sample position is rounded, and a long orbit
amplifies that difference past the recheck margin; such samples must still be
rechecked (the late-step rule), so every frame meets the whole contract
against the oracle.  Small frames on the axis slice and on random slice
frames."""
import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import binding, scenes
from parity import assert_parity, compare, to_numpy

pytestmark = pytest.mark.gpu


def frames():
    out = []
    for mi in (16, 20, 24):
        rng = np.random.default_rng(1000 + mi)
        for i in range(40):
            s = scenes.default_scene(width=64, height=48, c=[float(x) for x in rng.uniform(-0.9, 0.9, 8)],
                                     max_iter=mi, march_steps=256, bisect_steps=8,
                                     precision=scenes.PRECISION_FP32_RECHECK)
            if i % 2:
                s["slice_basis"] = scenes.random_slice_frame(rng)
            if i % 3 == 0:
                s["modulus_mode"] = scenes.MODULUS_DUALNUM
                out.append((f"dualnum_mi{mi}_{i}", s))
            elif i < 6:
                out.append((f"euclid8_mi{mi}_{i}", s))
    rng = np.random.default_rng(32)
    for i in range(4):
        s = scenes.default_scene(width=64, height=48, c=[float(x) for x in rng.uniform(-0.6, 0.6, 8)],
                                 max_iter=32, march_steps=256, bisect_steps=8, precision=scenes.PRECISION_FP32_RECHECK)
        if i % 2:
            s["slice_basis"] = scenes.random_slice_frame(rng)
        out.append((f"euclid8_mi32_{i}", s))
    return out


FRAMES = frames()


@pytest.fixture(scope="module")
def rdr():
    r = binding.Renderer(0)
    yield r
    r.close()


@pytest.mark.parametrize("name,scene", FRAMES, ids=[n for n, _ in FRAMES])
def test_long_orbits_meet_contract(rdr, name, scene):
    g = to_numpy(rdr.render(scene), scene["width"], scene["height"])
    assert_parity(compare(g, oracle.render(scene)), what=name)
