"""Seeded random frames across the whole parameter space, each against the
oracle on the whole contract: image sizes 8-90 x 8-70, c ~ U[-0.9, 0.9]^8,
max_iter 1-24, 1-599 march steps, 0-15 bisection steps, escape radius 2-8,
field of view 20-100 degrees, eyes inside and outside the box, random slice
frames and origins, both traversals, both squares and moduli, the specular
term, in the FP32 + FP64 recheck and all-FP64 modes."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import binding, scenes
from parity import assert_parity, compare, to_numpy

pytestmark = pytest.mark.gpu


def random_frames(seed=99, n=80):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        w, h = int(rng.integers(8, 90)), int(rng.integers(8, 70))
        s = scenes.default_scene(width=w, height=h, c=[float(x) for x in rng.uniform(-0.9, 0.9, 8)],
                                 max_iter=int(rng.integers(1, 25)), march_steps=int(rng.integers(1, 600)),
                                 bisect_steps=int(rng.integers(0, 16)))
        s["escape_radius"] = float(rng.choice([2.0, 3.0, 4.0, 8.0]))
        s["fov_y_deg"] = float(rng.uniform(20, 100))
        if rng.random() < 0.3:
            s["eye"] = [float(x) for x in rng.uniform(-2.5, 2.5, 3)] if rng.random() < 0.5 else [0.3, -0.2, 3.0]
        if rng.random() < 0.5:
            s["slice_basis"] = scenes.random_slice_frame(rng)
        if rng.random() < 0.25:
            s["slice_origin"] = [float(x) for x in rng.normal(0, 0.3, 8)]
        if rng.random() < 0.3:
            s["traversal"] = scenes.TRAVERSAL_DE
        if rng.random() < 0.25:
            s["square_mode"] = scenes.SQUARE_PAPER_COMPONENTWISE
        if rng.random() < 0.3:
            s["modulus_mode"] = scenes.MODULUS_DUALNUM
        if rng.random() < 0.2:
            s["k_specular"] = 0.4
        s["precision"] = scenes.PRECISION_FP32_RECHECK if rng.random() < 0.7 else scenes.PRECISION_FP64
        out.append((f"r{i}", s))
    return out


FRAMES = random_frames()


@pytest.fixture(scope="module")
def rdr():
    r = binding.Renderer(0)
    yield r
    r.close()


@pytest.mark.parametrize("name,scene", FRAMES, ids=[n for n, _ in FRAMES])
def test_random_frame_meets_contract(rdr, name, scene):
    g = to_numpy(rdr.render(scene), scene["width"], scene["height"])
    rep = compare(g, oracle.render(scene))
    assert_parity(rep, what=f"{name} {scene['width']}x{scene['height']} max_iter {scene['max_iter']}")
    assert rep["miss_planes_ok"], rep
    assert math.isfinite(rep["max_depth_err"])
