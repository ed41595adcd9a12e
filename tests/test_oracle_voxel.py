"""Pins of the FP64 oracle's voxel occupancy grid (Fig. voxels): cell centres
against their definition, the c = 0 closed form (every cell's escape count is
that of |p|^(2^n) against R, so the occupied cells are the centres in the ball
|p| <= R^(2^-max_iter)), mirror symmetry for a complex c, and cell lists against
the whole grid.  No GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import scenes
from test_oracle_render import ball_radius, c0_count


def centres(s, g):
    lo, hi = np.array(s["box_min"]), np.array(s["box_max"])
    ax = [lo[a] + (np.arange(g) + 0.5) * (hi[a] - lo[a]) / g for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([x, y, z], axis=-1)  # [k, j, i, 3]


def test_cell_centres_and_index_order():
    s = scenes.default_scene(box_min=[-2.0, -1.0, 0.5], box_max=[2.0, 3.0, 1.5])
    g = 7
    cen = centres(s, g)
    rng = np.random.default_rng(0)
    for lin in rng.integers(0, g ** 3, 40):
        k, j, i = lin // (g * g), (lin // g) % g, lin % g
        assert np.allclose(oracle.voxel_center(s, g, int(lin)), cen[k, j, i], rtol=0, atol=1e-15)


@pytest.mark.parametrize("frame", ["axis", "rotated"])
def test_c0_grid_closed_form(frame):
    g = 24
    s = scenes.default_scene(c=[0.0] * 8, max_iter=6)
    if frame == "rotated":
        rng = np.random.default_rng(4)
        q, _ = np.linalg.qr(rng.normal(size=(4, 3)))
        b = np.zeros((3, 8))
        b[:, :4] = q.T
        s["slice_basis"] = b.tolist()
    out = oracle.voxelize(s, g)
    r = np.linalg.norm(centres(s, g), axis=-1)
    R, mi = s["escape_radius"], s["max_iter"]
    want = np.vectorize(lambda x: c0_count(x, R, mi))(r)
    assert np.array_equal(out["count"], want)
    assert np.array_equal(out["occupancy"], (r <= ball_radius(R, mi)).astype(np.uint8))
    assert out["occupancy"].sum() > 100
    assert out["iters"] == int(np.where(want == 0, mi, want).sum())


def test_mirror_symmetry_complex_c():
    # c in the complex plane (components 0, 1): the set is symmetric under
    # z2 -> -z2, and the grid over the symmetric box mirrors in k.
    s = scenes.default_scene(c=[-0.4, 0.6, 0, 0, 0, 0, 0, 0], max_iter=10)
    out = oracle.voxelize(s, 30)
    assert np.array_equal(out["count"], out["count"][::-1, :, :])
    assert 0 < out["occupancy"].sum() < 30 ** 3


def test_cell_list_equals_whole_grid():
    s = scenes.default_scene(max_iter=9)
    g = 16
    full = oracle.voxelize(s, g)
    cells = np.random.default_rng(2).choice(g ** 3, 300, replace=False)
    part = oracle.voxelize(s, g, cells=cells)
    assert np.array_equal(part["count"], full["count"].reshape(-1)[cells])
    assert np.array_equal(part["occupancy"], full["occupancy"].reshape(-1)[cells])
    assert math.isfinite(part["iters"]) and part["iters"] > 0
