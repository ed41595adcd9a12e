"""Pins of the FP64 oracle's voxel-grid image (Fig. voxels: the ray-traced image
beside renders of voxel grids).

The oracle finds each pixel's first occupied cube by walking the ray cell by
cell.  It is pinned against the plain definition evaluated by brute force over
every cube (tiny grids, random occupancy, eye outside and inside the box), and
against closed forms: a full grid shows the box itself (slab entry and face),
an empty grid shows nothing, and the grid of the c = 0 ball shows the sphere
to within a cell.  No GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import scenes
from test_oracle_render import ball_radius

GAP = 1e-9  # pixels whose walk took a decision within this margin are compared only for validity


def small_scene(**over):
    # an off-axis camera: the default one looks down the z axis at a box that is
    # symmetric about it, so rays through symmetric pixels cross cell edges exactly
    base = dict(width=40, height=30, fov_y_deg=50.0, eye=[0.37, 0.23, 3.4], target=[0.05, -0.11, 0.02])
    base.update(over)
    return scenes.default_scene(**base)


@pytest.mark.parametrize("g,density,seed", [(1, 1.0, 0), (3, 0.3, 1), (5, 0.05, 2), (6, 0.2, 3), (7, 0.5, 4),
                                            (6, 0.0, 5)])
def test_walk_equals_brute_force(g, density, seed):
    rng = np.random.default_rng(seed)
    occ = (rng.random(g ** 3) < density).astype(np.uint8)
    s = small_scene()
    walk = oracle.voxel_render(s, occ)
    brute = oracle.voxel_render(s, occ, brute=True)
    ok = walk["gap"] > GAP
    assert ok.mean() > 0.99
    hw, hb = np.isfinite(walk["depth"]), np.isfinite(brute["depth"])
    assert np.array_equal(hw[ok], hb[ok])
    assert np.array_equal(walk["iter"][ok], brute["iter"][ok])
    both = ok & hw & hb
    assert np.allclose(walk["depth"][both], brute["depth"][both], rtol=0, atol=1e-12)
    assert np.array_equal(walk["normal"][both], brute["normal"][both])
    assert np.array_equal(walk["rgba"][ok], brute["rgba"][ok])
    if density > 0:
        assert hw.sum() > 0
    else:
        assert hw.sum() == 0


def test_walk_from_inside_the_box():
    rng = np.random.default_rng(8)
    g = 6
    occ = (rng.random(g ** 3) < 0.15).astype(np.uint8)
    s = small_scene(eye=[0.3, -0.2, 1.1], target=[-1.0, 0.4, -2.0])
    walk = oracle.voxel_render(s, occ)
    brute = oracle.voxel_render(s, occ, brute=True)
    ok = walk["gap"] > GAP
    assert ok.mean() > 0.99
    assert np.array_equal(walk["iter"][ok], brute["iter"][ok])
    hw = np.isfinite(walk["depth"])
    assert np.array_equal(hw[ok], np.isfinite(brute["depth"])[ok])
    both = ok & hw
    assert np.allclose(walk["depth"][both], brute["depth"][both], rtol=0, atol=1e-12)
    # the eye's own cell, when occupied, is hit at depth 0 with the fallback normal -d
    s_eye = dict(s)
    full = oracle.voxel_render(s_eye, np.ones(g ** 3, np.uint8))
    assert np.all(full["depth"] == 0.0) and np.all(full["iter"] == 1)
    o, d = oracle.camera_ray(s, 7, 9)
    assert np.allclose(full["normal"][9, 7], -d, rtol=0, atol=1e-15)


def slab(o, d, lo, hi):
    t0, t1, ax = -math.inf, math.inf, -1
    for a in range(3):
        if d[a] == 0:
            if not lo[a] <= o[a] <= hi[a]:
                return None
            continue
        ta, tb = sorted(((lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]))
        if ta > t0:
            t0, ax = ta, a
        t1 = min(t1, tb)
    return (t0, t1, ax) if max(t0, 0.0) < t1 else None


def test_full_and_empty_grid_closed_form():
    g = 9
    s = small_scene(box_min=[-1.5, -1.0, -0.5], box_max=[1.5, 1.0, 0.5])
    full = oracle.voxel_render(s, np.ones(g ** 3, np.uint8))
    empty = oracle.voxel_render(s, np.zeros(g ** 3, np.uint8))
    n_hit = 0
    for j in range(s["height"]):
        for i in range(s["width"]):
            o, d = oracle.camera_ray(s, i, j)
            r = slab(o, d, s["box_min"], s["box_max"])
            if r is None:
                assert not math.isfinite(full["depth"][j, i]) and full["iter"][j, i] == 0
                assert np.all(full["rgba"][j, i] == 0)
                continue
            n_hit += 1
            t0, _, ax = r
            assert full["depth"][j, i] == pytest.approx(t0, abs=1e-12)
            want = np.zeros(3)
            want[ax] = -np.sign(d[ax])
            assert np.array_equal(full["normal"][j, i], want)
            assert full["iter"][j, i] == 1 and full["rgba"][j, i, 3] == 255
            assert not math.isfinite(empty["depth"][j, i])
            # a ray crossing the box meets at least one cell and at most 3 g - 2
            assert 1 <= empty["iter"][j, i] <= 3 * g - 2
    assert n_hit > 300


def sphere_entry(o, d, rho):
    b = float(np.dot(o, d))
    disc = b * b - float(np.dot(o, o)) + rho * rho
    return (-b - math.sqrt(disc)) if disc > 0 else None


def test_c0_ball_grid_shows_the_sphere():
    # At c = 0 a cell is occupied when its centre lies in the ball of radius r,
    # so with h half a cell diagonal the occupied cubes cover the ball of radius
    # r - h and lie within the ball of radius r + h: a ray meeting the inner ball
    # hits between the two spheres, a ray missing the outer ball misses.
    g, W, H = 40, 48, 48
    s = scenes.default_scene(c=[0.0] * 8, max_iter=8, width=W, height=H, fov_y_deg=60.0)
    occ = oracle.voxelize(s, g)["occupancy"]
    img = oracle.voxel_render(s, occ)
    r = ball_radius(s["escape_radius"], s["max_iter"])
    h = 0.5 * math.sqrt(3.0) * 4.0 / g
    n_in = n_out = 0
    for j in range(H):
        for i in range(W):
            o, d = oracle.camera_ray(s, i, j)
            depth = img["depth"][j, i]
            t_inner, t_outer = sphere_entry(o, d, r - h), sphere_entry(o, d, r + h)
            if t_inner is not None:
                assert t_outer - 1e-12 <= depth <= t_inner + 1e-12
                n_in += 1
            elif t_outer is None:
                assert not math.isfinite(depth)
                n_out += 1
    assert n_in > 300 and n_out > 300
