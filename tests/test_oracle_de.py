"""Pins of the FP64 oracle's distance-estimate sphere tracing (Method,
"Ray-Marching", Eq. distfract2).

At c = 0 every iterate is a power of the start point: |zeta_n| = |p|^(2^n) and
the derivative recurrence gives |zeta'_n| = 2^n |p|^(2^n - 1), so the estimate is
0.5 |p| ln |p| whatever the escape step.  It is a lower bound of the distance
|p| - 1 to the unit sphere, so sphere tracing never crosses that sphere and
stops between it and the sphere where the estimate equals epsilon.  No GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import scenes
from test_oracle_render import c0_count


def de_scene(**over):
    base = dict(traversal=scenes.TRAVERSAL_DE, de_epsilon=1e-3, de_max_steps=512)
    base.update(over)
    return scenes.default_scene(**base)


def rotated_basis(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(4, 3)))
    b = np.zeros((3, 8))
    b[:, :4] = q.T
    return b.tolist()


@pytest.mark.parametrize("frame", ["axis", "rotated"])
def test_c0_estimate_closed_form(frame):
    s = de_scene(c=[0.0] * 8, max_iter=12)
    if frame == "rotated":
        s["slice_basis"] = rotated_basis(7)
    rng = np.random.default_rng(1)
    for _ in range(300):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        r = rng.uniform(1.01, 3.5)
        n, dist, it = oracle.de_distance(s, r * v)
        assert n == c0_count(r, s["escape_radius"], s["max_iter"]) and n > 0
        assert dist == pytest.approx(0.5 * r * math.log(r), rel=1e-12)
        assert it == n
    for _ in range(50):
        v = rng.normal(size=3)
        n, dist, it = oracle.de_distance(s, rng.uniform(0.0, 0.99) * v / np.linalg.norm(v))
        assert n == 0 and dist == 0.0 and it == s["max_iter"]


def sphere_entry(o, d, r):
    b = float(np.dot(o, d))
    disc = b * b - float(np.dot(o, o)) + r * r
    return (-b - math.sqrt(disc)) if disc > 0 else None, disc


def test_c0_sphere_traced_image():
    W = H = 48
    eps = 1e-3
    s = de_scene(c=[0.0] * 8, width=W, height=H, fov_y_deg=60.0, de_epsilon=eps)
    r_eps = 1.0
    for _ in range(60):  # 0.5 r ln r = eps
        r_eps = r_eps - (0.5 * r_eps * math.log(r_eps) - eps) / (0.5 * math.log(r_eps) + 0.5)
    out = oracle.render(s)
    R, mi = s["escape_radius"], s["max_iter"]
    n_hit = n_miss = 0
    for j in range(H):
        for i in range(W):
            o, d = oracle.camera_ray(s, i, j)
            t1, disc1 = sphere_entry(o, d, 1.0)
            te, disce = sphere_entry(o, d, r_eps)
            depth = out["depth"][j, i]
            if disc1 > 0.05:
                assert math.isfinite(depth)
                assert te - 1e-12 <= depth <= t1 + 1e-12
                r = float(np.linalg.norm(o + depth * d))
                assert out["iter"][j, i] == (c0_count(r, R, mi) or mi)
                tr = oracle.trace_pixel(s, i, j)
                assert tr["de_steps"] > 1 and tr["hit"] == 1
                n_hit += 1
            elif disce <= 0:
                assert not math.isfinite(depth) and np.all(out["rgba"][j, i] == 0)
                n_miss += 1
    assert n_hit > 200 and n_miss > 200


def test_bounding_sphere():
    W = H = 32
    s = de_scene(c=[0.0] * 8, width=W, height=H, fov_y_deg=60.0)
    inner = oracle.render(dict(s, de_bound_radius=0.9))
    for j in range(H):
        for i in range(W):
            o, d = oracle.camera_ray(s, i, j)
            t9, disc = sphere_entry(o, d, 0.9)
            if disc > 1e-9:
                # the first sample, at the sphere's entry, is inside the ball of the set
                assert inner["depth"][j, i] == pytest.approx(t9, abs=1e-12)
                assert inner["iter"][j, i] == s["max_iter"]
            elif disc < -1e-9:
                assert not math.isfinite(inner["depth"][j, i]) and inner["iter"][j, i] == 0
    # a bounding sphere that contains the set keeps every clear hit and miss
    free, wide = oracle.render(s), oracle.render(dict(s, de_bound_radius=1.5))
    for j in range(H):
        for i in range(W):
            o, d = oracle.camera_ray(s, i, j)
            _, disc1 = sphere_entry(o, d, 1.0)
            _, disc2 = sphere_entry(o, d, 1.01)
            if disc1 > 0.05 or disc2 < -0.05:
                assert math.isfinite(free["depth"][j, i]) == math.isfinite(wide["depth"][j, i])


def test_de_steps_bounded_and_miss_iter():
    s = de_scene(width=24, height=24, de_max_steps=3)
    for i, j in ((3, 4), (12, 12), (20, 5)):
        tr = oracle.trace_pixel(s, i, j)
        assert tr["de_steps"] <= 3
    out = oracle.render(s)
    full = oracle.render(de_scene(width=24, height=24))
    # with three steps, no ray reaches further than with 512
    assert np.isfinite(out["depth"]).sum() <= np.isfinite(full["depth"]).sum()
