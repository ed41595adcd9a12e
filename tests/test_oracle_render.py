"""Pins of the FP64 oracle's renderer: camera orientation, the box clip, the
c = 0 case whose filled set is the closed-form ball |p| <= R^(2^-max_iter)
(hit mask, analytic ray-sphere depth, radial normal, per-sample escape counts),
mirror symmetry, brute-force march/bisection brackets on tiny images, and the
invariants of the two modulus readings."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import scenes


def cam_basis(s):
    f = np.subtract(s["target"], s["eye"]).astype(float)
    f /= np.linalg.norm(f)
    r = np.cross(f, s["up"])
    r /= np.linalg.norm(r)
    return f, r, np.cross(r, f)


def test_camera_orientation_and_fov():
    s = scenes.default_scene(width=64, height=48)
    f, r, u = cam_basis(s)
    o, d = oracle.camera_ray(s, 0, 0)  # top-left pixel
    assert np.allclose(o, s["eye"])
    assert abs(np.linalg.norm(d) - 1.0) < 1e-15
    assert d[0] < 0 and d[1] > 0 and d[2] < 0  # looking down -z from +z: left is -x, top is +y
    o, d = oracle.camera_ray(s, 63, 47)  # bottom-right
    assert d[0] > 0 and d[1] < 0
    # the vertical angle of the centre-column ray through row j is atan((1 - (2j+1)/H) tan(fov/2))
    s = scenes.default_scene(width=33, height=21)
    th = math.tan(math.radians(22.5))
    for j in (0, 5, 10, 20):
        _, d = oracle.camera_ray(s, 16, j)
        want = math.atan((1.0 - (2 * j + 1) / 21.0) * th)
        assert abs(math.atan2(d[1], -d[2]) - want) < 1e-14
    # horizontal extent follows the aspect ratio
    _, d = oracle.camera_ray(s, 0, 10)
    want = math.atan((-1.0 + 1.0 / 33.0) * th * 33.0 / 21.0)
    assert abs(math.atan2(d[0], -d[2]) - want) < 1e-14


def brute_box(o, d, lo, hi, n=200001, tmax=20.0):
    t = np.linspace(0.0, tmax, n)
    p = o[None, :] + t[:, None] * d[None, :]
    inside = np.all((p >= lo) & (p <= hi), axis=1)
    if not inside.any():
        return None
    idx = np.nonzero(inside)[0]
    return t[idx[0]], t[idx[-1]], t[1] - t[0]


def test_box_clip_against_brute_force():
    rng = np.random.default_rng(5)
    s = scenes.default_scene()
    lo, hi = np.array(s["box_min"]), np.array(s["box_max"])
    n_hit = 0
    for _ in range(300):
        o = rng.uniform(-5, 5, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        hit, t0, t1 = oracle.box_clip(s, o, d)
        bf = brute_box(o, d, lo, hi)
        if bf is None:
            assert not hit or (t1 - t0) < 1e-3
            continue
        if bf[1] - bf[0] < 3 * bf[2]:
            continue  # grazing within the brute-force resolution
        assert hit
        n_hit += 1
        assert abs(t0 - bf[0]) <= bf[2] and abs(t1 - bf[1]) <= bf[2]
    assert n_hit > 30
    # axis-parallel rays: d has zero components
    hit, t0, t1 = oracle.box_clip(s, [0.5, 0.5, 3.5], [0.0, 0.0, -1.0])
    assert hit and t0 == 1.5 and t1 == 5.5
    hit, _, _ = oracle.box_clip(s, [2.5, 0.0, 3.5], [0.0, 0.0, -1.0])
    assert not hit
    # origin inside the box: t_in clamps to 0
    hit, t0, t1 = oracle.box_clip(s, [0.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    assert hit and t0 == 0.0 and t1 == 2.0


def ball_radius(R, max_iter):
    return R ** (2.0 ** (-max_iter))


def c0_count(r, R, max_iter):
    if r <= 1.0:
        return 0
    n = max(1, int(math.floor(math.log2(math.log(R) / math.log(r)))) + 1)
    return n if n <= max_iter else 0


def slab(o, d, lo, hi):
    t0, t1 = -math.inf, math.inf
    for a in range(3):
        if d[a] == 0.0:
            if o[a] < lo[a] or o[a] > hi[a]:
                return None
            continue
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    t0 = max(t0, 0.0)
    return (t0, t1) if t0 < t1 else None


@pytest.mark.parametrize("frame", ["axis", "rotated"])
def test_c0_ball_closed_form(frame):
    W = H = 48
    s = scenes.default_scene(c=[0.0] * 8, width=W, height=H, fov_y_deg=60.0)
    if frame == "rotated":
        # any orthonormal frame inside the real-quaternion subspace sees the same ball
        rng = np.random.default_rng(3)
        q, _ = np.linalg.qr(rng.normal(size=(4, 3)))
        b = np.zeros((3, 8))
        b[:, :4] = q.T
        s["slice_basis"] = b.tolist()
    R, N, B, mi = s["escape_radius"], s["march_steps"], s["bisect_steps"], s["max_iter"]
    rs = ball_radius(R, mi)
    out = oracle.render(s)
    lo, hi = np.array(s["box_min"]), np.array(s["box_max"])
    l = np.array(s["light_dir"]) / np.linalg.norm(s["light_dir"])
    n_hit = n_checked_miss = 0
    for j in range(H):
        for i in range(W):
            o, d = oracle.camera_ray(s, i, j)
            clip = slab(o, d, lo, hi)
            assert clip is not None
            t_in, t_out = clip
            delta = (t_out - t_in) / N
            b = float(np.dot(o, d))
            disc = b * b - float(np.dot(o, o)) + rs * rs
            depth = out["depth"][j, i]
            if disc > 0 and 2 * math.sqrt(disc) > 2.5 * delta:
                # chord longer than two sample spacings: a hit at the analytic depth
                t_hit = -b - math.sqrt(disc)
                assert math.isfinite(depth)
                assert abs(depth - t_hit) <= delta / 2 ** (B + 1) + 1e-12
                assert out["iter"][j, i] == mi
                p = o + depth * d
                nrm = out["normal"][j, i]
                # F = |p|^(2^(n*+1)) at c = 0: its central differences in closed form
                h, e = s["normal_h"], 2.0 ** (mi + 1)
                g = np.array([np.linalg.norm(p + h * ax) ** e - np.linalg.norm(p - h * ax) ** e
                              for ax in np.eye(3)])
                assert float(np.dot(nrm, g / np.linalg.norm(g))) > 1.0 - 1e-9
                # and the field is radial up to the finite-difference bias
                assert float(np.dot(nrm, p / np.linalg.norm(p))) > math.cos(math.radians(3.0))
                gn = g / np.linalg.norm(g)
                v = min(1.0, 0.15 + 0.85 * max(0.0, float(np.dot(gn, l))))
                assert abs(int(out["rgba"][j, i, 0]) - math.floor(255 * v + 0.5)) <= 1
                assert out["rgba"][j, i, 3] == 255
                n_hit += 1
            elif disc < 0:
                assert not math.isfinite(depth)
                assert np.all(out["normal"][j, i] == 0) and np.all(out["rgba"][j, i] == 0)
                # a miss reports the largest closed-form escape count over its samples
                want = max(c0_count(float(np.linalg.norm(o + (t_in + k * delta) * d)), R, mi)
                           for k in range(N + 1))
                assert out["iter"][j, i] == want
                n_checked_miss += 1
    assert n_hit > 50 and n_checked_miss > 500


def test_mirror_symmetry_complex_c():
    # With c in the complex subalgebra the set is symmetric under the third real
    # coordinate's sign flip, so the views from (0,0,+3.5) and (0,0,-3.5) are
    # left-right mirror images.
    c = [-0.5, 0.55, 0, 0, 0, 0, 0, 0]
    W, H = 40, 30
    front = oracle.render(scenes.default_scene(c=c, width=W, height=H))
    back = oracle.render(scenes.default_scene(c=c, width=W, height=H, eye=[0.0, 0.0, -3.5]))
    hf = np.isfinite(front["depth"])
    hb = np.isfinite(back["depth"])[:, ::-1]
    assert hf.sum() > 50
    assert np.array_equal(hf, hb)
    assert np.array_equal(front["iter"], back["iter"][:, ::-1])
    assert np.allclose(front["depth"][hf], back["depth"][:, ::-1][hf], atol=1e-9)


def test_march_and_bisection_brackets_brute_force():
    s = scenes.default_scene(width=8, height=8, fov_y_deg=30.0)
    N, B = s["march_steps"], s["bisect_steps"]
    args = (s["c"], s["max_iter"], s["escape_radius"])
    hits = 0
    for j in range(8):
        for i in range(8):
            tr = oracle.trace_pixel(s, i, j)
            o, d = tr["o"], tr["d"]

            def cls(t):
                return oracle.classify(oracle.slice_point(s, o + t * d), *args)[0]

            if not tr["box_hit"]:
                continue
            kf = tr["k_first"]
            counts = []
            last = N if kf < 0 else kf - 1
            for k in range(last + 1):
                n = cls(tr["t_in"] + k * tr["delta"])
                assert n != 0
                counts.append(n)
            if kf < 0:
                assert tr["esc_max"] == max(counts)
                continue
            hits += 1
            assert cls(tr["t_in"] + kf * tr["delta"]) == 0
            if kf == 0:
                continue
            # final bracket: lo outside, hi inside, width delta / 2^B
            assert cls(tr["lo"]) == tr["n_star"] and tr["n_star"] > 0
            assert cls(tr["hi"]) == 0
            assert abs((tr["hi"] - tr["lo"]) - tr["delta"] / 2 ** B) <= 1e-12
            assert tr["t_in"] + (kf - 1) * tr["delta"] - 1e-12 <= tr["lo"] < tr["hi"] <= tr["t_in"] + kf * tr["delta"] + 1e-12
            # a fine brute-force scan of the bracket finds an outside->inside transition in it
            ts = np.linspace(tr["lo"], tr["hi"], 65)
            inside = [cls(t) == 0 for t in ts]
            assert not inside[0] and inside[-1]
            assert abs(tr["depth"] - 0.5 * (tr["lo"] + tr["hi"])) < 1e-12
    assert hits >= 8


def test_dualnum_ignores_the_dual_half():
    # Under the dual-number modulus |q_r|^2 the real half evolves alone, so the
    # image does not depend on the dual half of c; with c_d = 0 on the default
    # slice the dual half stays zero and both moduli agree.
    base = dict(width=24, height=24, modulus_mode=scenes.MODULUS_DUALNUM)
    a = oracle.render(scenes.default_scene(**base))
    c = list(scenes.C_DEFAULT[:4]) + [0.7, -0.3, 0.2, 0.9]
    b = oracle.render(scenes.default_scene(c=c, **base))
    assert np.array_equal(a["iter"], b["iter"]) and np.array_equal(a["depth"], b["depth"])
    c0 = list(scenes.C_DEFAULT[:4]) + [0.0] * 4
    e8 = oracle.render(scenes.default_scene(c=c0, width=24, height=24))
    dn = oracle.render(scenes.default_scene(c=c0, **base))
    assert np.array_equal(e8["iter"], dn["iter"]) and np.array_equal(e8["depth"], dn["depth"])


def test_pixel_list_equals_full_image():
    s = scenes.default_scene(width=20, height=12)
    full = oracle.render(s)
    pix = scenes.sample_pixels(20, 12, 50, seed=3)
    part = oracle.render(s, pixels=pix)
    assert np.array_equal(part["iter"], full["iter"].reshape(-1)[pix])
    assert np.array_equal(part["depth"], full["depth"].reshape(-1)[pix])
    assert np.array_equal(part["rgba"], full["rgba"].reshape(-1, 4)[pix])


def test_normal_overflow_guard_c0():
    # At c = 0 the field is F(q) = |q|^(2^(n*+1)) in closed form.  Where any of the
    # six neighbours has F > 2^100 the normal is -d; elsewhere it is the
    # normalised central difference.  h = 0.01 gives both cases in one image.
    W = H = 40
    s = scenes.default_scene(c=[0.0] * 8, width=W, height=H, fov_y_deg=60.0, normal_h=0.01)
    out = oracle.render(s)
    e = 2.0 ** (s["max_iter"] + 1)
    n_guard = n_grad = 0
    for j in range(H):
        for i in range(W):
            depth = out["depth"][j, i]
            if not np.isfinite(depth):
                continue
            o, d = oracle.camera_ray(s, i, j)
            p = o + depth * d
            logs = [e * math.log(np.linalg.norm(p + sg * s["normal_h"] * ax)) for ax in np.eye(3) for sg in (1, -1)]
            nrm = out["normal"][j, i]
            if max(logs) > 100 * math.log(2.0):
                assert np.allclose(nrm, -d, atol=0), (i, j)
                n_guard += 1
            else:
                F = np.exp(logs)
                g = np.array([F[0] - F[1], F[2] - F[3], F[4] - F[5]])
                assert float(np.dot(nrm, g / np.linalg.norm(g))) > 1.0 - 1e-9
                n_grad += 1
    assert n_guard > 10 and n_grad > 10, (n_guard, n_grad)


def test_c0_ball_specular_closed_form():
    # Eq. phong with the specular term on the c = 0 ball: the expected shade from
    # the closed-form central-difference normal, the reflected light
    # r = 2n(n.l) - l and the unit vector to the eye v = -d.
    W = H = 40
    ks, sh = 0.6, 20.0
    s = scenes.default_scene(c=[0.0] * 8, width=W, height=H, fov_y_deg=60.0, k_specular=ks, shininess=sh,
                             light_dir=[0.3, 0.4, 1.0])
    mi = s["max_iter"]
    out = oracle.render(s)
    l = np.array(s["light_dir"]) / np.linalg.norm(s["light_dir"])
    n_hit = n_lit = 0
    for j in range(H):
        for i in range(W):
            depth = out["depth"][j, i]
            if not math.isfinite(depth):
                continue
            o, d = oracle.camera_ray(s, i, j)
            p = o + depth * d
            h, e = s["normal_h"], 2.0 ** (mi + 1)
            g = np.array([np.linalg.norm(p + h * ax) ** e - np.linalg.norm(p - h * ax) ** e for ax in np.eye(3)])
            n = g / np.linalg.norm(g)
            ndl = float(np.dot(n, l))
            spec = 0.0
            if ndl > 0:
                r = 2.0 * ndl * n - l
                rv = -float(np.dot(r, d))
                if rv > 0:
                    spec = ks * rv ** sh
            v = min(1.0, 0.15 + 0.85 * max(0.0, ndl) + spec)
            assert abs(int(out["rgba"][j, i, 0]) - math.floor(255 * v + 0.5)) <= 1
            n_hit += 1
            n_lit += spec * 255 > 10
    assert n_hit > 50 and n_lit > 5  # the highlight is on the visible cap
