"""Distance-estimate sphere tracing (the paper's own traversal, Eq. distfract2)
on the GPU against the FP64 oracle.

FP64 and FP32 with the FP64 recheck are held to the render's full parity
contract.  Plain FP32 is outside it: it accumulates the ray parameter in
single precision, so a sample whose estimate lies within rounding of epsilon
can stop one step earlier or later; its hit/miss class and the contract hold
on all but a few pixels, and the depth on >= 99 % of common hits (the step
moves it by up to one estimate, below epsilon).  The recheck mode re-evaluates
such samples (and those whose escape test came within the margin of R^2) in
FP64 and re-traces in FP64 the pixels whose decisions could differ."""
import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import binding, scenes
from parity import DEPTH_TOL, assert_parity, compare, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdr():
    r = binding.Renderer(0)
    yield r
    r.close()


def de(**over):
    base = dict(traversal=scenes.TRAVERSAL_DE)
    base.update(over)
    return scenes.default_scene(**base)


CASES = {
    "c0": de(c=[0.0] * 8, width=96, height=96, fov_y_deg=60.0),
    "default": de(width=160, height=120),
    "bound_sphere": de(width=160, height=120, de_bound_radius=1.8),
    "highres": de(c=list(scenes.PAPER_C_VALUES["highres"]), width=160, height=120, max_iter=15),
    "test2_f": de(c=list(scenes.PAPER_C_VALUES["test2_f"]), width=160, height=120, max_iter=15),
    "eps_1e-4": de(width=160, height=120, de_epsilon=1e-4),
    "half_steps": de(width=128, height=96, de_step_scale=0.5),
    "dualnum": de(width=128, height=96, modulus_mode=scenes.MODULUS_DUALNUM),
    "componentwise": de(width=128, height=96, square_mode=scenes.SQUARE_PAPER_COMPONENTWISE),
    "few_steps": de(width=96, height=64, de_max_steps=4),
    "random_slice": dict(scenes.batch_scenes(seed=1, n=3)[2], traversal=scenes.TRAVERSAL_DE, width=128, height=96,
                         max_iter=12),
    "tiny": de(width=1, height=1),
    "ragged": de(width=37, height=19),
}


def de_fp32_contract(rep, g, o, what):
    n = rep["pixels"]
    assert rep["flips"] <= 1e-3 * n, (what, rep)
    assert rep["iter_mismatch"] <= max(2, 2e-4 * n), (what, rep)
    gd, od = g["depth"].reshape(-1).astype(np.float64), o["depth"].reshape(-1)
    both = np.isfinite(gd) & np.isfinite(od)
    if both.any():
        assert np.mean(np.abs(gd[both] - od[both]) <= DEPTH_TOL) >= 0.99, (what, rep)
    assert rep["normal_ok_frac"] >= 0.99 and rep["rgba_ok_frac"] >= 0.99, (what, rep)
    assert rep["miss_planes_ok"], (what, rep)


@pytest.mark.parametrize("name", sorted(CASES))
def test_de_against_oracle(rdr, name):
    s = CASES[name]
    o = oracle.render(s)
    g64 = to_numpy(rdr.render(dict(s, precision=scenes.PRECISION_FP64)), s["width"], s["height"])
    assert_parity(compare(g64, o), what=f"DE FP64 {name}")
    out = rdr.render(dict(s, precision=scenes.PRECISION_FP32))
    g32 = to_numpy(out, s["width"], s["height"])
    de_fp32_contract(compare(g32, o), g32, o, f"DE FP32 {name}")
    st = binding.stats_dict(out["stats"])
    assert st["hits"] == int(np.isfinite(g32["depth"]).sum())
    assert st["samples"] >= st["hits"]
    out_rc = rdr.render(dict(s, precision=scenes.PRECISION_FP32_RECHECK))
    g_rc = to_numpy(out_rc, s["width"], s["height"])
    assert_parity(compare(g_rc, o), what=f"DE FP32+recheck {name}")


def test_de_full_hd_sampled(rdr):
    s = de(width=1920, height=1080, max_iter=16)
    out = rdr.render(s)
    g = to_numpy(out, 1920, 1080)
    hit_pix = np.flatnonzero(np.isfinite(g["depth"].reshape(-1)))[:2000]
    pix = np.union1d(scenes.sample_pixels(1920, 1080, 3000, seed=4), hit_pix)
    o = oracle.render(s, pixels=pix)
    sub = {k: g[k].reshape((-1,) + g[k].shape[2:])[pix] for k in ("iter", "depth", "normal", "rgba")}
    de_fp32_contract(compare(sub, o), sub, o, "DE 1080p sampled")
    st = binding.stats_dict(out["stats"])
    # sphere tracing takes far fewer samples than the 513-sample march
    assert st["samples"] < 40 * 1920 * 1080


def test_de_full_hd_recheck_meets_contract(rdr):
    # the default c at 1080p (many hits), every pixel, FP32 + FP64 recheck
    s = de(width=1920, height=1080, max_iter=16, precision=scenes.PRECISION_FP32_RECHECK)
    out = rdr.render(s)
    g = to_numpy(out, 1920, 1080)
    rep = compare(g, oracle.render(s))
    assert_parity(rep, what="DE 1080p FP32+recheck, whole frame")
    st = binding.stats_dict(out["stats"])
    # every hit is re-traced in FP64, and the misses with a decision close to
    # a threshold: a small fraction of the frame
    hits = int(np.isfinite(g["depth"]).sum())
    assert st["rechecks"] > 0 and hits <= st["fixups"] < hits + 0.01 * 1920 * 1080, st


def test_de_noalloc_equals_render(rdr):
    import torch
    s = de(width=200, height=150)
    ref = to_numpy(rdr.render(s), 200, 150)
    out = binding.alloc_outputs(200, 150)
    torch.cuda.synchronize()
    binding.dqj_render_noalloc(s, binding.outputs_of(out), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    g = to_numpy(out, 200, 150)
    for k in ("iter", "depth", "normal", "rgba"):
        assert np.array_equal(g[k], ref[k]), k


def test_de_served_equals_alone(rdr):
    import time

    import torch
    reqs = [CASES["default"], CASES["highres"], dict(CASES["default"], precision=scenes.PRECISION_FP64),
            scenes.default_scene(width=96, height=64)]
    outs = [binding.alloc_outputs(s["width"], s["height"]) for s in reqs]
    torch.cuda.synchronize()
    ctx = binding.dqj_create(0)
    try:
        tickets = [binding.dqj_submit(ctx, s, binding.outputs_of(o)) for s, o in zip(reqs, outs)]
        t0 = time.time()
        for t in tickets:
            while True:
                done, st = binding.dqj_poll(ctx, t)
                if done:
                    assert st == binding.DQJ_OK
                    break
                assert time.time() - t0 < 60
                time.sleep(0.001)
    finally:
        binding.dqj_destroy(ctx)
    for s, o in zip(reqs, outs):
        a, b = to_numpy(o, s["width"], s["height"]), to_numpy(rdr.render(s), s["width"], s["height"])
        for k in ("iter", "depth", "normal", "rgba"):
            assert np.array_equal(a[k], b[k]), k
