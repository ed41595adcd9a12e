"""GPU (CUDA path through the C ABI) versus the FP64 oracle on the same seeded
scenes: whole images at sizes the oracle renders in seconds (several tiles and
ragged tails), sampled pixels of the full-size 1920x1080 frames in the launch
configuration the benchmark times, and the edge cases of the method."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import binding, scenes
from parity import assert_parity, compare, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdr():
    import torch
    assert torch.cuda.is_available()
    r = binding.Renderer(0)
    yield r
    r.close()


def gpu_render(rdr, s, **kw):
    out = rdr.render(s, **kw)
    res = to_numpy(out, s["width"], s["height"])
    res["stats"] = binding.stats_dict(out["stats"])
    return res


def run_parity(rdr, s, what, flip_frac=1e-3):
    g = gpu_render(rdr, s)
    o = oracle.render(s)
    rep = compare(g, o, flip_frac)
    assert_parity(rep, flip_frac, what)
    return g, o, rep


@pytest.mark.parametrize("precision", [scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK,
                                       scenes.PRECISION_FP64])
def test_single_frame_scene(rdr, precision):
    s = scenes.default_scene(precision=precision)
    g, o, rep = run_parity(rdr, s, f"256x256 precision {precision}")
    st = g["stats"]
    assert st["hits"] == rep["hits_gpu"]
    # the kernels count the same DQ iterations as the oracle, up to the samples
    # whose decisions differ (none expected here)
    assert abs(st["class_iters"] - o["class_iters"]) <= 1e-4 * o["class_iters"], (st, o["class_iters"])
    assert abs(st["normal_iters"] - o["normal_iters"]) <= 1e-3 * o["normal_iters"] + 100
    if precision == scenes.PRECISION_FP32_RECHECK:
        assert 0 < st["rechecks"] < 0.01 * st["samples"]
        assert st["overflow"] == 0


def test_c0_ball_on_gpu(rdr):
    # c = 0: filled set is the ball |p| <= R^(2^-max_iter); hits at the analytic
    # ray-sphere depth within the bisection bracket, iter = max_iter.
    s = scenes.default_scene(c=[0.0] * 8, width=96, height=80, fov_y_deg=60.0)
    g = gpu_render(rdr, s)
    rs = s["escape_radius"] ** (2.0 ** -s["max_iter"])
    n_hit = 0
    for j in range(s["height"]):
        for i in range(s["width"]):
            o, d = oracle.camera_ray(s, i, j)
            ok, t_in, t_out = oracle.box_clip(s, o, d)
            delta = (t_out - t_in) / s["march_steps"]
            b = float(np.dot(o, d))
            disc = b * b - float(np.dot(o, o)) + rs * rs
            if disc > 0 and 2 * math.sqrt(disc) > 2.5 * delta:
                t_hit = -b - math.sqrt(disc)
                assert abs(g["depth"][j, i] - t_hit) <= delta / 2 ** (s["bisect_steps"] + 1) + 2e-6
                assert g["iter"][j, i] == s["max_iter"]
                n_hit += 1
            elif disc < 0:
                assert not np.isfinite(g["depth"][j, i])
    assert n_hit > 100
    run_parity(rdr, s, "c=0 ball")


@pytest.mark.parametrize("name", sorted(scenes.PAPER_C_VALUES))
def test_paper_constants(rdr, name):
    s = scenes.default_scene(c=list(scenes.PAPER_C_VALUES[name]), width=128, height=96, max_iter=15)
    run_parity(rdr, s, name)


@pytest.mark.parametrize("w,h", [(1, 1), (3, 5), (7, 1), (1, 9), (37, 19), (33, 4), (8, 4)])
def test_ragged_and_tiny_images(rdr, w, h):
    run_parity(rdr, scenes.default_scene(width=w, height=h), f"{w}x{h}", flip_frac=0.0)


def test_pitch_and_partial_planes(rdr):
    import torch
    s = scenes.default_scene(width=45, height=30)
    out = binding.alloc_outputs(45, 30, pitch_px=64)
    for k in ("iter", "depth", "normal", "rgba"):
        out[k].fill_(7 if k != "depth" else 7.0)
    rdr.render(s, out)
    for k in ("iter", "depth", "normal", "rgba"):
        pad = out[k][:, 45:]
        assert torch.all(pad == 7), k
    o = oracle.render(s)
    assert_parity(compare(to_numpy(out, 45, 30), o), what="pitch 64")
    # only the depth plane
    only = {"depth": torch.empty((30, 45), device="cuda"), "pitch_px": 45}
    rdr.render(s, only)
    assert np.array_equal(only["depth"].cpu().numpy(), out["depth"][:, :45].cpu().numpy())


@pytest.mark.parametrize("over", [
    dict(bisect_steps=0), dict(march_steps=1), dict(max_iter=1), dict(max_iter=40),
    dict(eye=[0.3, -0.2, 0.1], target=[1.0, 1.0, 1.0]),  # eye inside the box
    dict(eye=[0.0, 0.0, 3.5], target=[0.0, 0.0, 9.0]),   # looking away: every ray misses
    dict(fov_y_deg=120.0),                               # many rays miss the box
    dict(escape_radius=2.0), dict(normal_h=1e-2),
    dict(square_mode=scenes.SQUARE_PAPER_COMPONENTWISE),
    dict(modulus_mode=scenes.MODULUS_DUALNUM),
    dict(square_mode=1, modulus_mode=1),
    dict(k_specular=0.5, shininess=16.0, light_dir=[0.3, 0.4, 1.0]),  # Eq. phong specular term
])
@pytest.mark.parametrize("precision", [scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK])
def test_edge_cases(rdr, over, precision):
    s = scenes.default_scene(width=64, height=48, precision=precision, **over)
    run_parity(rdr, s, f"{over} precision {precision}")


def test_random_slice_frames(rdr):
    for k, s in enumerate(scenes.batch_scenes(seed=1, n=6)):
        s.update(width=120, height=90)
        run_parity(rdr, s, f"batch scene {k}")


def test_deterministic(rdr):
    s = scenes.default_scene(width=200, height=120)
    a = gpu_render(rdr, s)
    b = gpu_render(rdr, s)
    for k in ("iter", "depth", "normal", "rgba"):
        assert np.array_equal(a[k], b[k]), k
    assert a["stats"] == b["stats"]


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_full_hd_sampled(rdr, seed):
    # The 1920x1080 frame in the configuration the benchmark times, compared on
    # sampled pixels (all GPU hit pixels up to 2000, plus 3000 random ones).
    s = scenes.full_hd_scene(seed)
    g = gpu_render(rdr, s)
    W = s["width"]
    hit_pix = np.flatnonzero(np.isfinite(g["depth"].reshape(-1)))[:2000]
    pix = np.union1d(scenes.sample_pixels(W, s["height"], 3000, seed=seed), hit_pix)
    o = oracle.render(s, pixels=pix)
    sub = {k: g[k].reshape((-1,) + g[k].shape[2:])[pix] for k in ("iter", "depth", "normal", "rgba")}
    rep = compare(sub, o)
    assert_parity(rep, what=f"1080p seed {seed}")
    assert g["stats"]["hits"] == int(np.isfinite(g["depth"]).sum())


@pytest.mark.parametrize("precision", [scenes.PRECISION_FP32_RECHECK, scenes.PRECISION_FP64])
def test_full_hd_precision_modes_sampled(rdr, precision):
    s = scenes.full_hd_scene(3, precision=precision)
    g = gpu_render(rdr, s)
    hit_pix = np.flatnonzero(np.isfinite(g["depth"].reshape(-1)))[:1000]
    pix = np.union1d(scenes.sample_pixels(s["width"], s["height"], 1500, seed=9), hit_pix)
    o = oracle.render(s, pixels=pix)
    sub = {k: g[k].reshape((-1,) + g[k].shape[2:])[pix] for k in ("iter", "depth", "normal", "rgba")}
    assert_parity(compare(sub, o), what=f"1080p precision {precision}")


@pytest.mark.parametrize("scene", ["single", "hd3", "batch2", "paper"])
def test_march_variants_bitwise_equal(rdr, scene, monkeypatch):
    # The two FP32 march kernels (one ray per lane; two rays per lane in float2
    # halves) run the same per-sample arithmetic in the same order, so their
    # images must be identical.
    if scene == "single":
        s = scenes.default_scene(width=200, height=150)
    elif scene == "hd3":
        s = scenes.full_hd_scene(3)
    elif scene == "batch2":
        s = scenes.batch_scenes(seed=1, n=3)[2]
    else:
        s = scenes.default_scene(c=list(scenes.PAPER_C_VALUES["highres"]), width=161, height=97, max_iter=15)
    outs = []
    for v in ("0", "1"):
        monkeypatch.setenv("DQJ_MARCH_VARIANT", v)
        outs.append(gpu_render(rdr, s))
    for o in outs[1:]:
        for k in ("iter", "depth", "normal", "rgba"):
            assert np.array_equal(o[k], outs[0][k]), k
        assert o["stats"] == outs[0]["stats"]


@pytest.mark.parametrize("scene", ["single", "ragged", "random_slice", "max_iter40"])
def test_split_march_equals_unsplit(rdr, scene, monkeypatch):
    # Frames with fewer tiles than the GPU has resident warps split each ray's
    # samples into ranges marched by different warps; the merge keeps the
    # ranges up to the first inside sample, so images and iteration counts
    # equal the unsplit march exactly.
    if scene == "single":
        s = scenes.default_scene()
    elif scene == "ragged":
        s = scenes.default_scene(width=131, height=77, march_steps=255)
    elif scene == "random_slice":
        s = dict(scenes.batch_scenes(seed=1, n=3)[2], width=200, height=150)
    else:
        s = scenes.default_scene(width=160, height=120, max_iter=40, march_steps=97)
    monkeypatch.setenv("DQJ_MARCH_SPLIT", "0")
    whole = gpu_render(rdr, s)
    monkeypatch.delenv("DQJ_MARCH_SPLIT")
    split = gpu_render(rdr, s)
    for k in ("iter", "depth", "normal", "rgba"):
        assert np.array_equal(split[k], whole[k]), k
    assert split["stats"] == whole["stats"]
    if scene in ("single", "ragged"):
        run_parity(rdr, s, f"split march {scene}")


def test_render_host_batch_equals_device_render(rdr):
    # host outputs through the double-buffered batch: every frame equals the
    # device render of the same scene, with ragged sizes and a host pitch
    import torch
    frames = [scenes.default_scene(width=w, height=h, max_iter=mi)
              for w, h, mi in ((96, 64, 12), (37, 19, 9), (128, 128, 16), (64, 48, 12), (1, 1, 5))]
    host = []
    for s in frames:
        w, h = s["width"], s["height"]
        pitch = w + 3
        host.append({"iter": torch.full((h, pitch), -7, dtype=torch.int32).pin_memory(),
                     "depth": torch.zeros((h, pitch), dtype=torch.float32).pin_memory(),
                     "normal": torch.zeros((h, pitch, 3), dtype=torch.float32).pin_memory(),
                     "rgba": torch.zeros((h, pitch, 4), dtype=torch.uint8).pin_memory(),
                     "stats": torch.zeros(binding.DQJ_NSTATS, dtype=torch.int64).pin_memory(), "pitch_px": pitch})
    binding.dqj_render_host_batch(rdr.ctx, frames, [binding.outputs_of(o) for o in host])
    binding.dqj_render_host_batch(rdr.ctx, [], [])
    for s, o in zip(frames, host):
        ref = rdr.render(s)
        w, h = s["width"], s["height"]
        for k in ("iter", "depth", "normal", "rgba"):
            assert np.array_equal(o[k][:, :w].numpy(), ref[k][:, :w].cpu().numpy()), k
        assert np.all(o["iter"][:, w:].numpy() == -7)
        assert binding.stats_dict(o["stats"]) == binding.stats_dict(ref["stats"])
    bad = [frames[0], dict(frames[1], max_iter=0)]
    with pytest.raises(binding.DqjError):
        binding.dqj_render_host_batch(rdr.ctx, bad, [binding.outputs_of(o) for o in host[:2]])


def test_render_host_single_frame_pageable_and_partial_planes(rdr):
    # dqj_render_host into ordinary (pageable) host memory, only two planes
    # requested: they equal the device render; the others are not touched
    import torch
    s = scenes.default_scene(width=80, height=60, max_iter=14)
    w, h = s["width"], s["height"]
    o = {"iter": None, "normal": None,
         "depth": torch.zeros((h, w), dtype=torch.float32),
         "rgba": torch.zeros((h, w, 4), dtype=torch.uint8), "stats": None, "pitch_px": w}
    binding.dqj_render_host(rdr.ctx, s, binding.outputs_of(o))
    ref = rdr.render(s)
    assert np.array_equal(o["depth"].numpy(), ref["depth"][:, :w].cpu().numpy())
    assert np.array_equal(o["rgba"].numpy(), ref["rgba"][:, :w].cpu().numpy())
    with pytest.raises(binding.DqjError):
        binding.dqj_render_host(rdr.ctx, dict(s, width=0), binding.outputs_of(o))
