"""CPU checks of the C ABI: the library loads, exports every function that
include/dqj.h declares, its defaults match the single-frame scene, and host-side
validation rejects bad parameter blocks with a message (no GPU needed)."""
import re

import numpy as np
import pytest

from paper_2303_14827_gb300 import binding, scenes


@pytest.fixture(scope="module")
def lib():
    return binding.load()


def test_exports_every_declared_symbol(lib):
    names = binding.declared_symbols()
    assert {"dqj_create", "dqj_render", "dqj_submit", "dqj_poll", "dqj_destroy", "dqj_last_error"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_default_params_match_single_frame_scene(lib):
    p = binding.dqj_default_params()
    d = binding.params_to_dict(p)
    want = scenes.default_scene()
    for k, v in want.items():
        assert np.allclose(np.asarray(d[k], dtype=float), np.asarray(v, dtype=float), rtol=0, atol=0), k
    assert binding.dqj_validate_params(p) == binding.DQJ_OK


BAD = [
    ("width", 0), ("width", 16385), ("height", -1), ("max_iter", 0), ("max_iter", 1025),
    ("escape_radius", 0.0), ("escape_radius", float("nan")), ("march_steps", 0), ("march_steps", 65536),
    ("bisect_steps", -1), ("bisect_steps", 31), ("fov_y_deg", 0.0), ("fov_y_deg", 180.0), ("normal_h", 0.0),
    ("precision", 3), ("recheck_margin", -0.1), ("square_mode", 2), ("modulus_mode", -1),
    ("box_min", [2.0, -2.0, -2.0]), ("light_dir", [0.0, 0.0, 0.0]), ("albedo", [1.5, 1.0, 1.0]),
    ("target", [0.0, 0.0, 3.5]), ("up", [0.0, 0.0, 1.0]), ("c", [float("inf")] + [0.0] * 7),
]


@pytest.mark.parametrize("field,value", BAD)
def test_validation_rejects(lib, field, value):
    s = scenes.default_scene(**{field: value})
    assert binding.dqj_validate_params(s) == binding.DQJ_ERR_INVALID
    assert binding.last_error()


def test_validation_rejects_non_orthonormal_basis(lib):
    b = [[1, 0, 0, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0, 0, 0], [0, 1e-6, 1, 0, 0, 0, 0, 0]]
    assert binding.dqj_validate_params(scenes.default_scene(slice_basis=b)) == binding.DQJ_ERR_INVALID
    assert "orthonormal" in binding.last_error()


def test_validation_accepts_config_scenes(lib):
    assert binding.dqj_validate_params(scenes.default_scene()) == binding.DQJ_OK
    assert binding.dqj_validate_params(scenes.full_hd_scene(0)) == binding.DQJ_OK
    for s in scenes.batch_scenes(1, 8):
        assert binding.dqj_validate_params(s) == binding.DQJ_OK


def test_null_arguments_are_errors_not_crashes(lib):
    assert lib.dqj_validate_params(None) == binding.DQJ_ERR_INVALID
    assert lib.dqj_create(None, None) == binding.DQJ_ERR_INVALID
    assert lib.dqj_destroy(None) == binding.DQJ_ERR_INVALID
    assert lib.dqj_render(None, None, None, None) == binding.DQJ_ERR_INVALID
    assert binding.last_error()


def test_serve_stats_layout_matches_header():
    text = open(binding.HEADER).read()
    assert re.search(r"#define DQJ_NSERVE_STATS (\d+)", text).group(1) == str(len(binding.SERVE_STAT_NAMES))


def test_voxelize_validation_on_a_mock_context(monkeypatch):
    ctx = binding.dqj_create(-1)
    try:
        s = scenes.default_scene()
        for g in (0, binding.DQJ_VOXEL_MAX_GRID + 1):
            with pytest.raises(binding.DqjError) as ei:
                binding.dqj_voxelize(ctx, s, g, 4096, 8192)
            assert ei.value.status == binding.DQJ_ERR_INVALID and "grid_n" in binding.last_error()
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_voxelize(ctx, s, 8, None, None)
        assert "both NULL" in binding.last_error()
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_voxelize(ctx, s, 8, 4096, 8193)
        assert "aligned" in binding.last_error()
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_voxelize(ctx, s, 8, 4096, 8192)
        assert "mock" in binding.last_error()
    finally:
        binding.dqj_destroy(ctx)
    text = open(binding.HEADER).read()
    assert re.search(r"#define DQJ_VOXEL_MAX_GRID (\d+)", text).group(1) == str(binding.DQJ_VOXEL_MAX_GRID)


def test_serve_policy_argument_errors():
    ctx = binding.dqj_create(-1)
    try:
        for policy in (binding.DQJ_SERVE_FIFO, binding.DQJ_SERVE_SHORTEST):
            binding.dqj_serve_policy(ctx, policy)
        with pytest.raises(binding.DqjError) as ei:
            binding.dqj_serve_policy(ctx, 2)
        assert ei.value.status == binding.DQJ_ERR_INVALID and "policy" in binding.last_error()
    finally:
        binding.dqj_destroy(ctx)
    text = open(binding.HEADER).read()
    assert re.search(r"#define DQJ_SERVE_FIFO (\d+)", text).group(1) == str(binding.DQJ_SERVE_FIFO)
    assert re.search(r"#define DQJ_SERVE_SHORTEST (\d+)", text).group(1) == str(binding.DQJ_SERVE_SHORTEST)


def test_render_voxels_validation_on_a_mock_context():
    ctx = binding.dqj_create(-1)
    try:
        s = scenes.default_scene(width=64, height=48)
        good = binding.make_outputs(pitch_px=64, depth=4096)
        for g in (0, binding.DQJ_VOXEL_MAX_GRID + 1):
            with pytest.raises(binding.DqjError) as ei:
                binding.dqj_render_voxels(ctx, s, g, 4096, good)
            assert ei.value.status == binding.DQJ_ERR_INVALID and "grid_n" in binding.last_error()
        with pytest.raises(binding.DqjError):
            binding.dqj_render_voxels(ctx, s, 8, None, good)
        assert "occupancy" in binding.last_error()
        with pytest.raises(binding.DqjError):
            binding.dqj_render_voxels(ctx, s, 8, 4096, binding.make_outputs(pitch_px=63, depth=4096))
        assert "pitch" in binding.last_error()
        with pytest.raises(binding.DqjError):
            binding.dqj_render_voxels(ctx, s, 8, 4096, binding.make_outputs(pitch_px=64, depth=4098))
        assert "aligned" in binding.last_error()
        with pytest.raises(binding.DqjError):
            binding.dqj_render_voxels(ctx, dict(s, width=0), 8, 4096, good)
        assert "width" in binding.last_error()
        with pytest.raises(binding.DqjError):
            binding.dqj_render_voxels(ctx, s, 8, 4096, good)
        assert "mock" in binding.last_error()
    finally:
        binding.dqj_destroy(ctx)


@pytest.mark.parametrize("field,value", [("traversal", 2), ("de_max_steps", 0), ("de_epsilon", 0.0),
                                         ("de_step_scale", 1.5), ("de_step_scale", 0.0), ("de_bound_radius", -1.0)])
def test_de_validation_rejects(lib, field, value):
    s = scenes.default_scene(traversal=scenes.TRAVERSAL_DE)
    s[field] = value
    p = binding.make_params(s)
    assert lib.dqj_validate_params(binding.ctypes.byref(p)) == binding.DQJ_ERR_INVALID
    assert field.split("_")[0] in binding.last_error()


def test_de_accepts_every_precision(lib):
    for prec in (scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK, scenes.PRECISION_FP64):
        p = binding.make_params(scenes.default_scene(traversal=scenes.TRAVERSAL_DE, precision=prec))
        assert lib.dqj_validate_params(binding.ctypes.byref(p)) == binding.DQJ_OK


def test_render_host_batch_argument_errors():
    ctx = binding.dqj_create(-1)
    try:
        with pytest.raises(binding.DqjError):
            binding.dqj_render_host_batch(ctx, [scenes.default_scene()], [binding.make_outputs(pitch_px=256)])
        assert "mock" in binding.last_error()
        p = binding.make_params(scenes.default_scene())
        o = binding.make_outputs(pitch_px=256)
        assert binding.load().dqj_render_host_batch(binding.ctypes.c_void_p(ctx), binding.ctypes.byref(p),
                                                    binding.ctypes.byref(o), -1) != binding.DQJ_OK
    finally:
        binding.dqj_destroy(ctx)


def test_render_batch_argument_errors():
    ctx = binding.dqj_create(-1)
    try:
        with pytest.raises(binding.DqjError):
            binding.dqj_render_batch(ctx, [scenes.default_scene()] * 2, [binding.make_outputs(pitch_px=256)] * 2, 0)
        assert "mock" in binding.last_error()
        L = binding.load()
        p = binding.make_params(scenes.default_scene())
        o = binding.make_outputs(pitch_px=256)
        c = binding.ctypes.c_void_p(ctx)
        assert L.dqj_render_batch(c, binding.ctypes.byref(p), binding.ctypes.byref(o), -1, None) != binding.DQJ_OK
        assert L.dqj_render_batch(c, None, None, 2, None) != binding.DQJ_OK
        assert L.dqj_render_batch(None, binding.ctypes.byref(p), binding.ctypes.byref(o), 1, None) != binding.DQJ_OK
        assert L.dqj_render_batch(c, None, None, 0, None) == binding.DQJ_ERR_INVALID  # mock: refused first
    finally:
        binding.dqj_destroy(ctx)


def test_tile_cache_parsing_on_a_mock_context(tmp_path):
    # the cache loader keeps valid entries and ignores malformed or inconsistent
    # ones (a mock context has device name "unknown" and 0 SMs)
    path = tmp_path / "tiles.json"
    path.write_text('{"device": "unknown", "sms": 0, "entries": [[1, 0, 0, 16, 4], [1, 1, 0, 9, 9], '
                    '[1, 9, 0, 8, 8], [0, 2, 1, 32, 1], [1, 3, 3, 64, 1], [x, y], [1, 2, 2, 4'
                    '}')
    ctx = binding.dqj_create(-1, autotune_cache=str(path))
    try:
        def shape(w, h, mi, precision=scenes.PRECISION_FP32):
            return binding.dqj_tile_shape(ctx, scenes.default_scene(width=w, height=h, max_iter=mi,
                                                                    precision=precision))
        assert shape(256, 256, 12) == (1, 16, 4)        # class 0, bucket 0: from the cache
        assert shape(512, 512, 12) == (1, 8, 8)         # 9 x 9 is not a 64-ray tile: default
        assert shape(1024, 1024, 16, scenes.PRECISION_FP64) == (0, 32, 1)
        assert shape(1920, 1080, 32) == (1, 64, 1)
        assert shape(1024, 1024, 24) == (1, 8, 8)       # truncated entry ignored
    finally:
        binding.dqj_destroy(ctx)
    wrong = tmp_path / "other.json"
    wrong.write_text('{"device": "some GPU", "sms": 152, "entries": [[1, 0, 0, 16, 4]]}')
    ctx = binding.dqj_create(-1, autotune_cache=str(wrong))
    try:  # a cache of another device is not used
        assert binding.dqj_tile_shape(ctx, scenes.default_scene(width=256, height=256)) == (1, 8, 8)
    finally:
        binding.dqj_destroy(ctx)


def test_tile_parts_of_pixels_partition_the_frame():
    """The owner map used to put dqj_render_tiles parts together: each pixel's
    part is its tile index (8 x 8 march tiles on a mock context, 8 x 4 for the
    distance-estimate traversal) mod the number of parts, so the parts cover
    the frame once and a tile never straddles two parts."""
    import numpy as np
    ctx = binding.dqj_create(-1)
    try:
        for scene, (tw, th) in ((scenes.default_scene(width=37, height=29), (8, 8)),
                                (scenes.default_scene(width=37, height=29, traversal=scenes.TRAVERSAL_DE), (8, 4))):
            assert (binding.dqj_tile_shape(ctx, scene)[1:] == (8, 8)) or scene["traversal"] == 1
            for parts in (1, 2, 3, 7):
                own = binding.tile_parts_of_pixels(ctx, scene, parts)
                assert own.shape == (29, 37) and own.min() >= 0 and own.max() < parts
                tiles_x = -(-37 // tw)
                for y in range(29):
                    for x in range(37):
                        assert own[y, x] == ((y // th) * tiles_x + x // tw) % parts
                # synthetic parts, each holding its own pixels, put back together
                whole = np.arange(29 * 37).reshape(29, 37)
                planes = [np.where(own == r, whole, -1) for r in range(parts)]
                put = planes[0].copy()
                for r in range(1, parts):
                    put[own == r] = planes[r][own == r]
                assert np.array_equal(put, whole)
    finally:
        binding.dqj_destroy(ctx)
