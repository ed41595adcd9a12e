"""Voxel occupancy grid (Fig. voxels) on the GPU against the FP64 oracle: whole
grids at 50^3 and 100^3 (the paper's sizes) and ragged sizes, every precision
mode, axis and random slice frames, and sampled cells of the largest grid.

The contract follows the render's: FP32 + recheck and FP64 match the oracle
cell for cell; plain FP32 may differ only on cells whose escape test was
decided within FP32 rounding of R^2, at most 1e-4 of the grid."""
import numpy as np
import pytest

import oracle
from paper_2303_14827_gb300 import binding, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = binding.dqj_create(0)
    yield c
    binding.dqj_destroy(c)


def gpu_voxels(ctx, s, g):
    import torch
    occ = torch.full((g, g, g), 7, dtype=torch.uint8, device="cuda")
    cnt = torch.full((g, g, g), 7, dtype=torch.int16, device="cuda")
    st = torch.zeros(binding.DQJ_NSTATS, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    binding.dqj_voxelize(ctx, s, g, occ, cnt, st, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return occ.cpu().numpy(), cnt.cpu().numpy().astype(np.int32), binding.stats_dict(st)


def check(ctx, s, g, budget=0.0):
    occ, cnt, st = gpu_voxels(ctx, s, g)
    o = oracle.voxelize(s, g)
    n = g ** 3
    off = (occ != o["occupancy"]) | (cnt != o["count"])
    assert off.sum() <= budget * n, (int(off.sum()), n)
    assert st["samples"] == n
    assert st["hits"] == int(occ.sum())
    if off.sum() == 0:
        assert st["class_iters"] == o["iters"] or s.get("precision") == scenes.PRECISION_FP32_RECHECK
    return occ, cnt, st, o


@pytest.mark.parametrize("g", [50, 100])
@pytest.mark.parametrize("precision", [scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK, scenes.PRECISION_FP64])
def test_paper_grid_sizes(ctx, g, precision):
    s = scenes.default_scene(precision=precision)
    budget = 1e-4 if precision == scenes.PRECISION_FP32 else 0.0
    occ, _, st, _ = check(ctx, s, g, budget)
    assert 0 < occ.sum() < g ** 3
    if precision == scenes.PRECISION_FP32_RECHECK:
        assert st["rechecks"] > 0


@pytest.mark.parametrize("g", [1, 7, 33, 65, 129])
def test_ragged_grids(ctx, g):
    check(ctx, scenes.default_scene(precision=scenes.PRECISION_FP32_RECHECK), g)


def test_random_slice_and_paper_constants(ctx):
    s = scenes.batch_scenes(seed=1, n=3)[2]  # random orthonormal slice frame: the general form
    check(ctx, dict(s, precision=scenes.PRECISION_FP32_RECHECK, max_iter=12), 60)
    for name in ("highres", "test2_f"):
        s = scenes.default_scene(c=list(scenes.PAPER_C_VALUES[name]), max_iter=15,
                                 precision=scenes.PRECISION_FP32_RECHECK)
        check(ctx, s, 64)


def test_modes(ctx):
    for over in (dict(square_mode=scenes.SQUARE_PAPER_COMPONENTWISE), dict(modulus_mode=scenes.MODULUS_DUALNUM)):
        check(ctx, scenes.default_scene(precision=scenes.PRECISION_FP32_RECHECK, **over), 48)


def test_largest_grid_sampled(ctx):
    import torch
    g = binding.DQJ_VOXEL_MAX_GRID
    s = scenes.default_scene(max_iter=16)
    occ = torch.empty(g ** 3, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(g ** 3, dtype=torch.int16, device="cuda")
    st = torch.zeros(binding.DQJ_NSTATS, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    binding.dqj_voxelize(ctx, s, g, occ, cnt, st, torch.cuda.current_stream().cuda_stream)
    cells = scenes.sample_pixels(g * g, g, 20000, seed=5)  # distinct linear cell indices
    idx = torch.from_numpy(cells).cuda()
    go, gc = occ[idx].cpu().numpy(), cnt[idx].cpu().numpy().astype(np.int32)
    inside = int(occ.sum(dtype=torch.int64))
    st = binding.stats_dict(st)
    o = oracle.voxelize(s, g, cells=cells)
    off = (go != o["occupancy"]) | (gc != o["count"])
    assert off.sum() <= 2, int(off.sum())
    assert st["samples"] == g ** 3 and st["hits"] == inside > 0
