"""Element-by-element comparison of a GPU render with the FP64 oracle.

Tolerances (the renderer's accuracy contract):
  * hit/miss may differ on at most 0.1% of the compared pixels (a sample whose
    exact FP64 decision lies within rounding of R^2 has two correct answers);
  * on every pixel whose hit/miss agrees, ``iter`` is identical;
  * on pixels that are hits in both, |depth error| <= 1e-4 scene units;
  * normals within 1 degree and RGBA within 1 LSB on >= 99% of common hits;
  * misses carry depth +inf, normal (0,0,0) and RGBA (0,0,0,0) exactly.
"""
from __future__ import annotations

import numpy as np

FLIP_FRAC = 1e-3
DEPTH_TOL = 1e-4
NORMAL_DEG = 1.0
GOOD_FRAC = 0.99


def to_numpy(out: dict, width: int, height: int) -> dict:
    """Crop torch output planes (pitch >= width) to numpy arrays."""
    r = {}
    for k in ("iter", "depth", "normal", "rgba"):
        if out.get(k) is not None:
            r[k] = out[k][:, :width].cpu().numpy()
    return r


def compare(gpu: dict, ref: dict, flip_frac: float = FLIP_FRAC) -> dict:
    gd = np.asarray(gpu["depth"], dtype=np.float64).reshape(-1)
    od = np.asarray(ref["depth"], dtype=np.float64).reshape(-1)
    n = gd.size
    hg, ho = np.isfinite(gd), np.isfinite(od)
    agree = hg == ho
    both = hg & ho
    gi = np.asarray(gpu["iter"]).reshape(-1)
    oi = np.asarray(ref["iter"]).reshape(-1)
    rep = {
        "pixels": n,
        "hits_gpu": int(hg.sum()),
        "hits_ref": int(ho.sum()),
        "flips": int((~agree).sum()),
        "iter_mismatch": int(((gi != oi) & agree).sum()),
        "max_depth_err": float(np.max(np.abs(gd[both] - od[both]))) if both.any() else 0.0,
    }
    gn = np.asarray(gpu["normal"], dtype=np.float64).reshape(-1, 3)
    on = np.asarray(ref["normal"], dtype=np.float64).reshape(-1, 3)
    if both.any():
        cos = np.clip(np.sum(gn[both] * on[both], axis=1), -1.0, 1.0)
        ang = np.degrees(np.arccos(cos))
        rep["normal_ok_frac"] = float(np.mean(ang <= NORMAL_DEG))
        rep["normal_p50_deg"] = float(np.median(ang))
        ga = np.asarray(gpu["rgba"]).reshape(-1, 4).astype(int)
        oa = np.asarray(ref["rgba"]).reshape(-1, 4).astype(int)
        diff = np.max(np.abs(ga[both] - oa[both]), axis=1)
        rep["rgba_ok_frac"] = float(np.mean(diff <= 1))
    else:
        rep["normal_ok_frac"] = rep["rgba_ok_frac"] = 1.0
    miss = ~hg
    rep["miss_planes_ok"] = bool(
        np.all(np.isinf(gd[miss]) & (gd[miss] > 0))
        and np.all(gn[miss] == 0.0)
        and np.all(np.asarray(gpu["rgba"]).reshape(-1, 4)[miss] == 0))
    rep["flip_budget"] = int(np.floor(flip_frac * n))
    return rep


def assert_parity(rep: dict, flip_frac: float = FLIP_FRAC, what: str = ""):
    msg = f"{what}: {rep}"
    assert rep["flips"] <= max(int(np.floor(flip_frac * rep["pixels"])), 0), msg
    assert rep["iter_mismatch"] == 0, msg
    assert rep["max_depth_err"] <= DEPTH_TOL, msg
    assert rep["normal_ok_frac"] >= GOOD_FRAC, msg
    assert rep["rgba_ok_frac"] >= GOOD_FRAC, msg
    assert rep["miss_planes_ok"], msg
