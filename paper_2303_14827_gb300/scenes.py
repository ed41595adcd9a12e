"""Seeded synthetic scenes for the dual-quaternion Julia renderer.

This module only builds parameter dicts (random numbers, a QR factorisation for
random slice frames, arrival times).  It holds none of the renderer's arithmetic,
so both the CUDA path and the independent FP64 checker read the same inputs from
it.  The dict field names are those of the C parameter block ``dqj_params``.

The paper (Kenwright, "Dual-Quaternion Julia Fractals") renders with no dataset:
its workloads are the constants c printed in its figure captions (Fig. test2,
Fig. highres2, Fig. highres), with iteration counts "typically between 6 and 15"
(Method, after Eq. dqjulia2).  The scenes below reuse those constants and draw
further ones at random with the same magnitude.
"""
from __future__ import annotations

import copy

import numpy as np

TRAVERSAL_MARCH = 0  # fixed-step march + bisection
TRAVERSAL_DE = 1     # distance-estimate sphere tracing (Eq. distfract2)
PRECISION_FP32 = 0
PRECISION_FP32_RECHECK = 1
PRECISION_FP64 = 2

SQUARE_ALGEBRAIC = 0
SQUARE_PAPER_COMPONENTWISE = 1
MODULUS_EUCLID8 = 0
MODULUS_DUALNUM = 1

#: c of the single-frame scene, (q_r | q_d), scalar first in each half.
C_DEFAULT = (-0.2, 0.6, 0.2, 0.2, 0.1, 0.0, 0.0, 0.05)

#: Constants printed in the paper's captions.  Fig. test2 (six random c; its
#: first dual scalar is printed "-023" and read as -0.23), Fig. highres2 (n=15),
#: Fig. highres (n=15).
PAPER_C_VALUES = {
    "test2_a": (-0.10, 0.8, -0.26, 0.15, -0.23, -0.38, -0.86, 0.64),
    "test2_b": (-0.67, -0.54, -0.07, 0.02, 0.06, -0.53, 0.15, -0.27),
    "test2_c": (-0.98, 0.27, 0.40, 0.20, -0.37, -0.41, -0.24, -0.34),
    "test2_d": (0.35, 0.78, 0.85, -0.57, -0.22, 0.06, -0.46, 0.05),
    "test2_e": (-0.17, -0.28, 0.11, 0.8, 0.06, 0.44, -0.66, 0.06),
    "test2_f": (-0.04, 0.95, 0.4, -0.43, 0.09, -0.45, -0.27, -0.31),
    "highres2": (-0.04, 0.95, 0.4, -0.43, 0.09, -0.35, -0.27, -0.31),
    "highres": (-0.39054, -0.58679, 0.0, 0.0, 0.0, 0.5632, 0.0, 0.05),
}

RESOLUTIONS = ((256, 256), (512, 512), (1024, 1024), (1920, 1080))
SERVE_RES_WEIGHTS = (0.4, 0.3, 0.2, 0.1)


def _axis_frame():
    b = np.zeros((3, 8))
    b[0, 0] = b[1, 1] = b[2, 2] = 1.0
    return b.tolist()


def default_scene(**overrides) -> dict:
    """256x256 single frame: c = C_DEFAULT, real-quaternion coords (0,1,2) free,
    the other five fixed at 0; max_iter 12, R = 4, 256 march steps over the
    [-2,2]^3 box, 8 bisection steps; eye at distance 3.5 on +z looking at the
    origin, 45 degree vertical field of view."""
    s = {
        "c": list(C_DEFAULT),
        "slice_origin": [0.0] * 8,
        "slice_basis": _axis_frame(),
        "eye": [0.0, 0.0, 3.5],
        "target": [0.0, 0.0, 0.0],
        "up": [0.0, 1.0, 0.0],
        "fov_y_deg": 45.0,
        "width": 256,
        "height": 256,
        "max_iter": 12,
        "escape_radius": 4.0,
        "march_steps": 256,
        "bisect_steps": 8,
        "normal_h": 1e-4,
        "box_min": [-2.0, -2.0, -2.0],
        "box_max": [2.0, 2.0, 2.0],
        "light_dir": [1.0, 1.0, 1.0],
        "k_ambient": 0.15,
        "k_diffuse": 0.85,
        "albedo": [1.0, 1.0, 1.0],
        "precision": PRECISION_FP32,
        "recheck_margin": 1e-3,
        "square_mode": SQUARE_ALGEBRAIC,
        "modulus_mode": MODULUS_EUCLID8,
        "k_specular": 0.0,
        "shininess": 32.0,
        "traversal": TRAVERSAL_MARCH,
        "de_max_steps": 512,
        "de_epsilon": 1e-3,
        "de_step_scale": 1.0,
        "de_bound_radius": 0.0,
    }
    for k, v in overrides.items():
        if k not in s:
            raise KeyError(f"unknown scene field {k!r}")
        s[k] = copy.deepcopy(v)
    return s


def random_c(rng: np.random.Generator, lo: float = -0.8, hi: float = 0.8) -> list:
    return rng.uniform(lo, hi, 8).tolist()


def full_hd_scene(seed: int, **overrides) -> dict:
    """1920x1080 frame, c ~ U[-0.8, 0.8]^8 from numpy default_rng(seed),
    max_iter 16, 512 march steps, 10 bisection steps, h = 1e-4."""
    rng = np.random.default_rng(seed)
    base = dict(c=random_c(rng), width=1920, height=1080, max_iter=16, march_steps=512,
                bisect_steps=10, normal_h=1e-4)
    base.update(overrides)
    return default_scene(**base)


def random_slice_frame(rng: np.random.Generator) -> list:
    """Orthonormal 3-frame in R^8: Q of the QR factorisation of an 8x3 Gaussian."""
    g = rng.standard_normal((8, 3))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q.T.tolist()


def batch_scenes(seed: int = 1, n: int = 64, **overrides) -> list:
    """Mixed batch: resolution uniform over RESOLUTIONS, c ~ U[-0.8,0.8]^8, a
    random slice frame, max_iter ~ U{8..32}; 512 march steps, 10 bisection steps."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w, h = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
        c = random_c(rng)
        frame = random_slice_frame(rng)
        mi = int(rng.integers(8, 33))
        s = default_scene(c=c, slice_basis=frame, width=w, height=h, max_iter=mi,
                          march_steps=512, bisect_steps=10)
        for k, v in overrides.items():
            s[k] = copy.deepcopy(v)
        out.append(s)
    return out


def serving_stream(seed: int = 2, n: int = 10000, rate_hz: float = 100.0,
                   step_sigma: float = 0.01, **overrides) -> list:
    """Poisson arrivals of render requests mimicking interactive exploration.

    Returns a list of (arrival_time_s, scene).  Resolution weights 0.4/0.3/0.2/0.1
    over RESOLUTIONS, max_iter ~ U{8..32}, c a Gaussian random walk (sigma per
    component per request) from C_DEFAULT, default slice, 512 march + 10 bisection
    steps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    c = np.array(C_DEFAULT, dtype=np.float64)
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        w, h = RESOLUTIONS[int(rng.choice(len(RESOLUTIONS), p=SERVE_RES_WEIGHTS))]
        mi = int(rng.integers(8, 33))
        c = c + rng.normal(0.0, step_sigma, 8)
        s = default_scene(c=c.tolist(), width=w, height=h, max_iter=mi, march_steps=512,
                          bisect_steps=10)
        for k, v in overrides.items():
            s[k] = copy.deepcopy(v)
        out.append((t, s))
    return out


def sample_pixels(width: int, height: int, count: int, seed: int = 0) -> np.ndarray:
    """Distinct linear pixel indices (row * width + col), sorted."""
    rng = np.random.default_rng(seed)
    n = width * height
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)
