"""The error bound behind the voxel-grid image's FP32 face choice (no GPU).

The walk compares FP32 face distances m = fma(k, sd32, base32), where sd32 and
base32 are the FP32 roundings of the FP64 values sd = size / d and
base = (box_min - eye) / d, and k is a cell-plane index 0..g.  It trusts the
FP32 order of two faces only when they differ by more than 2^-21 times the sum
of (g |sd| + |base|) over the axes.  That is safe when each m lies within
E = 2^-23 (g |sd| + |base|) of its exact value (three roundings of at most
2^-24 relative each), with a factor 2 to spare.  This test checks E directly
over random rays, including near-parallel axes, whose sd and base are large.
The single-rounding FMA is emulated exactly: the product of two FP32 values is
exact in FP64, and the sum is formed in exact rational arithmetic before the
one rounding to FP32."""
from fractions import Fraction

import numpy as np
import pytest


def fma32(a: np.float32, b: np.float32, c: np.float32) -> np.float32:
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    # nearest FP32 (ties to even) of an exact rational: round via FP64 only when
    # that is exact, else bracket with the two neighbouring FP32 values
    f = np.float32(float(exact))
    lo, hi = (f, np.nextafter(f, np.float32(np.inf))) if Fraction(float(f)) <= exact else \
        (np.nextafter(f, np.float32(-np.inf)), f)
    dl, dh = exact - Fraction(float(lo)), Fraction(float(hi)) - exact
    if dl < dh:
        return lo
    if dh < dl:
        return hi
    return lo if (int(lo.view(np.uint32)) & 1) == 0 else hi


@pytest.mark.parametrize("g", [50, 100, 1024])
def test_fp32_face_distance_error_bound(g):
    rng = np.random.default_rng(g)
    box_min, box_max, eye = -2.0, 2.0, 3.5
    size = (box_max - box_min) / g
    worst = 0.0
    for trial in range(60):
        # direction components from ~1 down to ~1e-6 (near-parallel axes)
        d = float(rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-6.0, 0.0))
        e = float(rng.uniform(-3.5, 3.5)) if trial % 2 else eye
        inv = 1.0 / d
        base, sd = (box_min - e) * inv, size * inv
        b32, d32 = np.float32(base), np.float32(sd)
        if not (np.isfinite(b32) and np.isfinite(d32)):
            continue
        bound = 2.0 ** -23 * (g * abs(float(d32)) + abs(float(b32)))
        ks = np.unique(np.concatenate([np.arange(0, min(g, 40) + 1), rng.integers(0, g + 1, 40), [g]]))
        for k in ks:
            m32 = fma32(np.float32(k), d32, b32)
            err = abs(Fraction(float(m32)) - (Fraction(int(k)) * Fraction(sd) + Fraction(base)))
            assert err <= Fraction(bound), (g, d, e, int(k), float(err), bound)
            worst = max(worst, float(err) / bound)
    assert worst > 0.05  # the samples come near the bound, so it is not vacuous
