"""Stored fixtures: the constants the paper prints (transcribed with their
figure citations) against the seeded scene module, and a small oracle render
kept as a regression fixture of the oracle (written by
tests/golden/make_oracle_golden.py, which calls only the oracle)."""
import math
import os

import numpy as np

import oracle  # noqa: F401
from paper_2303_14827_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_paper_c_values_transcription():
    rows = {}
    for line in open(os.path.join(GOLDEN, "paper_c_values.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[parts[0]] = tuple(float(x) for x in parts[2:])
    assert rows == {k: tuple(float(x) for x in v) for k, v in scenes.PAPER_C_VALUES.items()}


def test_oracle_small_frames_unchanged():
    import sys
    sys.path.insert(0, GOLDEN)
    import make_oracle_golden as mk
    want = {}
    totals = {}
    for line in open(os.path.join(GOLDEN, "oracle_small_frames.txt")):
        parts = line.split()
        if line.startswith("# ") and len(parts) == 6:
            totals[parts[1]] = (int(parts[3]), int(parts[5]))
            continue
        if line.startswith("#"):
            continue
        want[(parts[0], int(parts[1]), int(parts[2]))] = (int(parts[3]), float(parts[4]),
                                                          tuple(int(v) for v in parts[5:9]))
    for name in mk.CASES:
        r = mk.render(name)
        assert (r["class_iters"], r["normal_iters"]) == totals[name]
        h, w = r["iter"].shape
        for j in range(h):
            for i in range(w):
                it, dep, rgba = want[(name, i, j)]
                assert int(r["iter"][j, i]) == it
                d = float(r["depth"][j, i])
                assert (d == dep) or (math.isinf(d) and math.isinf(dep))
                assert tuple(int(v) for v in r["rgba"][j, i]) == rgba
        assert np.isfinite(r["depth"]).sum() > 0
