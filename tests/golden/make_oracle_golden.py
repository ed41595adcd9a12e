"""Write oracle_small_frames.txt: small FP64 oracle renders (the default scene
with the march, and with sphere tracing) kept as a regression fixture for the
oracle itself.  Calls only the oracle; run it again only when a change of the
oracle's arithmetic is intended, and name the passage that justifies it in the
commit.

    python tests/golden/make_oracle_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2303_14827_gb300 import scenes  # noqa: E402

CASES = {
    "march": dict(width=24, height=16),
    "de": dict(width=24, height=16, traversal=scenes.TRAVERSAL_DE),
}


def render(name):
    return oracle.render(scenes.default_scene(**CASES[name]), threads=1)


def main():
    lines = ["# name i j iter depth(repr) rgba  -- written by make_oracle_golden.py (oracle only)"]
    for name in CASES:
        r = render(name)
        h, w = r["iter"].shape
        lines.append(f"# {name} class_iters {r['class_iters']} normal_iters {r['normal_iters']}")
        for j in range(h):
            for i in range(w):
                rgba = " ".join(str(int(v)) for v in r["rgba"][j, i])
                lines.append(f"{name} {i} {j} {int(r['iter'][j, i])} {float(r['depth'][j, i])!r} {rgba}")
    with open(os.path.join(HERE, "oracle_small_frames.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
