"""Renders the scenes of tests/test_gpu_kernel_forms.py in a process whose
kernel-form switches (DQJ_BISECT_GROUP, DQJ_MARCH_SAMPLES; read once per
process) the test sets, and
saves the output planes and counters."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def scenes_list():
    from paper_2303_14827_gb300 import scenes
    rng = np.random.default_rng(3)
    out = []
    for prec in (scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK, scenes.PRECISION_FP64):
        out.append(scenes.default_scene(precision=prec))
        out.append(scenes.default_scene(width=203, height=117, precision=prec,
                                        slice_basis=scenes.random_slice_frame(rng)))
    for b in (0, 1, 4, 5):
        out.append(scenes.default_scene(width=96, height=80, bisect_steps=b))
    out.append(scenes.default_scene(width=120, height=90, square_mode=scenes.SQUARE_PAPER_COMPONENTWISE,
                                    precision=scenes.PRECISION_FP32_RECHECK))
    out.append(scenes.default_scene(width=1920, height=1080, max_iter=16, march_steps=512, bisect_steps=10,
                                    precision=scenes.PRECISION_FP32_RECHECK))
    # long orbits: normals of more than the late step evaluated in FP64
    out.append(scenes.default_scene(width=320, height=240, max_iter=32, precision=scenes.PRECISION_FP32_RECHECK))
    out.append(scenes.default_scene(width=320, height=240, max_iter=20, modulus_mode=scenes.MODULUS_DUALNUM,
                                    precision=scenes.PRECISION_FP32_RECHECK))
    # march rounds of two samples per ray: even and odd sample counts, one or
    # two or three samples in all, one or two steps, the dual-number modulus
    for prec in (scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK):
        out.append(scenes.default_scene(width=77, height=45, march_steps=255, precision=prec))
        out.append(scenes.default_scene(width=40, height=24, march_steps=1, precision=prec))
        out.append(scenes.default_scene(width=40, height=24, march_steps=2, precision=prec))
        out.append(scenes.default_scene(width=64, height=40, max_iter=1, precision=prec))
        out.append(scenes.default_scene(width=64, height=40, max_iter=2, march_steps=100, precision=prec))
        out.append(scenes.default_scene(width=96, height=64, max_iter=8, modulus_mode=scenes.MODULUS_DUALNUM,
                                        precision=prec))
    # FP32 frames with more tiles than resident warps take the unsplit march
    out.append(scenes.default_scene(width=640, height=480, precision=scenes.PRECISION_FP32))
    out.append(scenes.default_scene(width=641, height=483, march_steps=255, precision=scenes.PRECISION_FP32))
    for prec in (scenes.PRECISION_FP32, scenes.PRECISION_FP32_RECHECK):
        out.append(scenes.default_scene(width=640, height=480, march_steps=255, precision=prec,
                                        slice_basis=scenes.random_slice_frame(rng)))
    return out


def main(path):
    import torch
    from paper_2303_14827_gb300 import binding
    binding.load()
    res = {}
    with binding.Renderer(0) as r:
        for i, s in enumerate(scenes_list()):
            o = r.render(s)
            torch.cuda.synchronize()
            w = s["width"]
            for k in ("iter", "depth", "normal", "rgba", "stats"):
                v = o[k]
                res[f"{i}_{k}"] = (v if k == "stats" else v[:, :w]).cpu().numpy()
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
