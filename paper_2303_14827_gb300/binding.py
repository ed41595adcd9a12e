"""ctypes binding of libdqj (include/dqj.h), same names as the C ABI.

Argument marshalling only: every step of the render runs in the library's CUDA
kernels.  A missing library is an error (``RuntimeError``), never a fallback.
Torch is used only to own device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "dqj.h")

DQJ_OK = 0
DQJ_ERR_INVALID = 1
DQJ_ERR_NOMEM = 2
DQJ_ERR_BUSY = 3
DQJ_ERR_TIMEOUT = 4
DQJ_ERR_CUDA = 5
DQJ_ERR_NOT_FOUND = 6
DQJ_ERR_CANCELLED = 7
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "BUSY", 4: "TIMEOUT", 5: "CUDA", 6: "NOT_FOUND",
                7: "CANCELLED"}

DQJ_FP32, DQJ_FP32_RECHECK, DQJ_FP64 = 0, 1, 2
STAT_NAMES = ("class_iters", "normal_iters", "samples", "hits", "rechecks", "fixups", "fixup_iters", "overflow",
              "march_iters", "reserved")
DQJ_NSTATS = len(STAT_NAMES)


class DqjError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dqj status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dqj_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_uint64),
                ("max_pending", ctypes.c_int32), ("autotune_cache", ctypes.c_char_p)]


class dqj_params(ctypes.Structure):
    _fields_ = [
        ("c", ctypes.c_double * 8),
        ("slice_origin", ctypes.c_double * 8),
        ("slice_basis", (ctypes.c_double * 8) * 3),
        ("eye", ctypes.c_double * 3),
        ("target", ctypes.c_double * 3),
        ("up", ctypes.c_double * 3),
        ("fov_y_deg", ctypes.c_double),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("escape_radius", ctypes.c_double),
        ("march_steps", ctypes.c_int32),
        ("bisect_steps", ctypes.c_int32),
        ("normal_h", ctypes.c_double),
        ("box_min", ctypes.c_double * 3),
        ("box_max", ctypes.c_double * 3),
        ("light_dir", ctypes.c_double * 3),
        ("k_ambient", ctypes.c_double),
        ("k_diffuse", ctypes.c_double),
        ("albedo", ctypes.c_double * 3),
        ("precision", ctypes.c_int32),
        ("recheck_margin", ctypes.c_double),
        ("square_mode", ctypes.c_int32),
        ("modulus_mode", ctypes.c_int32),
        ("k_specular", ctypes.c_double),
        ("shininess", ctypes.c_double),
        ("traversal", ctypes.c_int32),
        ("de_max_steps", ctypes.c_int32),
        ("de_epsilon", ctypes.c_double),
        ("de_step_scale", ctypes.c_double),
        ("de_bound_radius", ctypes.c_double),
    ]


class dqj_outputs(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("rgba", ctypes.c_void_p), ("pitch_px", ctypes.c_int64), ("stats", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def declared_symbols() -> list[str]:
    """Function names declared in include/dqj.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dqj_[a-z_0-9]+)\s*\(", text)))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libdqj.so, building it with nvcc if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            try:
                _build.build()
            except Exception as e:  # pragma: no cover - depends on the toolchain
                if not os.path.exists(path):
                    raise RuntimeError(f"libdqj.so is missing and could not be built: {e}") from e
        if not os.path.exists(path):
            raise RuntimeError(f"libdqj.so not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.dqj_default_params.argtypes = [P(dqj_params)]
        L.dqj_validate_params.argtypes = [P(dqj_params)]
        L.dqj_create.argtypes = [P(dqj_config), P(ctypes.c_void_p)]
        L.dqj_render.argtypes = [ctypes.c_void_p, P(dqj_params), P(dqj_outputs), ctypes.c_void_p]
        L.dqj_render_tiles.argtypes = [ctypes.c_void_p, P(dqj_params), P(dqj_outputs), ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_int32]
        L.dqj_render_batch.argtypes = [ctypes.c_void_p, P(dqj_params), P(dqj_outputs), ctypes.c_int32,
                                       ctypes.c_void_p]
        L.dqj_render_host.argtypes = [ctypes.c_void_p, P(dqj_params), P(dqj_outputs)]
        L.dqj_render_host_batch.argtypes = [ctypes.c_void_p, P(dqj_params), P(dqj_outputs), ctypes.c_int32]
        L.dqj_submit.argtypes = [ctypes.c_void_p, P(dqj_params), P(dqj_outputs), P(ctypes.c_uint64)]
        L.dqj_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_int), P(ctypes.c_int)]
        L.dqj_destroy.argtypes = [ctypes.c_void_p]
        L.dqj_last_error.restype = ctypes.c_char_p
        L.dqj_last_error.argtypes = []
        L.dqj_fma_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_double)]
        L.dqj_render_noalloc.argtypes = [P(dqj_params), P(dqj_outputs), ctypes.c_void_p]
        L.dqj_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.dqj_tile_shape.argtypes = [ctypes.c_void_p, P(dqj_params), P(ctypes.c_int32), P(ctypes.c_int32),
                                     P(ctypes.c_int32)]
        L.dqj_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.dqj_pass_ms.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_float)]
        L.dqj_serve_stats.argtypes = [ctypes.c_void_p, P(ctypes.c_int64)]
        L.dqj_voxelize.argtypes = [ctypes.c_void_p, P(dqj_params), ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.dqj_serve_policy.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.dqj_render_voxels.argtypes = [ctypes.c_void_p, P(dqj_params), ctypes.c_int32, ctypes.c_void_p,
                                        P(dqj_outputs), ctypes.c_void_p]
        for name in declared_symbols():
            fn = getattr(L, name)
            if name != "dqj_last_error":
                fn.restype = ctypes.c_int
        _lib = L
        return L


def last_error() -> str:
    return (load().dqj_last_error() or b"").decode()


def check(status: int) -> int:
    if status != DQJ_OK:
        raise DqjError(status, last_error())
    return status


# --------------------------------------------------------------------------
# parameter blocks
# --------------------------------------------------------------------------
def make_params(scene: dict) -> dqj_params:
    p = dqj_params()
    p.c[:] = [float(x) for x in scene["c"]]
    p.slice_origin[:] = [float(x) for x in scene["slice_origin"]]
    for r in range(3):
        p.slice_basis[r][:] = [float(x) for x in scene["slice_basis"][r]]
    for k in ("eye", "target", "up", "box_min", "box_max", "light_dir", "albedo"):
        getattr(p, k)[:] = [float(x) for x in scene[k]]
    for k in ("fov_y_deg", "escape_radius", "normal_h", "k_ambient", "k_diffuse", "recheck_margin"):
        setattr(p, k, float(scene[k]))
    p.k_specular = float(scene.get("k_specular", 0.0))
    p.shininess = float(scene.get("shininess", 32.0))
    p.traversal = int(scene.get("traversal", 0))
    p.de_max_steps = int(scene.get("de_max_steps", 512))
    p.de_epsilon = float(scene.get("de_epsilon", 1e-3))
    p.de_step_scale = float(scene.get("de_step_scale", 1.0))
    p.de_bound_radius = float(scene.get("de_bound_radius", 0.0))
    for k in ("width", "height", "max_iter", "march_steps", "bisect_steps", "precision", "square_mode",
              "modulus_mode"):
        setattr(p, k, int(scene[k]))
    return p


def params_to_dict(p: dqj_params) -> dict:
    out = {}
    for name, _ in dqj_params._fields_:
        v = getattr(p, name)
        if name == "slice_basis":
            out[name] = [list(v[r]) for r in range(3)]
        elif isinstance(v, ctypes.Array):
            out[name] = list(v)
        else:
            out[name] = v
    return out


def dqj_default_params() -> dqj_params:
    p = dqj_params()
    check(load().dqj_default_params(ctypes.byref(p)))
    return p


def dqj_validate_params(scene_or_params) -> int:
    p = scene_or_params if isinstance(scene_or_params, dqj_params) else make_params(scene_or_params)
    return load().dqj_validate_params(ctypes.byref(p))


# --------------------------------------------------------------------------
# context and rendering
# --------------------------------------------------------------------------
def dqj_create(device: int = 0, mem_budget_bytes: int = 0, max_pending: int = 0,
               autotune_cache: str | None = None) -> int:
    cfg = dqj_config(device, mem_budget_bytes, max_pending,
                     autotune_cache.encode() if autotune_cache else None)
    h = ctypes.c_void_p()
    check(load().dqj_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def dqj_destroy(ctx: int) -> None:
    check(load().dqj_destroy(ctypes.c_void_p(ctx)))


def _ptr(t):
    if t is None or isinstance(t, int):
        return t
    return t.data_ptr()


def make_outputs(iter=None, depth=None, normal=None, rgba=None, pitch_px: int = 0, stats=None) -> dqj_outputs:
    return dqj_outputs(_ptr(iter), _ptr(depth), _ptr(normal), _ptr(rgba), int(pitch_px), _ptr(stats))


def dqj_render(ctx: int, scene: dict, outputs: dqj_outputs, stream: int = 0) -> None:
    """Enqueue a frame on a CUDA stream handle (int, e.g. torch stream.cuda_stream)."""
    p = make_params(scene)
    check(load().dqj_render(ctypes.c_void_p(ctx), ctypes.byref(p), ctypes.byref(outputs),
                            ctypes.c_void_p(stream)))


def dqj_render_tiles(ctx: int, scene: dict, outputs: dqj_outputs, stream: int, part: int, parts: int) -> None:
    """Enqueue the frame's tiles t with t mod parts == part (the frame split)."""
    p = make_params(scene)
    check(load().dqj_render_tiles(ctypes.c_void_p(ctx), ctypes.byref(p), ctypes.byref(outputs),
                                  ctypes.c_void_p(stream), part, parts))


def tile_parts_of_pixels(ctx: int, scene: dict, parts: int):
    """(height, width) int array: the part of dqj_render_tiles that renders each
    pixel (its tile index mod parts), for putting the parts' planes together."""
    import numpy as np
    if scene.get("traversal", 0) == 1:
        tw, th = 8, 4
    else:
        _, tw, th = dqj_tile_shape(ctx, scene)
    w, h = scene["width"], scene["height"]
    tiles_x = (w + tw - 1) // tw
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    return ((ys // th) * tiles_x + xs // tw) % parts


def dqj_render_batch(ctx: int, scenes: list, outputs: list, stream: int) -> None:
    """Enqueue scenes[i] into the DEVICE outputs outputs[i] (dqj_outputs) on
    `stream`, frames pipelined by the library."""
    n = len(scenes)
    if len(outputs) != n:
        raise ValueError("scenes and outputs differ in length")
    ps = (dqj_params * max(n, 1))(*[make_params(s) for s in scenes])
    os_ = (dqj_outputs * max(n, 1))(*outputs)
    check(load().dqj_render_batch(ctypes.c_void_p(ctx), ps, os_, n, ctypes.c_void_p(stream)))


def dqj_render_host(ctx: int, scene: dict, outputs: dqj_outputs) -> None:
    p = make_params(scene)
    check(load().dqj_render_host(ctypes.c_void_p(ctx), ctypes.byref(p), ctypes.byref(outputs)))


def dqj_render_host_batch(ctx: int, scenes: list, outputs: list) -> None:
    """Render scenes[i] into the HOST buffers outputs[i] (dqj_outputs), copies
    overlapped with the next frame's render; blocking."""
    n = len(scenes)
    if len(outputs) != n:
        raise ValueError("scenes and outputs differ in length")
    ps = (dqj_params * max(n, 1))(*[make_params(s) for s in scenes])
    os_ = (dqj_outputs * max(n, 1))(*outputs)
    check(load().dqj_render_host_batch(ctypes.c_void_p(ctx), ps, os_, int(n)))


DQJ_NOALLOC_MAX_PIXELS = 262144
DQJ_VOXEL_MAX_GRID = 1024


def dqj_render_noalloc(scene: dict, outputs: dqj_outputs, stream: int = 0) -> None:
    """Render on the current device without any device allocation: the scratch
    is a fixed array inside the library (for callers that must not allocate
    device memory).  At most DQJ_NOALLOC_MAX_PIXELS pixels; FP32 or FP64."""
    p = make_params(scene)
    check(load().dqj_render_noalloc(ctypes.byref(p), ctypes.byref(outputs), ctypes.c_void_p(stream)))


def dqj_submit(ctx: int, scene: dict, outputs: dqj_outputs) -> int:
    p = make_params(scene)
    t = ctypes.c_uint64(0)
    check(load().dqj_submit(ctypes.c_void_p(ctx), ctypes.byref(p), ctypes.byref(outputs), ctypes.byref(t)))
    return t.value


def dqj_poll(ctx: int, ticket: int):
    """(done, status) for a ticket; raises on an unknown ticket."""
    done, res = ctypes.c_int(0), ctypes.c_int(0)
    check(load().dqj_poll(ctypes.c_void_p(ctx), ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(res)))
    return bool(done.value), int(res.value)


def dqj_autotune(ctx: int, max_classes: int = 0) -> None:
    """Pick the fastest march tile shape per frame-size class and iteration bucket."""
    check(load().dqj_autotune(ctypes.c_void_p(ctx), int(max_classes)))


def dqj_tile_shape(ctx: int, scene: dict):
    """(variant, tile_w, tile_h) the context would use for the scene."""
    p = make_params(scene)
    v, w, h = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(load().dqj_tile_shape(ctypes.c_void_p(ctx), ctypes.byref(p), ctypes.byref(v), ctypes.byref(w),
                                ctypes.byref(h)))
    return v.value, w.value, h.value


def dqj_set_profiling(ctx: int, ring_frames: int) -> None:
    check(load().dqj_set_profiling(ctypes.c_void_p(ctx), int(ring_frames)))


def dqj_pass_ms(ctx: int, frames: int) -> list:
    """Per-pass ms [march, bisect, recheck, fixup] of the `frames` latest
    profiled renders, oldest first (waits for them)."""
    ms = (ctypes.c_float * (4 * frames))()
    check(load().dqj_pass_ms(ctypes.c_void_p(ctx), int(frames), ms))
    return [list(ms[4 * i:4 * i + 4]) for i in range(frames)]


def dqj_voxelize(ctx: int, scene: dict, grid_n: int, occupancy=None, counts=None, stats=None,
                 stream: int = 0) -> None:
    """Voxel occupancy grid into caller-owned device buffers (torch tensors or
    raw pointers): occupancy uint8[g^3], counts uint16 (int16 tensor) [g^3],
    stats int64[DQJ_NSTATS]."""
    p = make_params(scene)
    check(load().dqj_voxelize(ctypes.c_void_p(ctx), ctypes.byref(p), int(grid_n), _ptr(occupancy), _ptr(counts),
                              _ptr(stats), ctypes.c_void_p(stream)))


def dqj_render_voxels(ctx: int, scene: dict, grid_n: int, occupancy, outputs: dqj_outputs, stream: int = 0) -> None:
    """Image of a grid_n^3 occupancy grid (device uint8, as dqj_voxelize writes
    it) from the scene camera into caller-owned planes (see make_outputs)."""
    p = make_params(scene)
    check(load().dqj_render_voxels(ctypes.c_void_p(ctx), ctypes.byref(p), int(grid_n), _ptr(occupancy),
                                   ctypes.byref(outputs), ctypes.c_void_p(stream)))


SERVE_STAT_NAMES = ("launches", "restarts", "packed", "plain", "batches", "admit_ns", "completed", "loops",
                    "max_active", "overlapped")


DQJ_SERVE_FIFO, DQJ_SERVE_SHORTEST = 0, 1


def dqj_serve_policy(ctx: int, policy: int) -> None:
    """Order of the persistent launch's requests (see dqj_serve_policy in dqj.h)."""
    check(load().dqj_serve_policy(ctypes.c_void_p(ctx), int(policy)))


def dqj_serve_stats(ctx: int) -> dict:
    """Serving counters of a context (see dqj_serve_stats in dqj.h)."""
    v = (ctypes.c_int64 * len(SERVE_STAT_NAMES))()
    check(load().dqj_serve_stats(ctypes.c_void_p(ctx), v))
    return dict(zip(SERVE_STAT_NAMES, list(v)))


def dqj_fma_peak(device: int = 0, variant: int = 0, launches: int = 3) -> float:
    f = ctypes.c_double(0.0)
    check(load().dqj_fma_peak(int(device), int(variant), int(launches), ctypes.byref(f)))
    return f.value


# --------------------------------------------------------------------------
# torch convenience layer (allocation only)
# --------------------------------------------------------------------------
def alloc_outputs(width: int, height: int, device="cuda", pitch_px: int | None = None, stats: bool = True):
    """Allocate output planes as torch tensors (row pitch = pitch_px pixels)."""
    import torch
    pitch = pitch_px or width
    t = {
        "iter": torch.empty((height, pitch), dtype=torch.int32, device=device),
        "depth": torch.empty((height, pitch), dtype=torch.float32, device=device),
        "normal": torch.empty((height, pitch, 3), dtype=torch.float32, device=device),
        "rgba": torch.empty((height, pitch, 4), dtype=torch.uint8, device=device),
    }
    if stats:
        t["stats"] = torch.empty(DQJ_NSTATS, dtype=torch.int64, device=device)  # every entry is written
    t["pitch_px"] = pitch
    return t


def outputs_of(t: dict) -> dqj_outputs:
    return make_outputs(t.get("iter"), t.get("depth"), t.get("normal"), t.get("rgba"), t["pitch_px"],
                        t.get("stats"))


class Renderer:
    """A context plus torch-owned outputs; ``render`` returns the output dict."""

    def __init__(self, device: int = 0, **cfg):
        self.device = device
        self.ctx = dqj_create(device, **cfg)

    def render(self, scene: dict, out: dict | None = None, stream=None, sync: bool = True) -> dict:
        import torch
        if out is None:
            out = alloc_outputs(int(scene["width"]), int(scene["height"]), device=f"cuda:{self.device}")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        dqj_render(self.ctx, scene, outputs_of(out), s.cuda_stream)
        if sync:
            s.synchronize()
        return out

    def close(self):
        if self.ctx:
            dqj_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def stats_dict(stats_tensor) -> dict:
    v = [int(x) for x in stats_tensor.tolist()]
    return dict(zip(STAT_NAMES, v))
