"""FP64 CPU oracle for the dual-quaternion Julia isosurface renderer.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path (``paper_2303_14827_gb300``) and never imports it; the product path
never imports this.

The arithmetic lives in ``dqj_oracle.c`` (plain C, IEEE double, built with
``-O2 -ffp-contract=off``); this module only builds it with gcc and marshals
arguments through ctypes.  A scene is a plain dict with the field names of the
renderer's parameter block (see ``paper_2303_14827_gb300.scenes``).

Every function follows a passage of Kenwright, "Dual-Quaternion Julia Fractals":
the quaternion and dual-quaternion products of the appendix, the iteration of
Eq. dqjulia2 with the escape rule of "Practical Considerations", the 3-D slice of
"Dimension Reduction", the march of "Ray-Marching", the normal of
"Lighting/Illumination" and Eq. phong.  The readings taken where the paper is
silent or garbled are listed in the header of ``dqj_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dqj_oracle.c")
_LIB = os.path.join(_HERE, "libdqj_oracle.so")
_lock = threading.Lock()
_lib = None

SQUARE_ALGEBRAIC = 0
SQUARE_PAPER_COMPONENTWISE = 1
MODULUS_EUCLID8 = 0
MODULUS_DUALNUM = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Scene(ctypes.Structure):
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


class Trace(ctypes.Structure):
    _fields_ = [
        ("box_hit", ctypes.c_int32),
        ("hit", ctypes.c_int32),
        ("k_first", ctypes.c_int32),
        ("n_star", ctypes.c_int32),
        ("esc_max", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("t_in", ctypes.c_double),
        ("t_out", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("lo", ctypes.c_double),
        ("hi", ctypes.c_double),
        ("depth", ctypes.c_double),
        ("o", ctypes.c_double * 3),
        ("d", ctypes.c_double * 3),
        ("class_iters", ctypes.c_int64),
        ("normal_iters", ctypes.c_int64),
        ("de_steps", ctypes.c_int32),
        ("pad2", ctypes.c_int32),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_quat_mul.argtypes = [_D, _D, _D]
            L.or_quat_dot.argtypes = [_D, _D]
            L.or_quat_dot.restype = ctypes.c_double
            for name in ("or_dq_add", "or_dq_mul"):
                getattr(L, name).argtypes = [_D, _D, _D]
            L.or_dq_conj.argtypes = [_D, _D]
            L.or_dq_magnitude.argtypes = [_D, _D]
            L.or_dq_square.argtypes = [_D, ctypes.c_int, _D]
            L.or_modulus.argtypes = [_D, ctypes.c_int]
            L.or_modulus.restype = ctypes.c_double
            L.or_dq_julia.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _D]
            L.or_quat_julia.argtypes = [_D, _D, ctypes.c_int, _D]
            L.or_classify.argtypes = [_D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, _D, _I64]
            L.or_classify.restype = ctypes.c_int
            L.or_camera_ray.argtypes = [ctypes.POINTER(Scene), ctypes.c_int, ctypes.c_int, _D, _D]
            L.or_box_clip.argtypes = [ctypes.POINTER(Scene), _D, _D, _D, _D]
            L.or_box_clip.restype = ctypes.c_int
            L.or_slice_point.argtypes = [ctypes.POINTER(Scene), _D, _D]
            L.or_trace_pixel.argtypes = [ctypes.POINTER(Scene), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(Trace)]
            L.or_default_threads.restype = ctypes.c_int
            L.or_render.argtypes = [ctypes.POINTER(Scene), _I64, ctypes.c_int64, ctypes.c_int,
                                    _I32, _D, _D, _U8, _I64, _I64, _I64]
            L.or_render.restype = ctypes.c_int
            L.or_de_distance.argtypes = [ctypes.POINTER(Scene), _D, _D, _I64]
            L.or_de_distance.restype = ctypes.c_int
            L.or_voxel_center.argtypes = [ctypes.POINTER(Scene), ctypes.c_int32, ctypes.c_int64, _D]
            L.or_voxelize.argtypes = [ctypes.POINTER(Scene), ctypes.c_int32, _I64, ctypes.c_int64, ctypes.c_int,
                                      _U8, _I32, _I64]
            L.or_voxelize.restype = ctypes.c_int
            L.or_voxel_render.argtypes = [ctypes.POINTER(Scene), ctypes.c_int32, _U8, ctypes.c_int, _I64,
                                          ctypes.c_int64, ctypes.c_int, _I32, _D, _D, _U8, _D]
            L.or_voxel_render.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _vec(x, n: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


# --------------------------------------------------------------------------
# Algebra (appendix) -- thin wrappers used by the pins.
# --------------------------------------------------------------------------
def quat_mul(a, b) -> np.ndarray:
    a, b, out = _vec(a, 4), _vec(b, 4), np.zeros(4)
    lib().or_quat_mul(_dp(a), _dp(b), _dp(out))
    return out


def quat_dot(a, b) -> float:
    a, b = _vec(a, 4), _vec(b, 4)
    return lib().or_quat_dot(_dp(a), _dp(b))


def dq_add(a, b) -> np.ndarray:
    a, b, out = _vec(a, 8), _vec(b, 8), np.zeros(8)
    lib().or_dq_add(_dp(a), _dp(b), _dp(out))
    return out


def dq_mul(a, b) -> np.ndarray:
    a, b, out = _vec(a, 8), _vec(b, 8), np.zeros(8)
    lib().or_dq_mul(_dp(a), _dp(b), _dp(out))
    return out


def dq_conj(a) -> np.ndarray:
    a, out = _vec(a, 8), np.zeros(8)
    lib().or_dq_conj(_dp(a), _dp(out))
    return out


def dq_magnitude(a) -> np.ndarray:
    a, out = _vec(a, 8), np.zeros(8)
    lib().or_dq_magnitude(_dp(a), _dp(out))
    return out


def dq_square(a, square_mode: int = SQUARE_ALGEBRAIC) -> np.ndarray:
    a, out = _vec(a, 8), np.zeros(8)
    lib().or_dq_square(_dp(a), int(square_mode), _dp(out))
    return out


def modulus(a, modulus_mode: int = MODULUS_EUCLID8) -> float:
    a = _vec(a, 8)
    return lib().or_modulus(_dp(a), int(modulus_mode))


def dq_julia(z0, c, n: int, square_mode: int = SQUARE_ALGEBRAIC) -> np.ndarray:
    z0, c, out = _vec(z0, 8), _vec(c, 8), np.zeros(8)
    lib().or_dq_julia(_dp(z0), _dp(c), int(n), int(square_mode), _dp(out))
    return out


def quat_julia(q0, c, n: int) -> np.ndarray:
    q0, c, out = _vec(q0, 4), _vec(c, 4), np.zeros(4)
    lib().or_quat_julia(_dp(q0), _dp(c), int(n), _dp(out))
    return out


def classify(z0, c, max_iter: int, escape_radius: float = 4.0,
             square_mode: int = SQUARE_ALGEBRAIC, modulus_mode: int = MODULUS_EUCLID8):
    """Escape count in 1..max_iter, or 0 for inside; also the last modulus."""
    z0, c = _vec(z0, 8), _vec(c, 8)
    m = ctypes.c_double(0.0)
    it = ctypes.c_int64(0)
    n = lib().or_classify(_dp(z0), _dp(c), int(max_iter), float(escape_radius),
                          int(square_mode), int(modulus_mode), ctypes.byref(m), ctypes.byref(it))
    return n, m.value


# --------------------------------------------------------------------------
# Scene and rendering.
# --------------------------------------------------------------------------
def make_scene(p: dict) -> Scene:
    s = Scene()
    s.c[:] = [float(x) for x in p["c"]]
    s.slice_origin[:] = [float(x) for x in p["slice_origin"]]
    for r in range(3):
        s.slice_basis[r][:] = [float(x) for x in p["slice_basis"][r]]
    s.eye[:] = [float(x) for x in p["eye"]]
    s.target[:] = [float(x) for x in p["target"]]
    s.up[:] = [float(x) for x in p["up"]]
    s.fov_y_deg = float(p["fov_y_deg"])
    s.width, s.height, s.max_iter = int(p["width"]), int(p["height"]), int(p["max_iter"])
    s.escape_radius = float(p["escape_radius"])
    s.march_steps, s.bisect_steps = int(p["march_steps"]), int(p["bisect_steps"])
    s.normal_h = float(p["normal_h"])
    s.box_min[:] = [float(x) for x in p["box_min"]]
    s.box_max[:] = [float(x) for x in p["box_max"]]
    s.light_dir[:] = [float(x) for x in p["light_dir"]]
    s.k_ambient, s.k_diffuse = float(p["k_ambient"]), float(p["k_diffuse"])
    s.albedo[:] = [float(x) for x in p["albedo"]]
    s.square_mode = int(p.get("square_mode", 0))
    s.modulus_mode = int(p.get("modulus_mode", 0))
    s.k_specular = float(p.get("k_specular", 0.0))
    s.shininess = float(p.get("shininess", 32.0))
    s.traversal = int(p.get("traversal", 0))
    s.de_max_steps = int(p.get("de_max_steps", 512))
    s.de_epsilon = float(p.get("de_epsilon", 1e-3))
    s.de_step_scale = float(p.get("de_step_scale", 1.0))
    s.de_bound_radius = float(p.get("de_bound_radius", 0.0))
    return s


def camera_ray(p: dict, i: int, j: int):
    s = make_scene(p)
    o, d = np.zeros(3), np.zeros(3)
    lib().or_camera_ray(ctypes.byref(s), int(i), int(j), _dp(o), _dp(d))
    return o, d


def box_clip(p: dict, o, d):
    s = make_scene(p)
    o, d = _vec(o, 3), _vec(d, 3)
    t0, t1 = ctypes.c_double(0), ctypes.c_double(0)
    hit = lib().or_box_clip(ctypes.byref(s), _dp(o), _dp(d), ctypes.byref(t0), ctypes.byref(t1))
    return bool(hit), t0.value, t1.value


def slice_point(p: dict, pt) -> np.ndarray:
    s = make_scene(p)
    pt, out = _vec(pt, 3), np.zeros(8)
    lib().or_slice_point(ctypes.byref(s), _dp(pt), _dp(out))
    return out


def trace_pixel(p: dict, i: int, j: int) -> dict:
    s = make_scene(p)
    t = Trace()
    lib().or_trace_pixel(ctypes.byref(s), int(i), int(j), ctypes.byref(t))
    out = {name: getattr(t, name) for name, _ in Trace._fields_ if name not in ("o", "d", "pad", "pad2")}
    out["o"] = np.array(t.o[:])
    out["d"] = np.array(t.d[:])
    return out


def default_threads() -> int:
    return int(lib().or_default_threads())


def render(p: dict, pixels=None, threads: int = 0, want_pixel_iters: bool = False) -> dict:
    """Render the scene (or the listed linear pixel indices) in FP64.

    Returns dict(iter int32, depth f64, normal f64[...,3], rgba u8[...,4],
    class_iters, normal_iters, threads).  Whole images come back shaped
    [height, width, ...]; pixel lists come back flat in list order.
    """
    s = make_scene(p)
    if pixels is None:
        n = int(p["width"]) * int(p["height"])
        shape = (int(p["height"]), int(p["width"]))
        pix_arr = None
    else:
        pix_arr = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).reshape(-1))
        n = pix_arr.size
        shape = (n,)
    it = np.zeros(n, np.int32)
    dep = np.zeros(n, np.float64)
    nor = np.zeros((n, 3), np.float64)
    rgba = np.zeros((n, 4), np.uint8)
    piters = np.zeros(n, np.int64) if want_pixel_iters else None
    ci, ni = ctypes.c_int64(0), ctypes.c_int64(0)
    used = lib().or_render(
        ctypes.byref(s),
        pix_arr.ctypes.data_as(_I64) if pix_arr is not None else None,
        ctypes.c_int64(n), int(threads),
        it.ctypes.data_as(_I32), _dp(dep), _dp(nor), rgba.ctypes.data_as(_U8),
        piters.ctypes.data_as(_I64) if piters is not None else None,
        ctypes.byref(ci), ctypes.byref(ni))
    out = {
        "iter": it.reshape(shape),
        "depth": dep.reshape(shape),
        "normal": nor.reshape(shape + (3,)),
        "rgba": rgba.reshape(shape + (4,)),
        "class_iters": int(ci.value),
        "normal_iters": int(ni.value),
        "threads": int(used),
    }
    if piters is not None:
        out["pixel_iters"] = piters.reshape(shape)
    return out


def voxel_center(p: dict, g: int, lin: int) -> np.ndarray:
    """Scene-space centre of linear voxel cell `lin` of the g^3 grid over the box."""
    out = np.zeros(3)
    lib().or_voxel_center(ctypes.byref(make_scene(p)), int(g), int(lin), _dp(out))
    return out


def voxelize(p: dict, g: int, cells=None, threads: int = 0) -> dict:
    """Voxel occupancy grid (Fig. voxels) in FP64: occupancy u8 (1 inside) and
    escape count int32 (0 inside) per cell.  Whole grids come back shaped
    [g, g, g] indexed [k, j, i] (x fastest); cell lists come back flat."""
    s = make_scene(p)
    if cells is None:
        n, shape, arr = g ** 3, (g, g, g), None
    else:
        arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
        n, shape = arr.size, (arr.size,)
    occ = np.zeros(n, np.uint8)
    cnt = np.zeros(n, np.int32)
    it = ctypes.c_int64(0)
    used = lib().or_voxelize(ctypes.byref(s), int(g), arr.ctypes.data_as(_I64) if arr is not None else None,
                             ctypes.c_int64(n), int(threads), occ.ctypes.data_as(_U8), cnt.ctypes.data_as(_I32),
                             ctypes.byref(it))
    return {"occupancy": occ.reshape(shape), "count": cnt.reshape(shape), "iters": int(it.value),
            "threads": int(used)}


def voxel_render(p: dict, occupancy, pixels=None, brute: bool = False, threads: int = 0) -> dict:
    """Image of a g^3 occupancy grid (u8, indexed [k, j, i] or flat) from the
    scene camera (Fig. voxels): the first occupied cube each pixel's ray
    crosses, found by the cell-by-cell walk, or with brute=True by the plain
    definition over all cubes (tiny grids).  Returns iter (cells crossed up to
    the hit), depth, normal (face normal), rgba, and gap, the smallest margin of
    a floating-point decision of the walk per pixel; shapes as render()."""
    s = make_scene(p)
    occ = np.ascontiguousarray(np.asarray(occupancy, dtype=np.uint8).reshape(-1))
    g = int(round(occ.size ** (1.0 / 3.0)))
    if g ** 3 != occ.size:
        raise ValueError("occupancy must hold g^3 cells")
    if pixels is None:
        n = int(p["width"]) * int(p["height"])
        shape = (int(p["height"]), int(p["width"]))
        pix_arr = None
    else:
        pix_arr = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).reshape(-1))
        n, shape = pix_arr.size, (pix_arr.size,)
    it = np.zeros(n, np.int32)
    dep = np.zeros(n, np.float64)
    nor = np.zeros((n, 3), np.float64)
    rgba = np.zeros((n, 4), np.uint8)
    gap = np.zeros(n, np.float64)
    used = lib().or_voxel_render(ctypes.byref(s), g, occ.ctypes.data_as(_U8), 1 if brute else 0,
                                 pix_arr.ctypes.data_as(_I64) if pix_arr is not None else None, ctypes.c_int64(n),
                                 int(threads), it.ctypes.data_as(_I32), _dp(dep), _dp(nor),
                                 rgba.ctypes.data_as(_U8), _dp(gap))
    return {"iter": it.reshape(shape), "depth": dep.reshape(shape), "normal": nor.reshape(shape + (3,)),
            "rgba": rgba.reshape(shape + (4,)), "gap": gap.reshape(shape), "threads": int(used)}


def de_distance(p: dict, point) -> tuple:
    """Distance estimate (Eq. distfract2) at a scene point: (escape count or 0
    when inside, estimate, DQ iterations)."""
    d = ctypes.c_double(0.0)
    it = ctypes.c_int64(0)
    pt = np.ascontiguousarray(np.asarray(point, dtype=np.float64))
    n = lib().or_de_distance(ctypes.byref(make_scene(p)), _dp(pt), ctypes.byref(d), ctypes.byref(it))
    return int(n), float(d.value), int(it.value)
