"""Python face of the FP64 CPU oracle (``pr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg import this module; the library never does.  It builds the C
oracle with gcc (OpenMP, no FP contraction) on first use and wraps it with
ctypes.  It imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pr_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libpr_oracle.so")
_lock = threading.Lock()
_lib = None

BG = 0xFFFFFFFF


class OrView(C.Structure):
    _fields_ = [("tan_x", C.c_double), ("tan_y", C.c_double), ("z_near", C.c_double),
                ("pose0", C.c_double * 16), ("pose1", C.c_double * 16),
                ("fovea", C.c_double * 2), ("alpha", C.c_double), ("d", C.c_double * 2),
                ("light_w", C.c_double * 3), ("k_a", C.c_double), ("k_d", C.c_double),
                ("k_s", C.c_double), ("shininess", C.c_double),
                ("W", C.c_int32), ("H", C.c_int32), ("mode", C.c_int32), ("p_n", C.c_int32),
                ("p_lut", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (idempotent)."""
    with _lock:
        if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.or_render.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P, P, C.c_int64, P, P, P, P, P, P, P, P]
        L.or_eval.argtypes = [P, P, P, P, C.c_int64, C.c_int64, P]
        L.or_grad.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P, P, C.c_int64, P, P, P, P, P]
        L.or_pixels.argtypes = [P, P, C.c_int64, P, P, P]
        L.or_q.argtypes = [P, P, P]
        L.or_qinv.argtypes = [P, P, P]
        L.or_light.argtypes = [P, C.c_double, P]
        L.or_p.argtypes = [C.c_double, C.c_double]
        L.or_p.restype = C.c_double
        L.or_pinv.argtypes = [C.c_double, C.c_double]
        L.or_pinv.restype = C.c_double
        L.or_num_threads.restype = C.c_int
        L.or_unfoveate.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int32, C.c_double, P, C.c_int64, P, P]
        L.or_mip_levels.argtypes = [C.c_int64, C.c_int64, P]
        L.or_mip_levels.restype = C.c_int64
        L.or_unfoveate_lod.argtypes = [P, P, C.c_int64, C.c_int64]
        L.or_unfoveate_lod.restype = C.c_double
        _lib = L
    return _lib


def _f32(x) -> float:
    return float(np.float32(x))


def make_view(view) -> OrView:
    """Widen a ``scenes.View``-like object (any object with the same fields)
    into the oracle's FP64 view record.  The method's inputs are the FP32
    values the library takes (camera, poses, fovea, scan direction), so each
    field is rounded to FP32 first and then widened exactly."""
    v = OrView()
    v.W, v.H, v.mode = int(view.W), int(view.H), int(view.mode)
    v.tan_x, v.tan_y, v.z_near = _f32(view.tan_x), _f32(view.tan_y), _f32(view.z_near)
    p0 = np.asarray(view.pose0, dtype=np.float32).astype(np.float64).reshape(16)
    p1 = np.asarray(view.pose1, dtype=np.float32).astype(np.float64).reshape(16)
    for k in range(16):
        v.pose0[k] = p0[k]
        v.pose1[k] = p1[k]
    v.fovea[0], v.fovea[1] = _f32(view.fovea[0]), _f32(view.fovea[1])
    v.alpha = _f32(view.alpha)
    v.d[0], v.d[1] = _f32(view.d[0]), _f32(view.d[1])
    for k in range(3):
        v.light_w[k] = _f32(view.light_w[k])
    v.k_a, v.k_d = _f32(view.k_a), _f32(view.k_d)
    v.k_s, v.shininess = _f32(getattr(view, "k_s", 0.0)), _f32(getattr(view, "shininess", 1.0))
    lut = getattr(view, "p_lut", None)
    if lut is not None:
        # the FP32 samples the library takes, widened exactly; kept alive on the record
        arr = np.ascontiguousarray(np.asarray(lut, dtype=np.float32).astype(np.float64))
        v._keep = arr
        v.p_n = arr.size - 1
        v.p_lut = arr.ctypes.data
    return v


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def render(view, pos, vel, col, tri, pix=None, near=False):
    """FP64 render of the listed pixels (all when ``pix`` is None).

    Returns a dict of numpy arrays: id (uint32), depth (float32), s (float64),
    rgb (float64 [n,3]), bmin (winner's smallest barycentric), gap (relative
    depth gap to the next hit), cos (|cosine| between the ray and the
    winner's plane normal: the conditioning of its depth) and, with
    ``near=True``, near (edge margin of every potential occluder; costs a
    second sweep)."""
    L = lib()
    v = make_view(view)
    pos, vel, col = _d(pos), _d(vel), _d(col)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    if pix is None:
        n = int(view.W) * int(view.H)
        pixp = None
    else:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        n = int(pix.shape[0])
        pixp = pix
    out = {"id": np.empty(n, np.uint32), "depth": np.empty(n, np.float32), "s": np.empty(n, np.float64),
           "rgb": np.empty((n, 3), np.float64), "bmin": np.empty(n, np.float64), "gap": np.empty(n, np.float64),
           "cos": np.empty(n, np.float64)}
    if near:
        out["near"] = np.empty(n, np.float64)
    L.or_render(C.byref(v), pos.shape[0], tri.shape[0], _ptr(pos), _ptr(vel), _ptr(col), _ptr(tri),
                _ptr(pixp), n, _ptr(out["id"]), _ptr(out["depth"]), _ptr(out["s"]), _ptr(out["rgb"]),
                _ptr(out["bmin"]), _ptr(out["gap"]), _ptr(out.get("near")), _ptr(out["cos"]))
    return out


def evaluate(view, pos, vel, tri, lin: int, tri_id: int):
    """(b0, b1, b2, s, hit, display edge distance) of one triangle at one
    pixel, in FP64."""
    L = lib()
    v = make_view(view)
    pos, vel = _d(pos), _d(vel)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    out = np.empty(6, np.float64)
    L.or_eval(C.byref(v), _ptr(pos), _ptr(vel), _ptr(tri), int(lin), int(tri_id), _ptr(out))
    return out


def grad(view, pos, vel, col, tri, ids, g, pix=None):
    """FP64 gradient of sum(g * rgb) w.r.t. colours, positions, velocities
    ([V,3] each), visible ids held fixed."""
    L = lib()
    v = make_view(view)
    pos, vel, col = _d(pos), _d(vel), _d(col)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    g = _d(g).reshape(-1, 3)
    if pix is not None:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
    n = ids.shape[0]
    V = pos.shape[0]
    dcol, dpos, dvel = np.zeros((V, 3)), np.zeros((V, 3)), np.zeros((V, 3))
    L.or_grad(C.byref(v), V, tri.shape[0], _ptr(pos), _ptr(vel), _ptr(col), _ptr(tri), _ptr(pix), n,
              _ptr(ids), _ptr(g), _ptr(dcol), _ptr(dpos), _ptr(dvel))
    return dcol, dpos, dvel


def pixels(view, pix=None):
    """Per-pixel time t, display location x [n,2] and ray direction [n,3]."""
    L = lib()
    v = make_view(view)
    if pix is None:
        n = int(view.W) * int(view.H)
    else:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        n = pix.shape[0]
    t, x, d = np.empty(n), np.empty((n, 2)), np.empty((n, 3))
    L.or_pixels(C.byref(v), _ptr(pix), n, _ptr(t), _ptr(x), _ptr(d))
    return t, x, d


def q(view, u):
    """Framebuffer -> display map of the oracle (unit coordinates)."""
    L = lib()
    v = make_view(view)
    u = _d(u).reshape(2)
    x = np.empty(2)
    L.or_q(C.byref(v), _ptr(u), _ptr(x))
    return x


def qinv(view, x):
    L = lib()
    v = make_view(view)
    x = _d(x).reshape(2)
    u = np.empty(2)
    L.or_qinv(C.byref(v), _ptr(x), _ptr(u))
    return u


def light(view, t: float):
    L = lib()
    v = make_view(view)
    out = np.empty(3)
    L.or_light(C.byref(v), float(t), _ptr(out))
    return out


def p(dist: float, alpha: float) -> float:
    return lib().or_p(float(dist), float(alpha))


def pinv(r: float, alpha: float) -> float:
    return lib().or_pinv(float(r), float(alpha))


def unfoveate(view, rgb, Wd: int, Hd: int, method: str = "mip", sigma: float = 0.5, pix=None):
    """Display image I_u(x) = I_f(q^-1(x)) of a planar framebuffer image rgb
    [3][H][W] (Sec. 3.1.1, "Display"): method "mip" (MIP pyramid, tri-linear,
    3-tap cubic) or "projected" (5 x 5 Gaussian reconstruction filter of
    width sigma display pixels).  Returns (out [3][npix] or [3][Hd][Wd],
    margin [npix]): margin = distance in texels of the discrete texel choices
    from their decision boundaries."""
    L = lib()
    v = make_view(view)
    img = np.ascontiguousarray(np.asarray(rgb, dtype=np.float32).reshape(-1))
    assert img.size == 3 * view.W * view.H
    if pix is None:
        npix, pp = Wd * Hd, None
    else:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        npix, pp = pix.size, pix.ctypes.data_as(C.c_void_p)
    out = np.empty(3 * npix)
    margin = np.empty(npix)
    L.or_unfoveate(C.byref(v), img.ctypes.data_as(C.c_void_p), int(Wd), int(Hd), 0 if method == "mip" else 1,
                   float(sigma), pp, int(npix), out.ctypes.data_as(C.c_void_p), margin.ctypes.data_as(C.c_void_p))
    out = out.reshape(3, npix) if pix is not None else out.reshape(3, Hd, Wd)
    return out, margin


def unfoveate_lod(view, x, Wd: int, Hd: int) -> float:
    v = make_view(view)
    xx = _d(x).reshape(2)
    return lib().or_unfoveate_lod(C.byref(v), _ptr(xx), int(Wd), int(Hd))


def mip_levels(W: int, H: int):
    L = lib()
    n = L.or_mip_levels(int(W), int(H), None)
    dims = np.empty(2 * n, dtype=np.int64)
    L.or_mip_levels(int(W), int(H), dims.ctypes.data_as(C.c_void_p))
    return [(int(dims[2 * k]), int(dims[2 * k + 1])) for k in range(n)]


def num_threads() -> int:
    return int(lib().or_num_threads())
