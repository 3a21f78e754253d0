"""ctypes binding of libpr (include/pr.h), one Python function per C entry
point with the same name.  Argument marshalling only: tensors and arrays are
passed as raw pointers (device or host), the current torch CUDA stream as
the stream, and a non-OK status raises PrError.  Every step of the path runs
in the library's CUDA kernels; there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PR_OK, PR_ERR_INVALID_ARG, PR_ERR_CUDA, PR_ERR_OOM, PR_ERR_OVERFLOW, PR_ERR_TIMEOUT, PR_ERR_NONFINITE, \
    PR_ERR_NO_CUDA = range(8)
PR_CLASSIC, PR_ROLLING, PR_FOVEATED, PR_BOTH = range(4)
PR_BOUND_ZENON, PR_BOUND_ADAPTIVE, PR_BOUND_HULL, PR_BOUND_QUAD, PR_BOUND_TRIVIAL = range(5)
PR_FOV_SECTOR, PR_FOV_SIMPLE, PR_FOV_RECURSIVE = range(3)
FOV_BOUND_NAMES = {"sector": PR_FOV_SECTOR, "simple": PR_FOV_SIMPLE, "recursive": PR_FOV_RECURSIVE}
BOUND_NAMES = {"zenon": 0, "adaptive": 1, "hull": 2, "quad": 3, "trivial": 4}
BG = 0xFFFFFFFF

EXPORTS = ("pr_scene_upload", "pr_scene_update", "pr_scene_free", "pr_rasterize", "pr_shade", "pr_backward",
           "pr_workspace_create", "pr_workspace_free", "pr_rasterize_batch", "pr_graph_capture_batch",
           "pr_graph_launch", "pr_graph_free", "pr_scene_stats", "pr_workspace_stats", "pr_debug_bounds",
           "pr_debug_catch_interval", "pr_status_string", "pr_version", "pr_rasterize_noalloc",
           "pr_backward_batch", "pr_frame_batch", "pr_graph_capture_frame", "pr_unfoveate", "pr_foveation_create",
           "pr_foveation_free", "pr_graph_enqueue", "pr_graph_status", "pr_measure_fp32_peak",
           "pr_debug_scan_timeout", "pr_debug_halfplanes", "pr_scene_update_batch", "pr_unfoveate_batch")


class PrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class PrView(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("mode", C.c_int32), ("pad0", C.c_int32),
                ("tan_x", C.c_float), ("tan_y", C.c_float), ("z_near", C.c_float), ("alpha", C.c_float),
                ("pose0", C.c_float * 16), ("pose1", C.c_float * 16), ("fovea", C.c_float * 2),
                ("d", C.c_float * 2), ("light_w", C.c_float * 3), ("k_a", C.c_float), ("k_d", C.c_float),
                ("k_s", C.c_float), ("shininess", C.c_float), ("foveation", C.c_void_p)]


class PrParams(C.Structure):
    _fields_ = [("bound", C.c_int32), ("tile", C.c_int32), ("fp64_retest", C.c_int32), ("seg", C.c_int32),
                ("fov_bound", C.c_int32), ("graph_stage_times", C.c_int32)]


class PrStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("tests", "hits", "pairs", "items", "culled", "flagged", "changed",
                                          "pixels")] + [("stage_ms", C.c_float * 8), ("fp64_depth_err", C.c_float),
                                                        ("pad_stats", C.c_float)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, _ in self._fields_ if n not in ("stage_ms", "fp64_depth_err", "pad_stats")}
        d["stage_ms"] = [float(x) for x in self.stage_ms]
        d["fp64_depth_err"] = float(self.fp64_depth_err)
        return d


class PrBackwardView(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("view", PrView), ("id", C.c_void_p), ("grad_rgb", C.c_void_p),
                ("dcol", C.c_void_p), ("dpos", C.c_void_p), ("dvel", C.c_void_p)]


class PrUnfoveateParams(C.Structure):
    _fields_ = [("method", C.c_int32), ("Wd", C.c_int32), ("Hd", C.c_int32), ("sigma", C.c_float)]


class PrUnfoveateEntry(C.Structure):
    _fields_ = [("view", C.c_void_p), ("rgb", C.c_void_p), ("out", C.c_void_p), ("Wd", C.c_int32),
                ("Hd", C.c_int32)]


UNFOVEATE_METHODS = {"mip": 0, "projected": 1}


class PrFrameGrad(C.Structure):
    _fields_ = [("grad_rgb", C.c_void_p), ("target_rgb", C.c_void_p), ("dcol", C.c_void_p), ("dpos", C.c_void_p),
                ("dvel", C.c_void_p), ("target_u8", C.c_void_p), ("loss", C.c_void_p)]


class PrBatchView(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("view", PrView), ("id_out", C.c_void_p), ("depth_out", C.c_void_p),
                ("rgb_out", C.c_void_p), ("tile", C.c_int32), ("pad", C.c_int32)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpr.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.is_stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libpr.so is not built ({_build.LIB}); run paper_1806_05385_gb300.build")
        L = C.CDLL(_build.LIB)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "pr_scene_upload": ([P, P, P, P, I64, I64, P, C.POINTER(P)], I32),
            "pr_scene_update": ([P, P, P, P, P], I32),
            "pr_scene_update_batch": ([P, I32, P, P, P, P], I32),
            "pr_scene_free": ([P], None),
            "pr_rasterize": ([P, C.POINTER(PrView), C.POINTER(PrParams), P, P, P], I32),
            "pr_shade": ([P, C.POINTER(PrView), P, P, P], I32),
            "pr_backward": ([P, C.POINTER(PrView), P, P, P, P, P, P], I32),
            "pr_workspace_create": ([C.POINTER(P)], I32),
            "pr_workspace_free": ([P], None),
            "pr_rasterize_batch": ([P, C.POINTER(PrBatchView), I32, C.POINTER(PrParams), P], I32),
            "pr_graph_capture_batch": ([P, C.POINTER(PrBatchView), I32, C.POINTER(PrParams), P, C.POINTER(P)], I32),
            "pr_graph_launch": ([P, P], I32),
            "pr_graph_enqueue": ([P, P], I32),
            "pr_graph_status": ([P], I32),
            "pr_measure_fp32_peak": ([P, C.POINTER(C.c_double)], I32),
            "pr_debug_scan_timeout": ([P], I32),
            "pr_graph_free": ([P], None),
            "pr_scene_stats": ([P, C.POINTER(PrStats)], I32),
            "pr_workspace_stats": ([P, C.POINTER(PrStats)], I32),
            "pr_debug_bounds": ([P, P, P], I32),
            "pr_debug_halfplanes": ([P, P, P], I32),
            "pr_debug_catch_interval": ([C.POINTER(PrView), P, P, P], I32),
            "pr_status_string": ([I32], C.c_char_p),
            "pr_version": ([], I32),
            "pr_rasterize_noalloc": ([P, P, P, P, I64, I64, C.POINTER(PrView), C.POINTER(PrParams), P, P, P], I32),
            "pr_backward_batch": ([P, C.POINTER(PrBackwardView), I32, P], I32),
            "pr_unfoveate": ([P, C.POINTER(PrView), P, P, C.POINTER(PrUnfoveateParams), P], I32),
            "pr_unfoveate_batch": ([P, C.POINTER(PrUnfoveateEntry), I32, C.POINTER(PrUnfoveateParams), P], I32),
            "pr_foveation_create": ([P, I32, C.POINTER(P)], I32),
            "pr_foveation_free": ([P], None),
            "pr_frame_batch": ([P, C.POINTER(PrBatchView), I32, C.POINTER(PrParams), C.POINTER(PrFrameGrad), P], I32),
            "pr_graph_capture_frame": ([P, C.POINTER(PrBatchView), I32, C.POINTER(PrParams), C.POINTER(PrFrameGrad), P,
                                        C.POINTER(P)], I32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def status_string(s: int) -> str:
    return load().pr_status_string(int(s)).decode()


def _check(s: int, where: str):
    if s != PR_OK:
        raise PrError(s, where)


def _ptr(a):
    """Raw pointer of a torch tensor, numpy array or None (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return C.c_void_p(a)
    raise TypeError(f"cannot pass {type(a)} as a buffer")


def current_stream():
    import torch
    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


def make_view(v) -> PrView:
    """PrView from any object with the fields of ``scenes.View``."""
    out = PrView()
    out.W, out.H, out.mode = int(v.W), int(v.H), int(v.mode)
    out.tan_x, out.tan_y, out.z_near, out.alpha = float(v.tan_x), float(v.tan_y), float(v.z_near), float(v.alpha)
    p0 = np.asarray(v.pose0, dtype=np.float32).reshape(16)
    p1 = np.asarray(v.pose1, dtype=np.float32).reshape(16)
    for k in range(16):
        out.pose0[k] = float(p0[k])
        out.pose1[k] = float(p1[k])
    out.fovea[0], out.fovea[1] = float(v.fovea[0]), float(v.fovea[1])
    out.d[0], out.d[1] = float(v.d[0]), float(v.d[1])
    for k in range(3):
        out.light_w[k] = float(v.light_w[k])
    out.k_a, out.k_d = float(v.k_a), float(v.k_d)
    out.k_s, out.shininess = float(getattr(v, "k_s", 0.0)), float(getattr(v, "shininess", 1.0))
    lut = getattr(v, "p_lut", None)
    out.foveation = foveation_handle(lut) if lut is not None else None
    return out


def make_params(bound=PR_BOUND_ZENON, tile=0, fp64_retest=0, seg=0, fov_bound=PR_FOV_SECTOR,
                graph_stage_times=0) -> PrParams:
    if isinstance(bound, str):
        bound = BOUND_NAMES[bound]
    if isinstance(fov_bound, str):
        fov_bound = FOV_BOUND_NAMES[fov_bound]
    return PrParams(int(bound), int(tile), int(fp64_retest), int(seg), int(fov_bound), int(graph_stage_times))


# ------------------------------------------------------------------ entry points

def pr_scene_upload(pos, vel, col, tri, stream=None) -> int:
    """Returns the scene handle (an int)."""
    L = load()
    h = C.c_void_p()
    V = int(pos.shape[0])
    T = int(tri.shape[0])
    _check(L.pr_scene_upload(_ptr(pos), _ptr(vel), _ptr(col), _ptr(tri), V, T,
                             stream if stream is not None else current_stream(), C.byref(h)), "pr_scene_upload")
    return h.value


def pr_scene_update(scene, pos=None, vel=None, col=None, stream=None):
    _check(load().pr_scene_update(C.c_void_p(scene), _ptr(pos), _ptr(vel), _ptr(col),
                                  stream if stream is not None else current_stream()), "pr_scene_update")


def pr_scene_update_batch(scenes, pos=None, vel=None, col=None, stream=None):
    """pr_scene_update for several scenes in one call: scenes a list of
    handles; pos, vel, col lists of CUDA tensors (entries may be None) or
    None."""
    n = len(scenes)
    hs = (C.c_void_p * n)(*[C.c_void_p(h) for h in scenes])

    def arr(lst):
        if lst is None:
            return None
        a = (C.c_void_p * n)()
        for k, t in enumerate(lst):
            p = _ptr(t)
            a[k] = p.value if p is not None else None
        return a
    pa, va, ca = arr(pos), arr(vel), arr(col)
    _check(load().pr_scene_update_batch(hs, n, pa, va, ca, stream if stream is not None else current_stream()),
           "pr_scene_update_batch")


def pr_scene_free(scene):
    if scene:
        load().pr_scene_free(C.c_void_p(scene))


def pr_rasterize(scene, view, params=None, id_out=None, depth_out=None, stream=None):
    pv = view if isinstance(view, PrView) else make_view(view)
    pp = params if params is not None else make_params()
    _check(load().pr_rasterize(C.c_void_p(scene), C.byref(pv), C.byref(pp), _ptr(id_out), _ptr(depth_out),
                               stream if stream is not None else current_stream()), "pr_rasterize")


def pr_shade(scene, view, ids, rgb_out, stream=None):
    pv = view if isinstance(view, PrView) else make_view(view)
    _check(load().pr_shade(C.c_void_p(scene), C.byref(pv), _ptr(ids), _ptr(rgb_out),
                           stream if stream is not None else current_stream()), "pr_shade")


def pr_backward(scene, view, ids, grad_rgb, dcol=None, dpos=None, dvel=None, stream=None):
    pv = view if isinstance(view, PrView) else make_view(view)
    _check(load().pr_backward(C.c_void_p(scene), C.byref(pv), _ptr(ids), _ptr(grad_rgb), _ptr(dcol), _ptr(dpos),
                              _ptr(dvel), stream if stream is not None else current_stream()), "pr_backward")


def pr_backward_batch(ws, entries, stream=None):
    """entries: list of (scene, view, ids, grad_rgb, dcol, dpos, dvel), CUDA tensors."""
    arr = (PrBackwardView * len(entries))()
    for k, (scene, view, ids, g, dc, dp, dv) in enumerate(entries):
        arr[k].scene = C.c_void_p(scene)
        arr[k].view = view if isinstance(view, PrView) else make_view(view)
        for name, buf in (("id", ids), ("grad_rgb", g), ("dcol", dc), ("dpos", dp), ("dvel", dv)):
            p = _ptr(buf)
            setattr(arr[k], name, p.value if p is not None else None)
    _check(load().pr_backward_batch(C.c_void_p(ws), arr, len(entries),
                                    stream if stream is not None else current_stream()), "pr_backward_batch")


def pr_workspace_create() -> int:
    h = C.c_void_p()
    _check(load().pr_workspace_create(C.byref(h)), "pr_workspace_create")
    return h.value


def pr_workspace_free(ws):
    if ws:
        load().pr_workspace_free(C.c_void_p(ws))


def make_batch(entries):
    """entries: list of (scene, view, id_out, depth_out, rgb_out[, tile])."""
    arr = (PrBatchView * len(entries))()
    keep = []
    for k, e in enumerate(entries):
        scene, view, ido, dpo, rgb = e[:5]
        tile = e[5] if len(e) > 5 else 0
        arr[k].scene = C.c_void_p(scene)
        arr[k].view = view if isinstance(view, PrView) else make_view(view)
        for name, buf in (("id_out", ido), ("depth_out", dpo), ("rgb_out", rgb)):
            p = _ptr(buf)
            setattr(arr[k], name, p.value if p is not None else None)
            keep.append(buf)
        arr[k].tile = int(tile)
    return arr, keep


def pr_rasterize_batch(ws, entries, params=None, stream=None):
    arr, _keep = make_batch(entries)
    pp = params if params is not None else make_params()
    _check(load().pr_rasterize_batch(C.c_void_p(ws), arr, len(entries), C.byref(pp),
                                     stream if stream is not None else current_stream()), "pr_rasterize_batch")


def pr_graph_capture_batch(ws, entries, params=None, stream=None) -> int:
    arr, _keep = make_batch(entries)
    pp = params if params is not None else make_params()
    h = C.c_void_p()
    _check(load().pr_graph_capture_batch(C.c_void_p(ws), arr, len(entries), C.byref(pp),
                                         stream if stream is not None else current_stream(), C.byref(h)),
           "pr_graph_capture_batch")
    return h.value


def make_grads(grads):
    """grads: list (one per view) of None or a dict with any of grad_rgb,
    target_rgb, target_u8, dcol, dpos, dvel, loss (CUDA tensors)."""
    arr = (PrFrameGrad * len(grads))()
    keep = []
    for k, g in enumerate(grads):
        for name, buf in (g or {}).items():
            p = _ptr(buf)
            setattr(arr[k], name, p.value if p is not None else None)
            keep.append(buf)
    return arr, keep


def pr_frame_batch(ws, entries, grads, params=None, stream=None):
    """A training frame: the batched forward, then the adjoint of every view
    whose grads entry is given (see make_grads)."""
    arr, _keep = make_batch(entries)
    garr, _gkeep = make_grads(grads)
    pp = params if params is not None else make_params()
    _check(load().pr_frame_batch(C.c_void_p(ws), arr, len(entries), C.byref(pp), garr,
                                 stream if stream is not None else current_stream()), "pr_frame_batch")


def pr_graph_capture_frame(ws, entries, grads, params=None, stream=None) -> int:
    arr, _keep = make_batch(entries)
    garr, _gkeep = make_grads(grads)
    pp = params if params is not None else make_params()
    h = C.c_void_p()
    _check(load().pr_graph_capture_frame(C.c_void_p(ws), arr, len(entries), C.byref(pp), garr,
                                         stream if stream is not None else current_stream(), C.byref(h)),
           "pr_graph_capture_frame")
    return h.value


def pr_foveation_create(samples) -> int:
    """Handle of a sampled foveation function p (float32 [n + 1], p at
    d_k = k sqrt(2) / n, p[0] = 0, strictly increasing)."""
    arr = np.ascontiguousarray(np.asarray(samples, dtype=np.float32))
    h = C.c_void_p()
    _check(load().pr_foveation_create(arr.ctypes.data_as(C.c_void_p), int(arr.size - 1), C.byref(h)),
           "pr_foveation_create")
    return h.value


def pr_foveation_free(handle):
    if handle:
        load().pr_foveation_free(C.c_void_p(handle))


_foveations = {}


def foveation_handle(samples) -> int:
    """The (cached, process-lifetime) handle of a sample table, so that views
    may carry their p as samples."""
    arr = np.ascontiguousarray(np.asarray(samples, dtype=np.float32))
    key = arr.tobytes()
    with _lock:
        h = _foveations.get(key)
    if h is None:
        h = pr_foveation_create(arr)
        with _lock:
            _foveations[key] = h
    return h


def pr_unfoveate(ws, view, rgb, out, Wd: int, Hd: int, method: str = "mip", sigma: float = 0.5, stream=None):
    """Display image out [3][Hd][Wd] from the framebuffer image rgb
    [3][H][W] of `view` (CUDA tensors): method "mip" or "projected"."""
    pp = PrUnfoveateParams(UNFOVEATE_METHODS[method] if isinstance(method, str) else int(method), int(Wd), int(Hd),
                           float(sigma))
    v = view if isinstance(view, PrView) else make_view(view)
    _check(load().pr_unfoveate(C.c_void_p(ws), C.byref(v), _ptr(rgb), _ptr(out), C.byref(pp),
                               stream if stream is not None else current_stream()), "pr_unfoveate")


def pr_unfoveate_batch(ws, entries, method: str = "mip", sigma: float = 0.5, stream=None):
    """The display step of many views in one sequence: entries are
    (view, rgb, out, Wd, Hd) with CUDA tensors rgb [3][H][W] and out
    [3][Hd][Wd]; out of each equals pr_unfoveate's."""
    views = [v if isinstance(v, PrView) else make_view(v) for v, *_ in entries]
    arr = (PrUnfoveateEntry * max(1, len(entries)))()
    for k, ((_, rgb, out, Wd, Hd), v) in enumerate(zip(entries, views)):
        arr[k] = PrUnfoveateEntry(C.cast(C.pointer(v), C.c_void_p), _ptr(rgb), _ptr(out), int(Wd), int(Hd))
    pp = PrUnfoveateParams(UNFOVEATE_METHODS[method] if isinstance(method, str) else int(method), 0, 0, float(sigma))
    _check(load().pr_unfoveate_batch(C.c_void_p(ws), arr, len(entries), C.byref(pp),
                                     stream if stream is not None else current_stream()), "pr_unfoveate_batch")


def pr_graph_launch(graph, stream=None):
    _check(load().pr_graph_launch(C.c_void_p(graph), stream if stream is not None else current_stream()),
           "pr_graph_launch")


def pr_graph_enqueue(graph, stream=None):
    """Launch one replay without waiting; read its status with pr_graph_status
    once the stream has passed it."""
    _check(load().pr_graph_enqueue(C.c_void_p(graph), stream if stream is not None else current_stream()),
           "pr_graph_enqueue")


def pr_graph_status(graph):
    _check(load().pr_graph_status(C.c_void_p(graph)), "pr_graph_status")


def pr_debug_scan_timeout(stream=None) -> int:
    """Status of the scan's bounded-wait probe (PR_ERR_TIMEOUT expected)."""
    return int(load().pr_debug_scan_timeout(stream if stream is not None else current_stream()))


def pr_measure_fp32_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    out = C.c_double(0.0)
    _check(load().pr_measure_fp32_peak(stream if stream is not None else current_stream(), C.byref(out)),
           "pr_measure_fp32_peak")
    return out.value


def pr_graph_free(graph):
    if graph:
        load().pr_graph_free(C.c_void_p(graph))


def pr_scene_stats(scene) -> dict:
    s = PrStats()
    _check(load().pr_scene_stats(C.c_void_p(scene), C.byref(s)), "pr_scene_stats")
    return s.as_dict()


def pr_workspace_stats(ws) -> dict:
    s = PrStats()
    _check(load().pr_workspace_stats(C.c_void_p(ws), C.byref(s)), "pr_workspace_stats")
    return s.as_dict()


def pr_debug_bounds(scene, T: int):
    box = np.empty((T, 4), np.int32)
    tr = np.empty((T, 2), np.float32)
    _check(load().pr_debug_bounds(C.c_void_p(scene), _ptr(box), _ptr(tr)), "pr_debug_bounds")
    return box, tr


def pr_debug_halfplanes(scene, T: int):
    """Stage (a) half-planes of the last pr_rasterize on the scene: hp
    [T][8][4] (nx, ny, c, -) and info [T] (count | 0x100 when they are
    framebuffer lines)."""
    hp = np.empty((T, 8, 4), np.float32)
    info = np.empty(T, np.int32)
    _check(load().pr_debug_halfplanes(C.c_void_p(scene), _ptr(hp), _ptr(info)), "pr_debug_halfplanes")
    return hp, info


def pr_debug_catch_interval(view, S, E):
    pv = view if isinstance(view, PrView) else make_view(view)
    S = np.ascontiguousarray(S, dtype=np.float32).reshape(9)
    E = np.ascontiguousarray(E, dtype=np.float32).reshape(9)
    out = np.empty(2, np.float32)
    ok = load().pr_debug_catch_interval(C.byref(pv), _ptr(S), _ptr(E), _ptr(out))
    return bool(ok == 1), out


def pr_rasterize_noalloc(pos, vel, col, tri, view, params=None, id_out=None, depth_out=None, stream=None):
    """Stages (a)-(c) with the library's fixed device scratch array (no
    allocation); every buffer must be a CUDA tensor."""
    pv = view if isinstance(view, PrView) else make_view(view)
    pp = params if params is not None else make_params()
    _check(load().pr_rasterize_noalloc(_ptr(pos), _ptr(vel), _ptr(col), _ptr(tri), int(pos.shape[0]),
                                       int(tri.shape[0]), C.byref(pv), C.byref(pp), _ptr(id_out), _ptr(depth_out),
                                       stream if stream is not None else current_stream()), "pr_rasterize_noalloc")


def pr_status_string(s: int) -> str:
    return status_string(s)


def pr_version() -> int:
    return int(load().pr_version())
