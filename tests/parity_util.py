"""GPU-vs-oracle comparison with the excusal rule for edge and depth ties.

A pixel whose triangle id differs between the CUDA path and the FP64 oracle
is excused only if the disagreement sits where the two arithmetics may
legitimately differ:
  * the pixel lies within ``tol_edge`` of an edge of the oracle's or the
    GPU's winner, or
  * both winners hit and their FP64 depths differ by less than
    ``tol_depth`` (relative).
Edge distance is measured in the unit the mode's arithmetic controls:
  * FP32 path: distance in unit display coordinates from the pixel's display
    location to the triangle projected at the pixel time.  FP32 carries a
    relative error of about 6e-8 per operation; the camera-space transform,
    the interpolation to the pixel time, the shear and the foveation power
    each add a few ulps of the coordinate magnitudes, so decisions within
    ~1e-6 of an edge (in display units, independent of the triangle's size)
    are not determined by FP32.  TOL_FP32 = 1e-5 leaves a factor 10 margin.
  * FP64 re-test: barycentric distance, 1e-6, the tolerance the method
    states for its FP64-checked result.
Depth ties use the same two values relative to the depth.
"""
import numpy as np

BG = 0xFFFFFFFF
TOL_FP32 = 1e-5
TOL_FP64 = 1e-6


def excused(oracle, view, sc, lin, oid, gid, o_bmin, fp64=False):
    tol = TOL_FP64 if fp64 else TOL_FP32
    ev_o = oracle.evaluate(view, sc.pos, sc.vel, sc.tri, int(lin), int(oid)) if oid != BG else None
    ev_g = oracle.evaluate(view, sc.pos, sc.vel, sc.tri, int(lin), int(gid)) if gid != BG else None

    def near_edge(ev):
        if ev is None:
            return False
        if fp64:
            return abs(min(ev[0], ev[1], ev[2])) < tol
        return ev[5] < tol

    if near_edge(ev_o) or near_edge(ev_g):
        return True
    if ev_o is not None and ev_g is not None and np.isfinite(ev_g[3]) and ev_g[3] > view.z_near:
        if abs(ev_g[3] - ev_o[3]) / ev_o[3] < tol:
            return True
    return False


def compare(oracle, view, sc, o, gpu_id, gpu_depth=None, gpu_rgb=None, pix=None, fp64=False,
            min_agree=0.9999, depth_rtol=1e-5, rgb_atol=1e-4):
    """o: oracle render of the pixels ``pix`` (all when None).  gpu_*: full
    [H*W] (rgb: [3, H*W]) numpy arrays.  Asserts the criteria and returns a
    small report."""
    n = view.W * view.H
    pix = np.arange(n) if pix is None else np.asarray(pix)
    gid = gpu_id.reshape(-1)[pix].astype(np.uint32)
    oid = o["id"].astype(np.uint32)
    mism = np.nonzero(gid != oid)[0]
    bad = []
    for m in mism:
        if not excused(oracle, view, sc, pix[m], oid[m], gid[m], o["bmin"][m], fp64):
            bad.append((int(pix[m]), int(oid[m]), int(gid[m])))
    agree = 1.0 - mism.size / max(1, pix.size)
    rep = {"pixels": int(pix.size), "mismatch": int(mism.size), "unexcused": bad[:10], "n_unexcused": len(bad),
           "agree": agree, "hit_frac": float((oid != BG).mean())}
    same = (gid == oid) & (oid != BG)
    if gpu_depth is not None:
        gd = gpu_depth.reshape(-1)[pix]
        bgd = gd[(oid == BG) & (gid == BG)]
        assert np.all(np.isinf(bgd)), "background depth must be +inf"
        rel = np.abs(gd[same].astype(np.float64) - o["s"][same]) / o["s"][same] if same.any() else np.zeros(1)
        # a ray that grazes its triangle has an ill-conditioned depth: the
        # FP32 error grows like 1/|cos| of the angle to the normal, so the
        # allowance is max(depth_rtol, 16 u / |cos|) with u = 2^-24
        cosg = o["cos"][same] if ("cos" in o and same.any()) else np.ones(1)
        allow = np.maximum(depth_rtol, 16.0 * 2.0 ** -24 / np.maximum(cosg, 1e-12))
        rep["depth_rel_max"] = float(rel.max()) if rel.size else 0.0
        rep["depth_over_allowance"] = float((rel / allow).max()) if rel.size else 0.0
    if gpu_rgb is not None:
        g = gpu_rgb.reshape(3, -1)[:, pix].T
        err = np.abs(g[same].astype(np.float64) - o["rgb"][same]) if same.any() else np.zeros((1, 3))
        rep["rgb_abs_max"] = float(err.max()) if err.size else 0.0
        bgr = g[(oid == BG) & (gid == BG)]
        assert np.all(bgr == 0), "background rgb must be 0"
    assert not bad, f"unexcused id mismatches: {rep}"
    assert agree >= min_agree, rep
    if gpu_depth is not None:
        assert rep["depth_over_allowance"] <= 1.0, rep
    if gpu_rgb is not None:
        assert rep["rgb_abs_max"] <= rgb_atol, rep
    return rep
