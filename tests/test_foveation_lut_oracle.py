"""Pins of the oracle's sampled foveation function (Sec. 3.1.1: any monotonic
p, inverted numerically; Sec. 6: lens distortion p = p_c o p_l); no GPU.

* p given by samples of the power map agrees with the analytic power map
  within the linear-interpolation bound h^2/8 max|p''| (here q and q^-1);
* q^-1 is the exact inverse of q for a sampled p (round trip to rounding);
* the identity samples p(d) = d make the foveated render equal the
  non-foveated one;
* the display step's level of detail for a sampled p matches a
  finite-difference Jacobian of q^-1.
"""
import math

import numpy as np
import pytest

from paper_1806_05385_gb300 import foveation as F
from paper_1806_05385_gb300 import scenes as S


def _view(mode=S.MODE_FOVEATED, p_lut=None, W=64, H=48, alpha=2.0):
    p0, p1 = S.head_poses(1.5, 0.3)
    return S.View(W=W, H=H, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode, fovea=(0.43, 0.56), alpha=alpha,
                  p_lut=p_lut)


def test_sampled_power_map_matches_analytic(oracle):
    n = 2048
    h = math.sqrt(2.0) / n
    va, vl = _view(), _view(p_lut=F.power_samples(2.0, n))
    # p(d) = D (d/D)^2 has p'' = 2/D: interpolation error <= h^2/8 * 2/D, plus FP32 rounding of the samples
    bound = h * h / 8 * 2 / math.sqrt(2.0) + 4e-7
    rng = np.random.default_rng(0)
    for _ in range(200):
        u = rng.uniform(0, 1, 2)
        assert np.abs(oracle.q(va, u) - oracle.q(vl, u)).max() <= bound
        x = oracle.q(va, u)
        # p^-1 has unbounded curvature at 0; compare away from the fovea
        if np.linalg.norm(x - np.array(va.fovea)) > 0.05:
            assert np.abs(oracle.qinv(va, x) - oracle.qinv(vl, x)).max() <= 1e-4


@pytest.mark.parametrize("samples", [F.lens_samples(2.0, 0.22, 0.24, 257), F.power_samples(3.0, 64)])
def test_sampled_inverse_is_exact(oracle, samples):
    v = _view(p_lut=samples)
    rng = np.random.default_rng(1)
    for _ in range(200):
        u = rng.uniform(0, 1, 2)
        assert np.abs(oracle.qinv(v, oracle.q(v, u)) - u).max() <= 1e-12


def test_identity_samples_render_as_not_foveated(oracle):
    n = 16
    ident = (np.arange(n + 1) * (math.sqrt(2.0) / n)).astype(np.float32)
    sc = S.random_triangles(300, 2)
    vf = _view(S.MODE_BOTH, ident)
    vr = _view(S.MODE_ROLLING)
    a = oracle.render(vf, sc.pos, sc.vel, sc.col, sc.tri)
    b = oracle.render(vr, sc.pos, sc.vel, sc.col, sc.tri)
    # the FP32 samples of the identity and the linear interpolation move x by
    # at most a few ulps: only pixels on an edge may change owner
    same = a["id"] == b["id"]
    assert same.mean() > 0.995
    assert np.allclose(a["depth"][same], b["depth"][same], rtol=1e-6)


def test_lod_of_sampled_p_is_largest_stretch(oracle):
    W, H, Wd, Hd = 200, 160, 300, 240
    v = _view(p_lut=F.lens_samples(2.0, 0.22, 0.24, 4096), W=W, H=H)
    rng = np.random.default_rng(4)
    checked = 0
    while checked < 20:
        x = rng.uniform(0.05, 0.95, size=2)
        if np.linalg.norm(x - np.array(v.fovea)) < 0.05:
            continue
        h = 1e-7
        J = np.empty((2, 2))
        for a in range(2):
            dx = np.zeros(2)
            dx[a] = h
            J[:, a] = (oracle.qinv(v, x + dx) - oracle.qinv(v, x - dx)) / (2 * h)
        smax = np.linalg.svd(J, compute_uv=False)[0]
        want = math.log2(smax * max(W / Wd, H / Hd))
        assert oracle.unfoveate_lod(v, x, Wd, Hd) == pytest.approx(want, abs=2e-3)
        checked += 1
