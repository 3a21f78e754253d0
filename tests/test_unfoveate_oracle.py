"""Pins of the display-unfoveation oracle (Sec. 3.1.1, "Display") against
closed forms and library filters; no GPU.

* a constant image stays constant (both methods, normalised weights);
* identity map at full size: the MIP path at level 0 is the separable
  [1/6, 2/3, 1/6] B-spline blur at texel centres (scipy), the projected
  path with a narrow filter is the image itself, with sigma = 1 it is the
  normalised 5 x 5 Gaussian blur (scipy);
* identity map at half size: level 1 = 2 x 2 block means (numpy), blurred;
* the level of detail matches log2 of the largest singular value of a
  finite-difference Jacobian of q^-1, times the size ratio;
* foveated: with a narrow filter the display pixel takes the framebuffer
  pixel whose q-image is nearest, so a coordinate ramp returns q^-1(x) to
  within half a framebuffer pixel.
"""
import math

import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _view(W, H, mode, fovea=(0.42, 0.57), alpha=2.0):
    p0, p1 = S.head_poses(1.0, 0.0)
    return S.View(W=W, H=H, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode, fovea=fovea, alpha=alpha)


def _img(W, H, seed=0):
    return np.random.default_rng(seed).uniform(size=(3, H, W)).astype(np.float32)


def _bspline_blur(img):
    k = np.array([1.0, 4.0, 1.0]) / 6.0
    out = scipy_ndimage.convolve1d(img.astype(np.float64), k, axis=-1, mode="nearest")
    return scipy_ndimage.convolve1d(out, k, axis=-2, mode="nearest")


@pytest.mark.parametrize("method", ["mip", "projected"])
def test_constant_image_stays_constant(oracle, method):
    v = _view(64, 48, S.MODE_BOTH)
    img = np.full((3, 48, 64), 0.375, np.float32)
    out, _ = oracle.unfoveate(v, img, 90, 70, method, 0.7)
    assert np.allclose(out, 0.375, atol=1e-14)


def test_identity_full_size_mip_is_bspline_blur(oracle):
    v = _view(40, 30, S.MODE_ROLLING)
    img = _img(40, 30)
    out, margin = oracle.unfoveate(v, img, 40, 30, "mip")
    assert np.allclose(out, _bspline_blur(img), atol=1e-12)
    assert np.allclose(margin, 0.5)          # texel centres: farthest from a flip


def test_identity_half_size_uses_level_one(oracle):
    v = _view(40, 32, S.MODE_CLASSIC)
    img = _img(40, 32, 1)
    out, _ = oracle.unfoveate(v, img, 20, 16, "mip")
    lvl1 = img.astype(np.float64).reshape(3, 16, 2, 20, 2).mean(axis=(2, 4))
    assert np.allclose(out, _bspline_blur(lvl1), atol=1e-12)


def test_mip_levels_halve_with_ceil():
    from oracle import oracle as O
    assert O.mip_levels(96, 80) == [(96, 80), (48, 40), (24, 20), (12, 10), (6, 5), (3, 3), (2, 2), (1, 1)]
    assert O.mip_levels(1, 1) == [(1, 1)]


def test_identity_projected_narrow_is_the_image(oracle):
    v = _view(36, 28, S.MODE_CLASSIC)
    img = _img(36, 28, 2)
    out, _ = oracle.unfoveate(v, img, 36, 28, "projected", 0.05)
    assert np.allclose(out, img, atol=1e-12)


def test_identity_projected_is_normalised_gaussian_blur(oracle):
    v = _view(36, 28, S.MODE_CLASSIC)
    img = _img(36, 28, 3).astype(np.float64)
    out, _ = oracle.unfoveate(v, img.astype(np.float32), 36, 28, "projected", 1.0)
    g = np.exp(-np.arange(-2, 3) ** 2 / 2.0)
    k = np.outer(g, g)
    ones = np.ones(img.shape[1:])
    norm = scipy_ndimage.convolve(ones, k, mode="constant", cval=0.0)
    ref = np.stack([scipy_ndimage.convolve(img[c], k, mode="constant", cval=0.0) for c in range(3)]) / norm
    assert np.allclose(out, ref.astype(np.float32).astype(np.float64), atol=2e-7)


def test_level_of_detail_is_largest_stretch(oracle):
    W, H, Wd, Hd = 200, 160, 300, 240
    v = _view(W, H, S.MODE_FOVEATED, alpha=2.0)
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.uniform(0.05, 0.95, size=2)
        h = 1e-6
        J = np.empty((2, 2))
        for a in range(2):
            dx = np.zeros(2)
            dx[a] = h
            J[:, a] = (oracle.qinv(v, x + dx) - oracle.qinv(v, x - dx)) / (2 * h)
        smax = np.linalg.svd(J, compute_uv=False)[0]
        want = math.log2(smax * max(W / Wd, H / Hd))
        assert oracle.unfoveate_lod(v, x, Wd, Hd) == pytest.approx(want, abs=1e-6)


def test_foveated_narrow_filter_returns_preimage(oracle):
    W, H, Wd, Hd = 80, 64, 80, 64
    v = _view(W, H, S.MODE_FOVEATED, fovea=(0.5, 0.5), alpha=2.0)
    ii, jj = np.meshgrid(np.arange(W), np.arange(H))
    img = np.stack([(ii + 0.5) / W, (jj + 0.5) / H, np.zeros_like(ii, float)]).astype(np.float32)
    out, _ = oracle.unfoveate(v, img, Wd, Hd, "projected", 0.01)
    rng = np.random.default_rng(5)
    checked = 0
    while checked < 50:
        a, b = rng.integers(0, Wd), rng.integers(0, Hd)
        u = oracle.qinv(v, np.array([(a + 0.5) / Wd, (b + 0.5) / Hd]))
        # the framebuffer maps onto a disc around the fovea (p <= identity);
        # display pixels beyond it have preimages outside [0,1]^2
        if not (3 / W < u[0] < 1 - 3 / W and 3 / H < u[1] < 1 - 3 / H):
            continue
        checked += 1
        # the chosen pixel lies in the 5 x 5 window around u; its q-image is
        # the nearest: its centre is within 2.5 framebuffer pixels of u
        assert abs(out[0, b, a] - u[0]) <= 2.5 / W and abs(out[1, b, a] - u[1]) <= 2.5 / H
