"""Display step (Sec. 3.1.1, "Display") on the GPU against the FP64 oracle,
on the same framebuffer image: every display pixel whose preimage q^-1(x)
lies in the framebuffer within 2e-5 (rgb in [0, 1], FP32 filter sums of at
most 25 terms); display pixels beyond the framebuffer's coverage (their
samples are tens of display pixels away, and the FP32 rounding of q scales
with that distance) within 1e-3; except, for both, where the oracle's
discrete choice (nearest texel of a level, or the pixel holding q^-1(x))
lies within 1e-3 texels of its decision boundary, where FP32 rounding may
tip it (at most 5 % of the pixels: when the display and framebuffer grids
are commensurate whole rows fall on texel midpoints)."""
import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S
from tests.test_parity_gpu import gpu_frame, small_case

pytestmark = pytest.mark.gpu

TOL = 2e-5


def _unfoveate_gpu(pr, view, img, Wd, Hd, method, sigma=0.5):
    import torch
    ws = pr.pr_workspace_create()
    try:
        rgb = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32).reshape(-1)).cuda()
        out = torch.empty(3 * Wd * Hd, device="cuda")
        pr.pr_unfoveate(ws, view, rgb, out, Wd, Hd, method, sigma)
        torch.cuda.synchronize()
        return out.cpu().numpy().reshape(3, Hd, Wd)
    finally:
        pr.pr_workspace_free(ws)


def _covered(view, Wd, Hd):
    """Display pixels whose preimage lies in the framebuffer (closed form of
    q^-1 for the power map; the identity when not foveated)."""
    a, b = np.meshgrid((np.arange(Wd) + 0.5) / Wd, (np.arange(Hd) + 0.5) / Hd)
    u0, u1 = a, b
    if view.mode in (S.MODE_FOVEATED, S.MODE_BOTH):
        e0, e1 = a - view.fovea[0], b - view.fovea[1]
        r = np.hypot(e0, e1)
        s = np.where(r > 0, (np.maximum(r, 1e-300) / np.sqrt(2.0)) ** (1.0 / view.alpha - 1.0), 0.0)
        u0, u1 = view.fovea[0] + e0 * s, view.fovea[1] + e1 * s
    return ((u0 >= 0) & (u0 <= 1) & (u1 >= 0) & (u1 <= 1)).reshape(-1)


def _check(oracle, pr, view, img, Wd, Hd, method, sigma=0.5):
    g = _unfoveate_gpu(pr, view, img, Wd, Hd, method, sigma)
    o, margin = oracle.unfoveate(view, img, Wd, Hd, method, sigma)
    err = np.abs(g - o).max(axis=0).reshape(-1)
    bad = err > np.where(_covered(view, Wd, Hd), TOL, 1e-3)
    excused = margin < 1e-3
    assert not np.any(bad & ~excused), (method, Wd, Hd, err[bad & ~excused][:5], np.flatnonzero(bad & ~excused)[:5])
    assert excused.mean() < 0.05  # regular grids put whole rows on texel midpoints
    return g


@pytest.mark.parametrize("method", ["mip", "projected"])
@pytest.mark.parametrize("mode", [S.MODE_FOVEATED, S.MODE_BOTH, S.MODE_ROLLING])
@pytest.mark.parametrize("size", [(1.0, 1.0), (1.5, 1.25), (0.5, 0.75)])
def test_unfoveate_random_image_matches_oracle(pr, oracle, method, mode, size):
    W, H = 131, 97  # ragged, pyramid levels of odd sizes
    rng = np.random.default_rng(int(10 * size[0]) + mode)
    img = rng.uniform(size=(3, H, W)).astype(np.float32)
    _, view = small_case(mode, W=W, H=H)
    Wd, Hd = int(W * size[0]), int(H * size[1])
    _check(oracle, pr, view, img, Wd, Hd, method, sigma=0.7)


@pytest.mark.parametrize("method", ["mip", "projected"])
def test_unfoveate_rendered_frame(pr, oracle, method):
    """The shaded foveated frame of the renderer, displayed at 1.5x its size."""
    sc, view = small_case(S.MODE_BOTH, seed=6, W=160, H=128, T=800)
    g = gpu_frame(pr, sc, view)
    img = g["rgb"].reshape(3, view.H, view.W)
    out = _check(oracle, pr, view, img, 240, 192, method)
    assert np.isfinite(out).all() and out.max() > 0.0


def test_unfoveate_degenerate_sizes_and_errors(pr, oracle):
    import torch
    _, view = small_case(S.MODE_FOVEATED, W=1, H=1)
    img = np.full((3, 1, 1), 0.3, np.float32)
    for m in ("mip", "projected"):
        out = _unfoveate_gpu(pr, view, img, 3, 2, m)
        assert np.allclose(out, 0.3, atol=1e-7)
    ws = pr.pr_workspace_create()
    try:
        rgb = torch.zeros(3, device="cuda")
        out = torch.zeros(3 * 4, device="cuda")
        with pytest.raises(pr.PrError):
            pr.pr_unfoveate(ws, view, rgb, out, 2, 2, "projected", 0.0)   # sigma must be > 0
        with pytest.raises(pr.PrError):
            pr.pr_unfoveate(ws, view, torch.zeros(3), out, 2, 2, "mip")  # host input
    finally:
        pr.pr_workspace_free(ws)
