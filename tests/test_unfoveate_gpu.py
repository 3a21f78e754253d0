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


def _batch_specs():
    """Views of mixed size, mode and foveation for the batched display step:
    ragged sizes, a 1x1 framebuffer, a sampled p, enlarged, shrunk and
    anisotropic displays."""
    import dataclasses
    from paper_1806_05385_gb300 import foveation as F
    lens = F.lens_samples(2.0, 0.22, 0.24, 1024)
    out = []
    for (W, H, mode, lut, Wd, Hd) in [(131, 97, S.MODE_FOVEATED, None, 196, 145),
                                      (64, 200, S.MODE_BOTH, None, 50, 300),
                                      (257, 129, S.MODE_ROLLING, None, 257, 129),
                                      (1, 1, S.MODE_CLASSIC, None, 3, 2),
                                      (160, 128, S.MODE_BOTH, lens, 200, 160),
                                      (33, 17, S.MODE_FOVEATED, None, 17, 9)]:
        _, view = small_case(mode, W=W, H=H)
        if lut is not None:
            view = dataclasses.replace(view, p_lut=lut)
        out.append((view, Wd, Hd))
    return out


def _batch_gpu(pr, specs, imgs, method, sigma, ws=None):
    import torch
    own = ws is None
    ws = pr.pr_workspace_create() if own else ws
    try:
        rgbs = [torch.from_numpy(np.ascontiguousarray(im, dtype=np.float32).reshape(-1)).cuda() for im in imgs]
        outs = [torch.full((3 * Wd * Hd,), -7.0, device="cuda") for _, Wd, Hd in specs]
        pr.pr_unfoveate_batch(ws, [(v, r, o, Wd, Hd) for (v, Wd, Hd), r, o in zip(specs, rgbs, outs)], method, sigma)
        torch.cuda.synchronize()
        return [o.cpu().numpy().reshape(3, Hd, Wd) for o, (_, Wd, Hd) in zip(outs, specs)]
    finally:
        if own:
            pr.pr_workspace_free(ws)


@pytest.mark.parametrize("method", ["mip", "projected"])
def test_unfoveate_batch_equals_per_view(pr, method):
    """The batched display step gives every view the same bits as its own
    pr_unfoveate call, and a second batch on the same workspace (reusing its
    pinned table) too."""
    specs = _batch_specs()
    rng = np.random.default_rng(17)
    imgs = [rng.uniform(size=(3, v.H, v.W)).astype(np.float32) for v, _, _ in specs]
    ws = pr.pr_workspace_create()
    try:
        for rnd in range(2):
            order = list(range(len(specs)))[::(-1 if rnd else 1)]
            got = _batch_gpu(pr, [specs[k] for k in order], [imgs[k] for k in order], method, 0.7, ws)
            for k, g in zip(order, got):
                v, Wd, Hd = specs[k]
                ref = _unfoveate_gpu(pr, v, imgs[k], Wd, Hd, method, sigma=0.7)
                assert np.array_equal(g.view(np.uint32), ref.view(np.uint32)), (method, k)
    finally:
        pr.pr_workspace_free(ws)


@pytest.mark.parametrize("method", ["mip", "projected"])
def test_unfoveate_batch_matches_oracle(pr, oracle, method):
    """The batch's outputs against the FP64 oracle, with the tolerances and
    excusals of the single-view test."""
    specs = [s for s in _batch_specs() if s[0].W > 1]
    rng = np.random.default_rng(23)
    imgs = [rng.uniform(size=(3, v.H, v.W)).astype(np.float32) for v, _, _ in specs]
    got = _batch_gpu(pr, specs, imgs, method, 0.7)
    for (v, Wd, Hd), img, g in zip(specs, imgs, got):
        o, margin = oracle.unfoveate(v, img, Wd, Hd, method, 0.7)
        err = np.abs(g - o).max(axis=0).reshape(-1)
        bad = err > np.where(_covered(v, Wd, Hd), TOL, 1e-3)
        assert not np.any(bad & ~(margin < 1e-3)), (method, v.W, v.H, Wd, Hd)


def test_unfoveate_batch_refuses_before_launching(pr):
    """An empty batch does nothing; a batch with one bad entry (host image,
    zero display size) is refused whole and writes no output."""
    import torch
    specs = _batch_specs()[:2]
    imgs = [np.zeros((3, v.H, v.W), np.float32) for v, _, _ in specs]
    ws = pr.pr_workspace_create()
    try:
        pr.pr_unfoveate_batch(ws, [], "mip")
        rgbs = [torch.from_numpy(im.reshape(-1)).cuda() for im in imgs]
        outs = [torch.full((3 * Wd * Hd,), -7.0, device="cuda") for _, Wd, Hd in specs]
        good = [(v, r, o, Wd, Hd) for (v, Wd, Hd), r, o in zip(specs, rgbs, outs)]
        bad_host = good[:1] + [(specs[1][0], imgs[1].reshape(-1), outs[1], specs[1][1], specs[1][2])]
        bad_size = good[:1] + [(specs[1][0], rgbs[1], outs[1], 0, specs[1][2])]
        for entries in (bad_host, bad_size):
            with pytest.raises(pr.PrError) as ei:
                pr.pr_unfoveate_batch(ws, entries, "mip")
            assert ei.value.status == pr.PR_ERR_INVALID_ARG
        with pytest.raises(pr.PrError):
            pr.pr_unfoveate_batch(ws, good, "projected", sigma=0.0)
        torch.cuda.synchronize()
        assert all(bool((o == -7.0).all()) for o in outs)
        pr.pr_unfoveate_batch(ws, good, "mip")
        torch.cuda.synchronize()
        assert all(bool((o == 0.0).all()) for o in outs)
    finally:
        pr.pr_workspace_free(ws)
