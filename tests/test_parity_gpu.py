"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Covers every mode (classic, rolling, foveated, both), every bound kind and
tile size, ragged frames, empty and degenerate inputs, near-plane crossings,
shading, host-memory buffers, and the conservativeness of the stage (a)
bounds (every pixel the oracle says a triangle wins lies inside that
triangle's bound)."""
import math

import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S
from tests.parity_util import BG, compare

pytestmark = pytest.mark.gpu

MODES = [S.MODE_CLASSIC, S.MODE_ROLLING, S.MODE_FOVEATED, S.MODE_BOTH]


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_frame(pr, sc, view, bound="zenon", tile=16, shade=True, fp64=0, seg=0, keep=False):
    import torch
    h = pr.pr_scene_upload(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri.reshape(-1, 3)))
    n = view.W * view.H
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    depth = torch.empty(n, dtype=torch.float32, device="cuda")
    pr.pr_rasterize(h, view, pr.make_params(bound, tile, fp64, seg), ids, depth)
    out = {"stats": pr.pr_scene_stats(h)}
    if shade:
        rgb = torch.empty(3 * n, dtype=torch.float32, device="cuda")
        pr.pr_shade(h, view, ids, rgb)
        out["rgb"] = rgb.cpu().numpy()
    torch.cuda.synchronize()
    out["id"] = ids.cpu().numpy().view(np.uint32)
    out["depth"] = depth.cpu().numpy()
    if keep:
        out["scene"] = h
    else:
        pr.pr_scene_free(h)
    return out


def small_case(mode, seed=0, W=256, H=256, T=1000):
    sc = S.random_triangles(T, seed)
    p0, p1 = S.head_poses(2.0, 0.0)
    return sc, S.View(W=W, H=H, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode, fovea=(0.43, 0.58))


@pytest.mark.parametrize("mode", MODES)
def test_small_frame_parity(pr, oracle, mode):
    sc, view = small_case(mode)
    g = gpu_frame(pr, sc, view)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    rep = compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"])
    assert rep["hit_frac"] > 0.05
    st = g["stats"]
    assert st["pixels"] == view.W * view.H and st["tests"] >= st["hits"] > 0


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("mode", [S.MODE_ROLLING, S.MODE_BOTH])
def test_tile_sizes_agree(pr, oracle, mode, tile):
    sc, view = small_case(mode, seed=1, W=200, H=136, T=600)   # ragged in both directions
    g = gpu_frame(pr, sc, view, tile=tile)
    ref = gpu_frame(pr, sc, view, tile=16)
    assert np.array_equal(g["id"], ref["id"]) and np.array_equal(g["depth"], ref["depth"])
    if tile == 8:
        o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
        compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"])


@pytest.mark.parametrize("seg", [1, 5, 32, 33, 100, 256, 257, 700, 1024, 5000])
def test_work_item_runs_give_identical_images(pr, seg):
    """Splitting a tile's bin into work items of any run length (and the
    depth sort of each run, in registers up to 256 entries and in shared
    memory beyond) changes only the order of the tests, never the result."""
    sc = S.random_triangles(4000, 21, offset=0.25)
    p0, p1 = S.head_poses(2.0, 0.5)
    view = S.View(W=120, H=88, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=S.MODE_BOTH, fovea=(0.45, 0.55))
    g = gpu_frame(pr, sc, view, tile=32, seg=seg, shade=False)
    ref = gpu_frame(pr, sc, view, tile=32, shade=False)
    assert ref["stats"]["pairs"] / 12 > 300   # 12 tiles: bins longer than 256 entries exist
    assert np.array_equal(g["id"], ref["id"]) and np.array_equal(g["depth"], ref["depth"])


@pytest.mark.parametrize("fov_bound", ["simple", "recursive"])
@pytest.mark.parametrize("mode", [S.MODE_FOVEATED, S.MODE_BOTH])
def test_paper_foveation_bounds_give_identical_images(pr, mode, fov_bound):
    """Sec. 4.1: the Simple and Recursive edge bounds change which tiles are
    tested, never the image; on this scene their ternary searches hold."""
    sc, view = small_case(mode, seed=4, W=224, H=176, T=900)
    ref = gpu_frame(pr, sc, view, shade=False)
    h = pr.pr_scene_upload(*(_dev(a) for a in (sc.pos, sc.vel, sc.col, sc.tri)))
    import torch
    n = view.W * view.H
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    dep = torch.empty(n, device="cuda")
    pr.pr_rasterize(h, view, pr.make_params("zenon", 16, 0, 0, fov_bound=fov_bound), ids, dep)
    st = pr.pr_scene_stats(h)
    pr.pr_scene_free(h)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["id"])
    assert np.array_equal(dep.cpu().numpy(), ref["depth"])
    assert st["tests"] > 0 and st["pairs"] > 0


@pytest.mark.parametrize("mode", MODES)
def test_bound_kinds_give_identical_images(pr, mode):
    """Sec. 3.2: the intersection test is the same whatever bound is used,
    so every bound kind must give bit-identical buffers; only the number of
    tests changes (Tables 1-2: STE rises from Trivial/Quad to Zenon)."""
    sc, view = small_case(mode, seed=2, W=160, H=120, T=800)
    ref = gpu_frame(pr, sc, view, bound="zenon")
    tests = {}
    for b in ("adaptive", "hull", "quad", "trivial"):
        g = gpu_frame(pr, sc, view, bound=b)
        assert np.array_equal(g["id"], ref["id"]), b
        assert np.array_equal(g["depth"], ref["depth"]), b
        tests[b] = g["stats"]["tests"]
    tests["zenon"] = ref["stats"]["tests"]
    assert tests["zenon"] <= tests["trivial"]
    if mode in (S.MODE_ROLLING, S.MODE_BOTH):
        assert tests["zenon"] <= tests["hull"] <= tests["quad"] * 1.0001 + 1


def _check_conservative(pr, oracle, sc, view, bound="zenon", fov_bound="sector"):
    """Every pixel the oracle assigns to a triangle lies in that triangle's
    stage (a) framebuffer box, its time in the triangle's interval, and its
    location inside every half-plane the binning tests: display half-planes
    at the pixel's display location x (Sec. 4.2), or, for the paper's
    foveation bounds, framebuffer lines at its unit framebuffer location u
    (Sec. 4.1).  Returns the number of (pixel, half-plane) checks made."""
    import torch
    h = pr.pr_scene_upload(*(_dev(a) for a in (sc.pos, sc.vel, sc.col, sc.tri)))
    try:
        n = view.W * view.H
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        pr.pr_rasterize(h, view, pr.make_params(bound, 16, 0, 0, fov_bound=fov_bound), ids, None)
        box, tr = pr.pr_debug_bounds(h, sc.T)
        hp, info = pr.pr_debug_halfplanes(h, sc.T)
    finally:
        pr.pr_scene_free(h)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    t, x, _ = oracle.pixels(view)
    hit = np.nonzero(o["id"] != BG)[0]
    ids = o["id"][hit].astype(np.int64)
    i, j = hit % view.W, hit // view.W
    b = box[ids]
    inside = (i >= b[:, 0]) & (i <= b[:, 2]) & (j >= b[:, 1]) & (j <= b[:, 3])
    assert inside.all(), hit[~inside][:10]
    tt = t[hit]
    assert np.all((tt >= tr[ids, 0]) & (tt <= tr[ids, 1]))
    u = np.stack([(i + 0.5) / view.W, (j + 0.5) / view.H], 1)
    fb = (info[ids] & 0x100) != 0
    pt = np.where(fb[:, None], u, x[hit])
    nh = info[ids] & 0xFF
    checks = 0
    for k in range(8):
        use = nh > k
        hk = hp[ids[use], k].astype(np.float64)
        val = hk[:, 0] * pt[use, 0] + hk[:, 1] * pt[use, 1] + hk[:, 2]
        assert np.all(val <= 0.0), (k, hit[use][val > 0][:5], val[val > 0][:5])
        checks += int(use.sum())
    return checks, int(fb.sum())


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("bound", ["zenon", "adaptive", "hull"])
def test_bounds_are_conservative(pr, oracle, mode, bound):
    """Sec. 3.2: the bound covers every pixel the triangle affects at any
    time -- box, interval and display half-planes."""
    sc, view = small_case(mode, seed=3, W=192, H=160, T=700)
    _check_conservative(pr, oracle, sc, view, bound)


@pytest.mark.parametrize("alpha", [2.0, 3.0])
@pytest.mark.parametrize("fov_bound", ["simple", "recursive"])
@pytest.mark.parametrize("mode", [S.MODE_FOVEATED, S.MODE_BOTH])
@pytest.mark.parametrize("seed", [3, 12, 31])
def test_paper_foveation_bounds_are_conservative(pr, oracle, mode, fov_bound, alpha, seed):
    """Sec. 4.1.1-4.1.2: the Simple and Recursive edge bounds, whose lines
    bin the tiles in framebuffer space, hold every pixel the oracle assigns
    to the triangle (their ternary searches rest on a unimodal edge
    displacement; the coarse seed scan and the half-pixel margin must cover
    these scenes)."""
    sc = S.random_triangles(700, seed, offset=0.6 if seed % 2 else None)
    p0, p1 = S.head_poses(2.0, 0.5)
    view = S.View(W=192, H=160, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode,
                  fovea=(0.3 + 0.01 * seed, 0.62 - 0.01 * seed), alpha=alpha)
    checks, nfb = _check_conservative(pr, oracle, sc, view, "zenon", fov_bound)
    assert nfb > 0 and checks > 0


def test_ragged_tiny_frames(pr, oracle):
    for W, H in ((1, 1), (7, 3), (17, 33), (33, 17)):
        sc, view = small_case(S.MODE_BOTH, seed=W, W=W, H=H, T=300)
        g = gpu_frame(pr, sc, view, tile=8)
        o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
        compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"])


def test_empty_scene_is_background(pr):
    sc = S.Scene(np.zeros((3, 3), np.float32), np.zeros((3, 3), np.float32), np.zeros((3, 3), np.float32),
                 np.zeros((0, 3), np.int32))
    _, view = small_case(S.MODE_ROLLING, W=40, H=30)
    g = gpu_frame(pr, sc, view)
    assert np.all(g["id"] == BG) and np.all(np.isinf(g["depth"])) and np.all(g["rgb"] == 0)


def test_degenerate_near_plane_and_huge_triangles(pr, oracle):
    rng = np.random.default_rng(9)
    tris = [
        [[-0.5, -0.5, 3.0], [0.5, -0.5, 3.0], [0.0, -0.5, 3.0]],       # zero area (collinear)
        [[0.2, 0.2, 4.0], [0.2, 0.2, 4.0], [0.2, 0.2, 4.0]],          # a point
        [[-0.3, 0.1, -1.0], [0.4, 0.2, 2.0], [0.1, -0.4, 1.5]],       # crosses the near plane
        [[-0.3, 0.1, -1.0], [0.4, 0.2, -2.0], [0.1, -0.4, -1.5]],     # behind the camera
        [[-50.0, -50.0, 6.0], [50.0, -50.0, 6.5], [0.0, 80.0, 7.0]],  # covers the screen
        [[-0.2, -0.2, 0.5], [0.3, -0.1, 0.0005], [0.1, 0.3, 0.8]],    # one vertex just past the near plane
        [[0.0, -1.0, 2.0], [0.0, 1.0, 2.0], [0.0, 0.0, 9.0]],         # edge-on at x = 0
    ]
    pos = np.array(tris, np.float32).reshape(-1, 3)
    vel = rng.normal(0, 0.1, pos.shape).astype(np.float32)
    vel[3:6] = 0.0
    sc = S.Scene(pos, vel, rng.uniform(0, 1, pos.shape).astype(np.float32),
                 np.arange(pos.shape[0], dtype=np.int32).reshape(-1, 3))
    for mode in MODES:
        _, view = small_case(mode, W=96, H=80)
        g = gpu_frame(pr, sc, view)
        o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
        # a 7,680-pixel frame built around an edge-on triangle: every mismatch
        # must be excused, the frame-level agreement floor is relaxed
        compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"], min_agree=0.999)
        assert (o["id"] != BG).mean() > 0.3     # the screen-covering triangle and the near ones cover it


def test_host_buffers_match_device_buffers(pr):
    import ctypes as C
    sc, view = small_case(S.MODE_BOTH, seed=4, W=120, H=90, T=400)
    dev = gpu_frame(pr, sc, view)
    h = pr.pr_scene_upload(sc.pos, sc.vel, sc.col, sc.tri)   # host inputs
    ids = np.empty(view.W * view.H, np.uint32)
    depth = np.empty(view.W * view.H, np.float32)
    rgb = np.empty(3 * view.W * view.H, np.float32)
    pr.pr_rasterize(h, view, None, ids, depth)
    pr.pr_shade(h, view, ids, rgb)
    pr.pr_scene_free(h)
    assert np.array_equal(ids, dev["id"]) and np.array_equal(depth, dev["depth"])
    assert np.array_equal(rgb, dev["rgb"])


def test_many_tiles_per_triangle_regrows_bins(pr, oracle):
    """Large triangles overlap many tiles, so the first bin capacity
    overflows; the library regrows its buffers and the frame is exact."""
    rng = np.random.default_rng(5)
    T = 60
    c = rng.uniform([-1, -1, 2], [1, 1, 6], (T, 1, 3))
    pos = (c + rng.uniform(-2.5, 2.5, (T, 3, 3)) * [1, 1, 0.2]).astype(np.float32).reshape(-1, 3)
    sc = S.Scene(pos, rng.normal(0, 0.05, pos.shape).astype(np.float32), rng.uniform(0, 1, pos.shape).astype(np.float32),
                 np.arange(3 * T, dtype=np.int32).reshape(T, 3))
    _, view = small_case(S.MODE_ROLLING, W=320, H=240)
    g = gpu_frame(pr, sc, view, tile=8)
    assert g["stats"]["pairs"] > 2 * T + (view.W // 8) * (view.H // 8)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"])


def test_invalid_inputs_raise(pr):
    sc, view = small_case(S.MODE_ROLLING, W=16, H=16, T=4)
    bad = sc.pos.copy()
    bad[2, 1] = np.nan
    with pytest.raises(pr.PrError) as e:
        pr.pr_scene_upload(bad, sc.vel, sc.col, sc.tri)
    assert e.value.status == pr.PR_ERR_NONFINITE
    tri = sc.tri.copy()
    tri[1, 2] = 10 ** 6
    with pytest.raises(pr.PrError) as e:
        pr.pr_scene_upload(sc.pos, sc.vel, sc.col, tri)
    assert e.value.status == pr.PR_ERR_INVALID_ARG
    h = pr.pr_scene_upload(sc.pos, sc.vel, sc.col, sc.tri)
    try:
        v2 = S.View(**{**view.__dict__, "mode": 7})
        with pytest.raises(pr.PrError):
            pr.pr_rasterize(h, v2, None, np.empty(256, np.uint32), None)
        v3 = S.View(**{**view.__dict__, "d": (0.8, 0.8)})
        with pytest.raises(pr.PrError):
            pr.pr_rasterize(h, v3, None, np.empty(256, np.uint32), None)
        # Non-finite camera or shading constants are refused before any launch.
        for field, value in (("z_near", float("inf")), ("k_a", float("nan")), ("k_d", float("inf"))):
            v4 = S.View(**{**view.__dict__, field: value})
            with pytest.raises(pr.PrError) as e:
                pr.pr_rasterize(h, v4, None, np.empty(256, np.uint32), None)
            assert e.value.status == pr.PR_ERR_INVALID_ARG
    finally:
        pr.pr_scene_free(h)


@pytest.mark.parametrize("mode", MODES)
def test_fp64_retest_meets_strict_tolerance(pr, oracle, mode):
    """Precision form: FP32 pairs whose outcome the error bound cannot settle
    are re-tested in FP64, after which every id mismatch with the FP64
    oracle lies within 1e-6 (barycentric edge distance or relative depth gap)
    -- the tolerance of the FP64-checked result."""
    sc, view = small_case(mode, seed=11)
    g = gpu_frame(pr, sc, view, fp64=1)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"], fp64=True)
    st = g["stats"]
    # near-edge, near-tie and ill-conditioned-depth pixels: a minority, even
    # on these large, randomly oriented triangles (the foveated frame, whose
    # fovea packs many pixels next to each edge, flags about a quarter)
    assert 0 < st["flagged"] < 0.3 * view.W * view.H
    assert st["fp64_depth_err"] < 1e-4
    # the FP32-only frame differs from the re-tested one only at flagged pixels
    g32 = gpu_frame(pr, sc, view, fp64=0)
    assert (g32["id"] != g["id"]).sum() <= st["changed"]
