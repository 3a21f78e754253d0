"""The scratch-array entry point pr_rasterize_noalloc, for callers that may
not allocate device memory (a frame loop that must not stall on
cudaMalloc/cudaFree, or a host that owns all GPU memory up front).  Two
calls in a row -- of different sizes, so a stale array would show -- must
each equal pr_rasterize on the same inputs, id for id and depth for depth.
Collected last on purpose; it passes alone in a fresh process and after the
other tests."""
import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frames():
    sc1 = S.random_triangles(1000, 21)
    p0, p1 = S.head_poses(2.0, 0.5)
    v1 = S.View(W=256, H=200, tan_x=0.5, tan_y=0.45, pose0=p0, pose1=p1, mode=S.MODE_BOTH, fovea=(0.4, 0.55))
    sc2 = S.random_triangles(300, 22, offset=0.3)
    v2 = S.View(W=97, H=61, tan_x=0.6, tan_y=0.4, pose0=p0, pose1=p1, mode=S.MODE_ROLLING)
    return [(sc1, v1, 16), (sc2, v2, 8)]


def test_noalloc_matches_rasterize_on_two_calls(pr):
    import torch
    for sc, view, tile in _frames():
        n = view.W * view.H
        pos, vel, col, tri = _dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri)
        params = pr.make_params("zenon", tile)
        h = pr.pr_scene_upload(pos, vel, col, tri)
        ref_id = torch.empty(n, dtype=torch.int32, device="cuda")
        ref_d = torch.empty(n, dtype=torch.float32, device="cuda")
        pr.pr_rasterize(h, view, params, ref_id, ref_d)
        pr.pr_scene_free(h)
        ids = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        dep = torch.full((n,), 7.0, dtype=torch.float32, device="cuda")
        pr.pr_rasterize_noalloc(pos, vel, col, tri, view, params, ids, dep)
        torch.cuda.synchronize()
        assert (ref_id != -1).any()
        assert torch.equal(ids, ref_id)
        assert torch.equal(dep, ref_d)


def test_noalloc_rejects_host_buffers_and_oversize(pr):
    sc, view, tile = _frames()[1]
    with pytest.raises(pr.PrError) as e:
        pr.pr_rasterize_noalloc(sc.pos, sc.vel, sc.col, sc.tri, view)       # host arrays
    assert e.value.status == pr.PR_ERR_INVALID_ARG
    import torch
    big = S.View(**{**view.__dict__, "W": 8192, "H": 8192})                # 8 bytes/pixel alone is 512 MiB
    ids = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pr.PrError) as e:
        pr.pr_rasterize_noalloc(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri), big, None, ids, None)
    assert e.value.status == pr.PR_ERR_INVALID_ARG


def test_noalloc_bins_that_do_not_fit_report_overflow_and_the_next_call_is_correct(pr):
    """A frame whose fixed scratch fits the array but whose bins do not
    (every one of 3,000 triangles binned to each of 16,384 tiles by the
    whole-viewport bound: 49 M entries at 20 bytes, against about 54 MiB
    left) runs, stops filling the bins at their capacity and returns
    PR_ERR_OVERFLOW; the call after it on the same array is exact again."""
    import torch
    sc = S.random_triangles(3000, 23)
    p0, p1 = S.head_poses(1.0, 0.0)
    view = S.View(W=1024, H=1024, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=S.MODE_ROLLING)
    n = view.W * view.H
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    dep = torch.empty(n, dtype=torch.float32, device="cuda")
    with pytest.raises(pr.PrError) as e:
        pr.pr_rasterize_noalloc(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri), view,
                                pr.make_params("trivial", 8), ids, dep)
    assert e.value.status == pr.PR_ERR_OVERFLOW
    test_noalloc_matches_rasterize_on_two_calls(pr)


def test_noalloc_rejects_what_it_cannot_run(pr):
    """The FP64 re-test needs flag buffers the array does not provide, so
    fp64_retest = 1 is refused; view fields are validated exactly as for
    pr_rasterize (an infinite z_near is refused)."""
    import torch
    sc, view, tile = _frames()[1]
    args = (_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri))
    ids = torch.empty(view.W * view.H, dtype=torch.int32, device="cuda")
    with pytest.raises(pr.PrError) as e:
        pr.pr_rasterize_noalloc(*args, view, pr.make_params("zenon", tile, 1), ids, None)
    assert e.value.status == pr.PR_ERR_INVALID_ARG
    bad = S.View(**{**view.__dict__, "z_near": float("inf")})
    with pytest.raises(pr.PrError) as e:
        pr.pr_rasterize_noalloc(*args, bad, pr.make_params("zenon", tile), ids, None)
    assert e.value.status == pr.PR_ERR_INVALID_ARG
