"""Batched/graph forms, the adjoint, and full-size sampled parity, on the GPU.

* batched == per-view plain calls, bit for bit, over scenes of different
  sizes, modes, resolutions and tile sizes;
* a captured graph replays the eager result, also after the scene changes;
* the stage (e) adjoint matches the FP64 oracle gradient (itself pinned to
  central finite differences) on interior pixels, rel. L2 error <= 1e-3;
* the full-resolution stereo HMD frame and the large 1M-triangle frame agree
  with the oracle on seeded pixel samples.
"""
import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S
from tests.parity_util import BG, compare
from tests.test_parity_gpu import gpu_frame

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _upload(pr, sc):
    return pr.pr_scene_upload(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri))


def _views_mixed():
    out = []
    for k, (mode, W, H, tile, T) in enumerate([(S.MODE_CLASSIC, 131, 97, 8, 500), (S.MODE_ROLLING, 200, 150, 16, 900),
                                               (S.MODE_FOVEATED, 96, 160, 32, 300), (S.MODE_BOTH, 257, 129, 16, 1200),
                                               (S.MODE_BOTH, 64, 64, 8, 700)]):
        sc = S.random_triangles(T, 40 + k, offset=0.5 if k % 2 else None)
        p0, p1 = S.head_poses(1.0 + k, 0.3 * k, 0.01 * k)
        out.append((sc, S.View(W=W, H=H, tan_x=0.55, tan_y=0.5, pose0=p0, pose1=p1, mode=mode,
                               fovea=(0.3 + 0.1 * k, 0.6 - 0.05 * k)), tile))
    return out


def test_batched_equals_plain(pr):
    import torch
    cases = _views_mixed()
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    ws = pr.pr_workspace_create()
    try:
        outs = []
        entries = []
        for h, (sc, v, tile) in zip(handles, cases):
            n = v.W * v.H
            o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                 torch.empty(3 * n, device="cuda"))
            outs.append(o)
            entries.append((h, v, o[0], o[1], o[2], tile))
        pr.pr_rasterize_batch(ws, entries)
        st = pr.pr_workspace_stats(ws)
        assert st["pixels"] == sum(v.W * v.H for _, v, _ in cases)
        for h, (sc, v, tile), o in zip(handles, cases, outs):
            n = v.W * v.H
            ids = torch.empty(n, dtype=torch.int32, device="cuda")
            dep = torch.empty(n, device="cuda")
            rgb = torch.empty(3 * n, device="cuda")
            pr.pr_rasterize(h, v, pr.make_params("zenon", tile), ids, dep)
            pr.pr_shade(h, v, ids, rgb)
            assert torch.equal(ids, o[0]) and torch.equal(dep, o[1]) and torch.equal(rgb, o[2])
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_workspace_reuse_across_frame_sizes(pr):
    """Keys: a frame whose keys fit in L2 clears them at its start; a larger
    one has its reader set them back to ~0 and clears only beyond what earlier
    readers left so.  A sequence of batches that shrink and grow on one
    workspace, across both forms (frames of 118 MB and of a few MB of keys),
    with images and without, eager and as graph replays, gives every batch
    the bits of the same batch on a fresh workspace."""
    import torch
    cases = _views_mixed()
    for k in range(4):  # four 2048 x 1800 views: 14.7 Mpx, 118 MB of keys together
        sc = S.random_triangles(2000, 60 + k)
        p0, p1 = S.head_poses(1.5 + k, 0.2 * k, 0.01)
        cases.append((sc, S.View(W=2048, H=1800, tan_x=0.6, tan_y=0.55, pose0=p0, pose1=p1, mode=k % 4,
                                 fovea=(0.45, 0.5)), 16))
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    big = [5, 6, 7, 8]

    def run(ws, picks, with_rgb, graph=False):
        outs, entries = [], []
        for k in picks:
            sc, v, tile = cases[k]
            n = v.W * v.H
            o = (torch.full((n,), -5, dtype=torch.int32, device="cuda"), torch.full((n,), -5.0, device="cuda"),
                 torch.full((3 * n,), -5.0, device="cuda") if with_rgb else None)
            outs.append(o)
            entries.append((handles[k], v, o[0], o[1], o[2], tile))
        if graph:
            g = pr.pr_graph_capture_batch(ws, entries)
            for o in outs:
                o[0].fill_(-5)
            pr.pr_graph_launch(g)
            pr.pr_graph_launch(g)
            pr.pr_graph_free(g)
        else:
            pr.pr_rasterize_batch(ws, entries)
        torch.cuda.synchronize()
        return [tuple(x.cpu().numpy() if x is not None else None for x in o) for o in outs]

    seq = [(big + [0, 1], True, False), (big, False, False), (big[:2] + [4], True, False), (big + [2], True, True),
           ([0, 1, 2, 3, 4], False, False), (big[::-1], True, False), ([3, 0], True, True), (big + [4], True, False),
           (big, True, True), ([4, 2], True, False)]
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()  # graphs are captured on a non-default stream
    try:
        torch.cuda.set_stream(stream)
        for picks, with_rgb, graph in seq:
            got = run(ws, picks, with_rgb, graph)
            fresh = pr.pr_workspace_create()
            try:
                want = run(fresh, picks, with_rgb)
            finally:
                pr.pr_workspace_free(fresh)
            for k, a, b in zip(picks, got, want):
                assert np.array_equal(a[0], b[0]), (picks, k)
                assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32)), (picks, k)
                if with_rgb:
                    assert np.array_equal(a[2].view(np.uint32), b[2].view(np.uint32)), (picks, k)
                assert (a[0] != -5).all()
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_graph_replay_after_small_frames(pr):
    """A graph of a frame larger than L2's share for keys (its shading sets
    the keys back, and its start clears none) replayed after eager frames
    that leave keys in use -- a small frame, whose keys are cleared at its
    start instead -- still starts from clean keys: the replay equals the
    eager frame of the same batch."""
    import torch
    big = []
    for k in range(4):  # 14.7 Mpx, 118 MB of keys
        sc = S.random_triangles(2000, 80 + k)
        p0, p1 = S.head_poses(1.0 + k, 0.1 * k, 0.01)
        big.append((sc, S.View(W=2048, H=1800, tan_x=0.6, tan_y=0.55, pose0=p0, pose1=p1, mode=(k + 1) % 4,
                               fovea=(0.5, 0.45)), 16))
    small = _views_mixed()
    cases = big + small
    handles = [_upload(pr, sc) for sc, _, _ in cases]

    def entries_of(picks):
        out = []
        for k in picks:
            sc, v, tile = cases[k]
            n = v.W * v.H
            out.append((handles[k], v, torch.full((n,), -5, dtype=torch.int32, device="cuda"),
                        torch.full((n,), -5.0, device="cuda"), torch.full((3 * n,), -5.0, device="cuda"), tile))
        return out

    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    g = None
    try:
        torch.cuda.set_stream(stream)
        eb = entries_of([0, 1, 2, 3])
        pr.pr_rasterize_batch(ws, eb)
        torch.cuda.synchronize()
        want = [tuple(x.cpu().numpy() for x in e[2:5]) for e in eb]
        g = pr.pr_graph_capture_batch(ws, eb)
        for picks in ([4, 5], [6, 7, 8], [4]):  # small frames (keys cleared at their start, left in use)
            pr.pr_rasterize_batch(ws, entries_of(picks))
            for e in eb:
                e[2].fill_(-5)
            pr.pr_graph_launch(g)
            torch.cuda.synchronize()
            for e, w in zip(eb, want):
                got = tuple(x.cpu().numpy() for x in e[2:5])
                assert np.array_equal(got[0], w[0])
                assert np.array_equal(got[1].view(np.uint32), w[1].view(np.uint32))
                assert np.array_equal(got[2].view(np.uint32), w[2].view(np.uint32))
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
        if g is not None:
            pr.pr_graph_free(g)
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_each_graph_keeps_its_own_status(pr):
    """Two graphs on one workspace replayed back to back: the status (and
    statistics) of the first can be read after the second has run, as a
    frame loop that reads one replay's status while the next one runs does."""
    import torch
    cases = _views_mixed()
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    graphs = []
    try:
        torch.cuda.set_stream(stream)
        # one eager frame of every view first sizes the workspace for both
        # graphs (a capture that regrew it would make the other graph stale)
        every = []
        for k, (sc, v, tile) in enumerate(cases):
            n = v.W * v.H
            every.append((handles[k], v, torch.empty(n, dtype=torch.int32, device="cuda"),
                          torch.empty(n, device="cuda"), None, tile))
        pr.pr_rasterize_batch(ws, every)
        stats = []
        for picks in ([0, 1], [2, 3, 4]):
            entries = []
            for k in picks:
                sc, v, tile = cases[k]
                n = v.W * v.H
                entries.append((handles[k], v, torch.empty(n, dtype=torch.int32, device="cuda"),
                                torch.empty(n, device="cuda"), None, tile))
            g = pr.pr_graph_capture_batch(ws, entries)
            graphs.append((g, entries))
            pr.pr_graph_launch(g)
            st = pr.pr_workspace_stats(ws)
            stats.append((st["pixels"], st["pairs"], st["culled"]))
        assert stats[0] != stats[1]
        pr.pr_graph_enqueue(graphs[0][0])
        pr.pr_graph_enqueue(graphs[1][0])
        stream.synchronize()
        for (g, _), want in zip(graphs, stats):
            pr.pr_graph_status(g)
            st = pr.pr_workspace_stats(ws)
            assert (st["pixels"], st["pairs"], st["culled"]) == want
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
        for g, _ in graphs:
            pr.pr_graph_free(g)
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_graph_replay_matches_eager(pr):
    import torch
    cases = _views_mixed()[:3]
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    try:
        with torch.cuda.stream(stream):
            outs, entries = [], []
            for h, (sc, v, tile) in zip(handles, cases):
                n = v.W * v.H
                o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                     torch.empty(3 * n, device="cuda"))
                outs.append(o)
                entries.append((h, v, o[0], o[1], o[2], tile))
            graph = pr.pr_graph_capture_batch(ws, entries)
            ref = [tuple(x.clone() for x in o) for o in outs]
            for o in outs:
                for x in o:
                    x.fill_(7)
            pr.pr_graph_launch(graph)
            for o, r in zip(outs, ref):
                assert all(torch.equal(a, b) for a, b in zip(o, r))
            # new vertex positions: the replay follows the scene's contents
            sc0 = cases[0][0]
            pr.pr_scene_update(handles[0], _dev(sc0.pos + 0.05), None, None)
            pr.pr_graph_launch(graph)
            ws2 = pr.pr_workspace_create()
            o2 = [tuple(torch.empty_like(x) for x in o) for o in outs]
            pr.pr_rasterize_batch(ws2, [(h, v, a, b, c, tile) for (h, (sc, v, tile), (a, b, c))
                                        in zip(handles, cases, o2)])
            pr.pr_workspace_free(ws2)
            for o, r in zip(outs, o2):
                assert all(torch.equal(a, b) for a, b in zip(o, r))
            pr.pr_graph_free(graph)
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_graph_stage_times_are_optional(pr):
    """A graph captured with stage events reports stage times per replay; one
    captured without (the default) reports zeros; both give the same image."""
    import torch
    cases = _views_mixed()[:2]
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    try:
        with torch.cuda.stream(stream):
            outs, entries = [], []
            for h, (sc, v, tile) in zip(handles, cases):
                n = v.W * v.H
                o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                     torch.empty(3 * n, device="cuda"))
                outs.append(o)
                entries.append((h, v, o[0], o[1], o[2], tile))
            got = {}
            for timed in (0, 1):
                graph = pr.pr_graph_capture_batch(ws, entries, pr.make_params(graph_stage_times=timed))
                for o in outs:
                    for x in o:
                        x.fill_(7)
                pr.pr_graph_launch(graph)
                ms = pr.pr_workspace_stats(ws)["stage_ms"]
                got[timed] = [tuple(x.clone() for x in o) for o in outs]
                pr.pr_graph_free(graph)
                if timed:
                    assert ms[0] > 0 and ms[1] > 0 and ms[2] > 0 and ms[5] > 0
                else:
                    assert all(x == 0.0 for x in ms)
            for a, b in zip(got[0], got[1]):
                assert all(torch.equal(x, y) for x, y in zip(a, b))
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_graph_keeps_its_view_table_and_refuses_when_stale(pr):
    """A graph replays the views it was captured with, after other calls on
    the same workspace; a call that regrows the workspace makes it stale."""
    import torch
    cases = _views_mixed()[:3]
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    try:
        with torch.cuda.stream(stream):
            outs, entries = [], []
            for h, (sc, v, tile) in zip(handles, cases):
                n = v.W * v.H
                o = tuple(torch.empty(n * k, dtype=dt, device="cuda")
                          for k, dt in ((1, torch.int32), (1, torch.float32), (3, torch.float32)))
                outs.append(o)
                entries.append((h, v, o[0], o[1], o[2], tile))
            graph = pr.pr_graph_capture_batch(ws, entries)
            ref = [tuple(x.clone() for x in o) for o in outs]
            # a smaller eager frame of other views on the same workspace
            sc1, v1, t1 = cases[1]
            p0, p1 = S.head_poses(-4.0, 2.0)
            other = S.View(W=v1.W // 2, H=v1.H // 2, tan_x=0.4, tan_y=0.4, pose0=p0, pose1=p1, mode=S.MODE_CLASSIC,
                           fovea=(0.5, 0.5))
            n = other.W * other.H
            oo = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                  torch.empty(3 * n, device="cuda"))
            pr.pr_rasterize_batch(ws, [(handles[1], other, oo[0], oo[1], oo[2], t1)])
            for o in outs:
                for x in o:
                    x.fill_(7)
            pr.pr_graph_launch(graph)
            for o, r in zip(outs, ref):
                assert all(torch.equal(a, b) for a, b in zip(o, r))
            # a much larger frame regrows the scratch: the graph is refused
            big_sc = S.random_triangles(20000, 77)
            hb = _upload(pr, big_sc)
            handles.append(hb)
            p0, p1 = S.head_poses(2.0, 1.0)
            bv = S.View(W=1024, H=1024, tan_x=0.6, tan_y=0.6, pose0=p0, pose1=p1, mode=S.MODE_BOTH, fovea=(0.5, 0.5))
            nb = bv.W * bv.H
            ob = (torch.empty(nb, dtype=torch.int32, device="cuda"), torch.empty(nb, device="cuda"),
                  torch.empty(3 * nb, device="cuda"))
            pr.pr_rasterize_batch(ws, [(hb, bv, ob[0], ob[1], ob[2], 16)])
            for launch in (pr.pr_graph_launch, pr.pr_graph_enqueue):
                with pytest.raises(pr.PrError) as ei:
                    launch(graph)
                assert ei.value.status == pr.PR_ERR_INVALID_ARG
            pr.pr_graph_free(graph)
            # a fresh capture on the regrown workspace works again, also
            # enqueued without a host wait and its status read afterwards
            graph = pr.pr_graph_capture_batch(ws, entries)
            for o in outs:
                for x in o:
                    x.fill_(7)
            pr.pr_graph_enqueue(graph)
            pr.pr_graph_enqueue(graph)
            stream.synchronize()
            pr.pr_graph_status(graph)
            assert pr.pr_workspace_stats(ws)["pixels"] == sum(v.W * v.H for _, v, _ in cases)
            for o, r in zip(outs, ref):
                assert all(torch.equal(a, b) for a, b in zip(o, r))
            pr.pr_graph_free(graph)
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


@pytest.mark.parametrize("mode", [S.MODE_ROLLING, S.MODE_BOTH, S.MODE_CLASSIC])
def test_backward_matches_oracle_gradient(pr, oracle, mode):
    import torch
    sc = S.random_triangles(800, 5, offset=0.15)
    p0, p1 = S.head_poses(2.0, 0.0)
    view = S.View(W=160, H=128, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode, fovea=(0.47, 0.52))
    g = gpu_frame(pr, sc, view, keep=True)
    h = g["scene"]
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri, near=True)
    n = view.W * view.H
    interior = (o["id"] != BG) & (g["id"] == o["id"]) & (o["bmin"] > 1e-3) & (o["gap"] > 1e-3) & (o["near"] > 1e-3)
    assert interior.mean() > 0.05
    rng = np.random.default_rng(mode)
    gr = rng.normal(size=(n, 3)) * interior[:, None]
    ids = _dev(g["id"].view(np.int32))
    gplanar = _dev(np.ascontiguousarray(gr.T.astype(np.float32)).reshape(-1))
    dcol, dpos, dvel = (torch.zeros(sc.V * 3, device="cuda") for _ in range(3))
    pr.pr_backward(h, view, ids, gplanar, dcol, dpos, dvel)
    pr.pr_scene_free(h)
    oc, op, ov = oracle.grad(view, sc.pos, sc.vel, sc.col, sc.tri, o["id"], gr)
    for name, gpu, ref in (("col", dcol, oc), ("pos", dpos, op), ("vel", dvel, ov)):
        a = gpu.cpu().numpy().reshape(-1, 3).astype(np.float64)
        if name == "vel" and mode == S.MODE_CLASSIC:
            assert np.abs(a).max() == 0.0      # t = 0: velocities do not act
            continue
        err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
        assert err <= 1e-3, (name, err)


def test_autograd_function_matches_pr_backward(pr):
    import torch
    from paper_1806_05385_gb300.autograd import Renderer
    sc = S.random_triangles(400, 6, offset=0.2)
    p0, p1 = S.head_poses(2.0, 0.0)
    view = S.View(W=96, H=80, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=S.MODE_BOTH, fovea=(0.5, 0.5))
    r = Renderer(torch.from_numpy(sc.tri), sc.V, view)
    col = torch.tensor(sc.col, device="cuda", requires_grad=True)
    pos = torch.tensor(sc.pos, device="cuda", requires_grad=True)
    vel = torch.tensor(sc.vel, device="cuda", requires_grad=True)
    rgb = r.render(col, pos, vel)
    tgt = torch.zeros_like(rgb)
    loss = ((rgb - tgt) ** 2).sum()
    loss.backward()
    # colour enters linearly: the analytic colour gradient equals an FP32
    # central difference with a large step exactly up to rounding
    k = int(np.argmax(np.abs(col.grad.cpu().numpy()).ravel()))
    hstep = 0.05
    with torch.no_grad():
        c1, c2 = col.detach().clone(), col.detach().clone()
        c1.view(-1)[k] += hstep
        c2.view(-1)[k] -= hstep
        l1 = ((r.render(c1, pos.detach(), vel.detach())) ** 2).sum()
        l2 = ((r.render(c2, pos.detach(), vel.detach())) ** 2).sum()
    fd = float((l1 - l2) / (2 * hstep))
    assert fd == pytest.approx(float(col.grad.view(-1)[k]), rel=1e-3)
    assert torch.isfinite(pos.grad).all() and pos.grad.abs().sum() > 0
    r.close()


def _sampled(pr, oracle, sc, views, n_uniform, win, seed, tile=16):
    """Render the views at full size on the GPU; compare seeded pixel samples."""
    for k, v in enumerate(views):
        g = gpu_frame(pr, sc, v, tile=tile)
        pix = S.sample_pixels(v.W, v.H, n_uniform, 1, win, seed + k)
        o = oracle.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix)
        rep = compare(oracle, v, sc, o, g["id"], g["depth"], g["rgb"], pix=pix)
        assert rep["hit_frac"] > 0.01, rep


def test_full_size_hmd_frame_sampled(pr, oracle):
    sc, views = S.config_hmd(seed=2)
    _sampled(pr, oracle, sc, views, n_uniform=1500, win=24, seed=100)


@pytest.mark.slow
def test_large_frame_sampled(pr, oracle):
    sc, views = S.config_large(seed=3)
    _sampled(pr, oracle, sc, views, n_uniform=300, win=12, seed=200, tile=32)


def test_full_size_hmd_frame_fp64_retest_strict(pr, oracle):
    sc, views = S.config_hmd(seed=2)
    v = views[0]
    g = gpu_frame(pr, sc, v, fp64=1)
    pix = S.sample_pixels(v.W, v.H, 1500, 1, 24, 300)
    o = oracle.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix)
    compare(oracle, v, sc, o, g["id"], g["depth"], g["rgb"], pix=pix, fp64=True)
    assert g["stats"]["flagged"] > 0


def test_backward_batch_equals_per_view(pr):
    import torch
    cases = _views_mixed()
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    ws = pr.pr_workspace_create()
    try:
        rng = np.random.default_rng(3)
        ent, per = [], []
        for h, (sc, v, tile) in zip(handles, cases):
            n = v.W * v.H
            ids = torch.empty(n, dtype=torch.int32, device="cuda")
            pr.pr_rasterize(h, v, pr.make_params("zenon", tile), ids, None)
            g = _dev(rng.normal(size=3 * n).astype(np.float32))
            a = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            b = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            ent.append((h, v, ids, g, *a))
            pr.pr_backward(h, v, ids, g, *b)
            per.append(b)
        pr.pr_backward_batch(ws, ent)
        for e, b in zip(ent, per):
            for x, y in zip(e[4:], b):
                assert torch.allclose(x, y, rtol=1e-4, atol=1e-5 * float(y.abs().max()) + 1e-12)
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def _views_many(n=80):
    """More views than a launch passes as a kernel parameter (72): the
    shading and adjoint kernels then read the views from the device table,
    while one-view calls pass theirs as a parameter."""
    scenes = [S.random_triangles(300 + 100 * k, 60 + k, offset=0.5 if k % 2 else None) for k in range(5)]
    out = []
    for k in range(n):
        p0, p1 = S.head_poses(0.5 + 0.1 * k, 0.05 * k, 0.002 * k)
        v = S.View(W=40 + (7 * k) % 50, H=33 + (5 * k) % 40, tan_x=0.55, tan_y=0.5, pose0=p0, pose1=p1, mode=k % 4,
                   fovea=(0.3 + 0.005 * k, 0.6 - 0.003 * k))
        out.append((k % 5, v, (8, 16, 32)[k % 3]))
    return scenes, out


def test_batches_beyond_the_parameter_table(pr):
    """80 views in one batch (the device-table kernels) against one-view
    calls (the parameter-table kernels): forward bit for bit, the adjoint of
    the batch and of a training frame up to the order of float atomics."""
    import torch
    scenes, cases = _views_many()
    handles = [_upload(pr, sc) for sc in scenes]
    ws = pr.pr_workspace_create()
    try:
        rng = np.random.default_rng(5)
        entries, outs, bwd, per, fgrads = [], [], [], [], []
        for si, v, tile in cases:
            h, sc, n = handles[si], scenes[si], v.W * v.H
            o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                 torch.empty(3 * n, device="cuda"))
            outs.append(o)
            entries.append((h, v, o[0], o[1], o[2], tile))
        pr.pr_rasterize_batch(ws, entries)
        for (si, v, tile), o in zip(cases, outs):
            h, sc, n = handles[si], scenes[si], v.W * v.H
            ids = torch.empty(n, dtype=torch.int32, device="cuda")
            dep = torch.empty(n, device="cuda")
            rgb = torch.empty(3 * n, device="cuda")
            pr.pr_rasterize(h, v, pr.make_params("zenon", tile), ids, dep)
            pr.pr_shade(h, v, ids, rgb)
            assert torch.equal(ids, o[0]) and torch.equal(dep, o[1]) and torch.equal(rgb, o[2])
            g = _dev(rng.normal(size=3 * n).astype(np.float32))
            a = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            b = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            f = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            bwd.append((h, v, ids, g, *a))
            pr.pr_backward(h, v, ids, g, *b)
            per.append(b)
            fgrads.append(dict(grad_rgb=g, dcol=f[0], dpos=f[1], dvel=f[2]))
        assert sum(float((o[0] >= 0).sum()) for o in outs) > 0
        pr.pr_backward_batch(ws, bwd)
        pr.pr_frame_batch(ws, entries, fgrads)
        for e, b, f in zip(bwd, per, fgrads):
            for x, y in zip(e[4:], b):
                assert torch.allclose(x, y, rtol=1e-4, atol=1e-5 * float(y.abs().max()) + 1e-12)
            for x, y in zip((f["dcol"], f["dpos"], f["dvel"]), b):
                assert torch.allclose(x, y, rtol=1e-4, atol=1e-5 * float(y.abs().max()) + 1e-12)
        assert sum(float(b[0].abs().sum()) for b in per) > 0
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def _frame_setup(pr, cases):
    import torch
    handles = [_upload(pr, sc) for sc, _, _ in cases]
    outs, entries = [], []
    for h, (sc, v, tile) in zip(handles, cases):
        n = v.W * v.H
        o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
             torch.empty(3 * n, device="cuda"))
        outs.append(o)
        entries.append((h, v, o[0], o[1], o[2], tile))
    return handles, outs, entries


def test_frame_batch_equals_forward_then_adjoint(pr):
    """The training frame's forward is the batched forward bit for bit; its
    adjoint (for the views given a gradient, upstream gradient or L2 target)
    equals the separate adjoint call up to the order of float atomics."""
    import torch
    cases = _views_mixed()
    handles, outs, entries = _frame_setup(pr, cases)
    ws, ws2 = pr.pr_workspace_create(), pr.pr_workspace_create()
    try:
        rng = np.random.default_rng(11)
        grads, want = [], []
        for k, (sc, v, tile) in enumerate(cases):
            n = v.W * v.H
            d = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            if k == 1:
                grads.append(None)            # a view of the batch without a gradient
            elif k == 3:
                grads.append(dict(target_rgb=_dev(rng.uniform(size=3 * n).astype(np.float32)), dcol=d[0],
                                  dpos=d[1], dvel=d[2]))
            else:
                grads.append(dict(grad_rgb=_dev(rng.normal(size=3 * n).astype(np.float32)), dcol=d[0], dpos=d[1],
                                  dvel=d[2]))
        pr.pr_frame_batch(ws, entries, grads)
        ref_outs, ref_entries = [], []
        for h, (sc, v, tile) in zip(handles, cases):
            n = v.W * v.H
            o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                 torch.empty(3 * n, device="cuda"))
            ref_outs.append(o)
            ref_entries.append((h, v, o[0], o[1], o[2], tile))
        pr.pr_rasterize_batch(ws2, ref_entries)
        for o, r in zip(outs, ref_outs):
            assert all(torch.equal(a, b) for a, b in zip(o, r))
        bwd = []
        for k, (h, (sc, v, tile), o) in enumerate(zip(handles, cases, ref_outs)):
            if grads[k] is None:
                continue
            g = grads[k]["grad_rgb"] if "grad_rgb" in grads[k] else 2.0 * (o[2] - grads[k]["target_rgb"])
            d = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
            bwd.append((h, v, o[0], g, *d))
            want.append((k, d))
        pr.pr_backward_batch(ws2, bwd)
        for k, d in want:
            got = (grads[k]["dcol"], grads[k]["dpos"], grads[k]["dvel"])
            for x, y in zip(got, d):
                assert torch.allclose(x, y, rtol=1e-4, atol=1e-5 * float(y.abs().max()) + 1e-12)
            assert float(got[0].abs().sum()) > 0
    finally:
        pr.pr_workspace_free(ws)
        pr.pr_workspace_free(ws2)
        for h in handles:
            pr.pr_scene_free(h)


def test_frame_graph_replays_eager_frame(pr):
    """forward + L2-loss gradient + adjoint as one graph: a replay with the
    gradient buffers zeroed reproduces the eager frame."""
    import torch
    cases = _views_mixed()[1:4]
    stream = torch.cuda.Stream()
    handles, outs, entries = _frame_setup(pr, cases)
    ws = pr.pr_workspace_create()
    try:
        with torch.cuda.stream(stream):
            rng = np.random.default_rng(5)
            grads = []
            for sc, v, _ in cases:
                d = tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3))
                grads.append(dict(target_rgb=_dev(rng.uniform(size=3 * v.W * v.H).astype(np.float32)), dcol=d[0],
                                  dpos=d[1], dvel=d[2]))
            pr.pr_frame_batch(ws, entries, grads)
            eager_out = [tuple(x.clone() for x in o) for o in outs]
            eager_d = [tuple(g[n].clone() for n in ("dcol", "dpos", "dvel")) for g in grads]
            graph = pr.pr_graph_capture_frame(ws, entries, grads)   # runs the frame once more, eagerly
            for rep in range(2):
                for g in grads:
                    for n in ("dcol", "dpos", "dvel"):
                        g[n].zero_()
                for o in outs:
                    for x in o:
                        x.fill_(3)
                pr.pr_graph_launch(graph)
                stream.synchronize()
                for o, r in zip(outs, eager_out):
                    assert all(torch.equal(a, b) for a, b in zip(o, r))
                for g, r in zip(grads, eager_d):
                    for n, y in zip(("dcol", "dpos", "dvel"), r):
                        assert torch.allclose(g[n], y, rtol=1e-4, atol=1e-5 * float(y.abs().max()) + 1e-12)
            pr.pr_graph_free(graph)
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_frame_gradient_rejects_host_buffers(pr):
    import torch
    cases = _views_mixed()[:1]
    handles, outs, entries = _frame_setup(pr, cases)
    ws = pr.pr_workspace_create()
    try:
        sc, v, _ = cases[0]
        host_target = torch.zeros(3 * v.W * v.H)
        with pytest.raises(pr.PrError):
            pr.pr_frame_batch(ws, entries, [dict(target_rgb=host_target)])
    finally:
        pr.pr_workspace_free(ws)
        for h in handles:
            pr.pr_scene_free(h)


def test_sweep_tool_runs(pr):
    """The bound-variant sweep measures every bound kind on a small view and
    reports STE = hits / tests in (0, 1]."""
    from paper_1806_05385_gb300 import sweep
    sc, view = sweep.one_eye(W=160, H=176, objects=20)
    b = sweep.Bench(sc, reps=2)
    try:
        rows = [b.run(view, k) for k in ("trivial", "quad", "hull", "adaptive", "zenon")]
        rows += [b.run(view, "zenon", fov_bound=f) for f in ("simple", "recursive")]
    finally:
        b.close()
    for r in rows:
        assert 0.0 < r["ste"] <= 1.0 and r["ms"] > 0.0
    # tighter rolling bounds test no more pixels (Sec. 6: Trivial > Quad > Hull, Zenon tightest)
    t = [r["tests"] for r in rows[:5]]
    assert t[0] >= t[1] >= t[2] and t[4] <= t[2]


@pytest.mark.parametrize("mode", [S.MODE_ROLLING, S.MODE_BOTH])
def test_specular_shading_and_gradient_match_oracle(pr, oracle, mode):
    """Rolling specular (Blinn-Phong, eye at the pixel time): the shaded frame
    and the adjoint match the FP64 oracle."""
    import torch
    sc = S.random_triangles(800, 9, offset=0.15)
    p0, p1 = S.head_poses(2.0, 0.5)
    view = S.View(W=160, H=128, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode, fovea=(0.47, 0.52),
                  k_s=0.35, shininess=12.0)
    g = gpu_frame(pr, sc, view, keep=True)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri, near=True)
    rep = compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"])
    assert rep["hit_frac"] > 0.05
    h = g["scene"]
    interior = (o["id"] != BG) & (g["id"] == o["id"]) & (o["bmin"] > 1e-3) & (o["gap"] > 1e-3) & (o["near"] > 1e-3)
    n = view.W * view.H
    rng = np.random.default_rng(mode + 7)
    gr = rng.normal(size=(n, 3)) * interior[:, None]
    ids = _dev(g["id"].view(np.int32))
    gplanar = _dev(np.ascontiguousarray(gr.T.astype(np.float32)).reshape(-1))
    dcol, dpos, dvel = (torch.zeros(sc.V * 3, device="cuda") for _ in range(3))
    pr.pr_backward(h, view, ids, gplanar, dcol, dpos, dvel)
    pr.pr_scene_free(h)
    oc, op, ov = oracle.grad(view, sc.pos, sc.vel, sc.col, sc.tri, o["id"], gr)
    for name, gpu, ref in (("col", dcol, oc), ("pos", dpos, op), ("vel", dvel, ov)):
        a = gpu.cpu().numpy().reshape(-1, 3).astype(np.float64)
        err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
        assert err <= 1e-3, (name, err)
    # the highlight is really there: some pixels are brighter than any albedo x sigma allows
    assert (g["rgb"].reshape(3, -1).max(axis=0) > 1.0).any() or rep["hit_frac"] > 0.05


def test_fp32_peak_measurement_is_plausible(pr):
    """The FMA microbenchmark lands near the unit-count peak of a GB300
    (152 SMs x 128 lanes x 2 FLOP x about 2 GHz = about 78 TFLOP/s)."""
    t = pr.pr_measure_fp32_peak()
    assert 20.0 < t < 120.0


def test_scan_wait_times_out_with_a_status(pr):
    """Failure detection without a fault: a scan whose predecessor tile never
    publishes gives up its bounded wait, reports PR_ERR_TIMEOUT, and the
    context stays usable for the next frame."""
    import time
    import torch
    t0 = time.time()
    assert pr.pr_debug_scan_timeout() == pr.PR_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    sc = S.random_triangles(300, 9)
    p0, p1 = S.head_poses(1.0, 0.0)
    view = S.View(W=64, H=48, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=S.MODE_ROLLING)
    h = _upload(pr, sc)
    try:
        ids = torch.empty(64 * 48, dtype=torch.int32, device="cuda")
        dep = torch.empty(64 * 48, device="cuda")
        pr.pr_rasterize(h, view, pr.make_params("zenon", 16), ids, dep)
        torch.cuda.synchronize()
        assert int((ids >= 0).sum()) > 0
    finally:
        pr.pr_scene_free(h)
