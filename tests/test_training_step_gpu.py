"""The training-step forms of the frame, on the GPU:

* the L2 loss against an 8-bit target image (target = value / 255): its
  gradient equals the float-target path with the same target, and the loss
  each view accumulates equals the FP64 oracle's sum over all pixels of
  (rgb - target)^2 (background counted with rgb = 0);
* a view with a gradient may leave its image unstored (rgb_out NULL);
* pr_scene_update is asynchronous: a non-finite value is reported by the
  next frame that reads the scene (PR_ERR_NONFINITE, its triangles culled),
  eagerly and through a captured graph, and a finite update clears it.
"""
import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S
from tests.test_batch_grad_gpu import _views_mixed

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _setup(pr, cases):
    import torch
    hs = [pr.pr_scene_upload(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri)) for sc, _, _ in cases]
    outs = [(torch.empty(v.W * v.H, dtype=torch.int32, device="cuda"), torch.empty(v.W * v.H, device="cuda"),
             torch.empty(3 * v.W * v.H, device="cuda")) for _, v, _ in cases]
    return hs, outs


def test_u8_target_loss_and_gradient(pr, oracle):
    import torch
    cases = _views_mixed()
    hs, outs = _setup(pr, cases)
    ws = pr.pr_workspace_create()
    rng = np.random.default_rng(23)
    try:
        u8 = [rng.integers(0, 256, size=3 * v.W * v.H, dtype=np.uint8) for _, v, _ in cases]
        loss = torch.zeros(len(cases), device="cuda")
        g8 = [dict(target_u8=_dev(t), loss=loss[k:k + 1], dcol=torch.zeros(3 * sc.V, device="cuda"),
                   dpos=torch.zeros(3 * sc.V, device="cuda"), dvel=torch.zeros(3 * sc.V, device="cuda"))
              for k, ((sc, v, _), t) in enumerate(zip(cases, u8))]
        ent = [(h, v, o[0], o[1], o[2], tile) for h, (_, v, tile), o in zip(hs, cases, outs)]
        pr.pr_frame_batch(ws, ent, g8)
        lossf = torch.zeros(len(cases), device="cuda")
        gf = [dict(target_rgb=_dev((t.astype(np.float32) / np.float32(255.0))), loss=lossf[k:k + 1],
                   dcol=torch.zeros(3 * sc.V, device="cuda"), dpos=torch.zeros(3 * sc.V, device="cuda"),
                   dvel=torch.zeros(3 * sc.V, device="cuda")) for k, ((sc, v, _), t) in enumerate(zip(cases, u8))]
        pr.pr_frame_batch(ws, ent, gf)
        torch.cuda.synchronize()
        for a, b in zip(g8, gf):
            for n in ("dcol", "dpos", "dvel"):
                y = b[n]
                assert torch.allclose(a[n], y, rtol=1e-4, atol=1e-5 * float(y.abs().max()) + 1e-12)
        assert torch.allclose(loss, lossf, rtol=1e-5)
        for k, (sc, v, _) in enumerate(cases):
            o = oracle.render(v, sc.pos, sc.vel, sc.col, sc.tri)
            tgt = (u8[k].astype(np.float64) / 255.0).reshape(3, -1).T
            want = float(((o["rgb"] - tgt) ** 2).sum())
            assert float(loss[k]) == pytest.approx(want, rel=1e-4), k
    finally:
        pr.pr_workspace_free(ws)
        for h in hs:
            pr.pr_scene_free(h)


def test_frame_without_stored_image(pr):
    """rgb_out NULL in a training frame: the same gradients and loss, and the
    ids and depths still written."""
    import torch
    cases = _views_mixed()[:3]
    hs, outs = _setup(pr, cases)
    ws = pr.pr_workspace_create()
    rng = np.random.default_rng(3)
    try:
        tg = [_dev(rng.integers(0, 256, size=3 * v.W * v.H, dtype=np.uint8)) for _, v, _ in cases]
        res = []
        for store in (True, False):
            loss = torch.zeros(len(cases), device="cuda")
            g = [dict(target_u8=t, loss=loss[k:k + 1], dpos=torch.zeros(3 * sc.V, device="cuda"))
                 for k, ((sc, _, _), t) in enumerate(zip(cases, tg))]
            ids = [torch.full((v.W * v.H,), -7, dtype=torch.int32, device="cuda") for _, v, _ in cases]
            ent = [(h, v, i, o[1], o[2] if store else None, tile) for h, (_, v, tile), o, i in zip(hs, cases, outs, ids)]
            pr.pr_frame_batch(ws, ent, g)
            torch.cuda.synchronize()
            res.append((loss.clone(), [x["dpos"].clone() for x in g], [i.clone() for i in ids]))
        assert torch.allclose(res[0][0], res[1][0], rtol=1e-5)
        for a, b in zip(res[0][1], res[1][1]):
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()) + 1e-12)
        for a, b in zip(res[0][2], res[1][2]):
            assert torch.equal(a, b) and int((a >= 0).sum()) > 0
    finally:
        pr.pr_workspace_free(ws)
        for h in hs:
            pr.pr_scene_free(h)


def test_gradient_sources_are_exclusive(pr):
    import torch
    cases = _views_mixed()[:1]
    hs, outs = _setup(pr, cases)
    ws = pr.pr_workspace_create()
    try:
        sc, v, tile = cases[0]
        n = v.W * v.H
        ent = [(hs[0], v, outs[0][0], outs[0][1], outs[0][2], tile)]
        both = dict(grad_rgb=torch.zeros(3 * n, device="cuda"), target_u8=torch.zeros(3 * n, dtype=torch.uint8,
                                                                                      device="cuda"))
        with pytest.raises(pr.PrError) as e:
            pr.pr_frame_batch(ws, ent, [both])
        assert e.value.status == pr.PR_ERR_INVALID_ARG
        with pytest.raises(pr.PrError) as e:   # a loss needs a target
            pr.pr_frame_batch(ws, ent, [dict(grad_rgb=torch.zeros(3 * n, device="cuda"),
                                             loss=torch.zeros(1, device="cuda"))])
        assert e.value.status == pr.PR_ERR_INVALID_ARG
    finally:
        pr.pr_workspace_free(ws)
        pr.pr_scene_free(hs[0])


def test_nonfinite_update_is_reported_by_the_next_frame(pr):
    import torch
    sc = S.random_triangles(500, 31)
    p0, p1 = S.head_poses(1.0, 0.0)
    view = S.View(W=96, H=72, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=S.MODE_ROLLING)
    h = pr.pr_scene_upload(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri))
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    try:
        n = view.W * view.H
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        dep = torch.empty(n, device="cuda")
        pr.pr_rasterize(h, view, None, ids, dep)
        ref = ids.clone()
        bad = sc.pos.copy()
        bad[7, 2] = np.inf
        pr.pr_scene_update(h, _dev(bad), None, None)          # returns at once
        with pytest.raises(pr.PrError) as e:
            pr.pr_rasterize(h, view, None, ids, dep)
        assert e.value.status == pr.PR_ERR_NONFINITE
        assert bool((ids == -1).all())                        # every triangle of the scene culled
        pr.pr_scene_update(h, _dev(sc.pos), None, None)
        pr.pr_rasterize(h, view, None, ids, dep)
        assert torch.equal(ids, ref)
        # through a captured graph: the replay after a bad update reports it
        with torch.cuda.stream(stream):
            rgb = torch.empty(3 * n, device="cuda")
            graph = pr.pr_graph_capture_batch(ws, [(h, view, ids, dep, rgb, 16)])
            pr.pr_scene_update(h, _dev(bad), None, None)
            with pytest.raises(pr.PrError) as e:
                pr.pr_graph_launch(graph)
            assert e.value.status == pr.PR_ERR_NONFINITE
            pr.pr_scene_update(h, _dev(sc.pos), None, None)
            pr.pr_graph_launch(graph)
            assert torch.equal(ids, ref)
            pr.pr_graph_free(graph)
    finally:
        pr.pr_workspace_free(ws)
        pr.pr_scene_free(h)


def test_scene_update_batch_equals_fresh_uploads(pr):
    """pr_scene_update_batch steps several scenes in one call: each frame
    equals the frame of a scene uploaded with the new arrays; an entry left
    None keeps that array; a non-finite entry is reported only by the next
    frame of its own scene."""
    import torch
    rng = np.random.default_rng(8)
    base = [S.random_triangles(300 + 100 * k, 50 + k) for k in range(3)]
    new = [S.Scene((sc.pos + rng.normal(0, 0.05, sc.pos.shape)).astype(np.float32),
                   (sc.vel + rng.normal(0, 0.01, sc.vel.shape)).astype(np.float32),
                   rng.uniform(0, 1, sc.col.shape).astype(np.float32), sc.tri) for sc in base]
    p0, p1 = S.head_poses(1.5, 0.2)
    view = S.View(W=80, H=64, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=S.MODE_BOTH, fovea=(0.4, 0.6))
    hs = [pr.pr_scene_upload(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri)) for sc in base]
    try:
        keep_vel = [_dev(nw.vel) for nw in new]
        keep_vel[1] = None                                   # scene 1 keeps its velocities
        pr.pr_scene_update_batch(hs, [_dev(nw.pos) for nw in new], keep_vel, [_dev(nw.col) for nw in new])
        n = view.W * view.H
        for k, (h, nw, sc) in enumerate(zip(hs, new, base)):
            ids, dep, rgb = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                             torch.empty(3 * n, device="cuda"))
            pr.pr_rasterize(h, view, None, ids, dep)
            pr.pr_shade(h, view, ids, rgb)
            want = S.Scene(nw.pos, sc.vel if k == 1 else nw.vel, nw.col, nw.tri)
            h2 = pr.pr_scene_upload(_dev(want.pos), _dev(want.vel), _dev(want.col), _dev(want.tri))
            ids2, dep2, rgb2 = torch.empty_like(ids), torch.empty_like(dep), torch.empty_like(rgb)
            pr.pr_rasterize(h2, view, None, ids2, dep2)
            pr.pr_shade(h2, view, ids2, rgb2)
            pr.pr_scene_free(h2)
            assert torch.equal(ids, ids2) and torch.equal(dep, dep2) and torch.equal(rgb, rgb2), k
        bad = new[2].col.copy()
        bad[3, 0] = np.nan
        pr.pr_scene_update_batch(hs, None, None, [None, None, _dev(bad)])
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        pr.pr_rasterize(hs[0], view, None, ids, None)        # untouched scene: fine
        with pytest.raises(pr.PrError) as e:
            pr.pr_rasterize(hs[2], view, None, ids, None)
        assert e.value.status == pr.PR_ERR_NONFINITE
        with pytest.raises(pr.PrError):
            pr.pr_scene_update_batch(hs, [new[0].pos, None, None], None, None)   # a host array
    finally:
        for h in hs:
            pr.pr_scene_free(h)
