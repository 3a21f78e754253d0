"""The batched and graph-captured training frame -- the path the benchmark
times -- held directly to the FP64 oracle (Sec. 5.2: the result is that of
ray tracing every pixel at its own time; Sec. 3: testing all primitives
against all pixels is the correct, slow definition).

* a mixed batch of small views (every mode, ragged sizes, tiles 8/16/32):
  pr_frame_batch and a replay of pr_graph_capture_frame, every pixel of
  every view against the oracle, and the adjoint against the oracle
  gradient on interior pixels;
* a batch shaped like the 64-view workload that spans its extremes (8
  views, 1k to 500k triangles, sides 512 to 2160, every mode twice, tiles
  8/16/32): a replay of the captured training-frame graph on seeded pixel
  samples of every view (2^16 uniform pixels and four 64 x 64 windows; for
  views of more than 100k triangles 2^14 and four 32 x 32 windows, which
  keeps the oracle's share of the test near a minute), the adjoint on an
  interior subset, in the FP32 form and in the precision form (strict rule);
* the differentiable 512 x 512, 10k-triangle joint frame: full-frame forward
  parity and the gradient of its L2 loss against the oracle on interior
  pixels;
* the precision form on the large 1M-triangle frame under the strict rule.
"""
import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S
from tests.parity_util import BG, compare
from tests.test_batch_grad_gpu import _views_mixed
from tests.test_parity_gpu import gpu_frame

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _grad_rel_err(gpu, ref):
    a = gpu.cpu().numpy().reshape(-1, 3).astype(np.float64)
    return np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300)


class Batch:
    """Scenes uploaded, output buffers and zeroed gradient inputs/outputs for
    a list of (scene, view, tile)."""

    def __init__(self, pr, cases):
        import torch
        self.pr, self.cases = pr, cases
        self.h = [pr.pr_scene_upload(_dev(sc.pos), _dev(sc.vel), _dev(sc.col), _dev(sc.tri)) for sc, _, _ in cases]
        self.out, self.entries, self.gin, self.gout = [], [], [], []
        for h, (sc, v, tile) in zip(self.h, cases):
            n = v.W * v.H
            o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                 torch.empty(3 * n, device="cuda"))
            self.out.append(o)
            self.entries.append((h, v, o[0], o[1], o[2], tile))
            self.gin.append(torch.zeros(3 * n, device="cuda"))
            self.gout.append(tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3)))
        self.grads = [dict(grad_rgb=g, dcol=d[0], dpos=d[1], dvel=d[2]) for g, d in zip(self.gin, self.gout)]

    def host(self, k):
        o = self.out[k]
        return o[0].cpu().numpy().view(np.uint32), o[1].cpu().numpy(), o[2].cpu().numpy()

    def zero_grads(self):
        for d in self.gout:
            for x in d:
                x.zero_()

    def close(self):
        for h in self.h:
            self.pr.pr_scene_free(h)


def _interior(o, gid):
    return (o["id"] != BG) & (gid == o["id"]) & (o["bmin"] > 1e-3) & (o["gap"] > 1e-3) & (o["near"] > 1e-3)


def _check_forward(oracle, b, k, pix=None, fp64=False):
    sc, v, _ = b.cases[k]
    gid, gd, grgb = b.host(k)
    o = oracle.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix)
    return compare(oracle, v, sc, o, gid, gd, grgb, pix=pix, fp64=fp64)


def _grad_subset(oracle, b, k, pix, rng):
    """Interior pixels among pix, the oracle render there (with the occluder
    margins), and a random upstream gradient on them."""
    sc, v, _ = b.cases[k]
    gid = b.host(k)[0]
    o = oracle.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix, near=True)
    inner = _interior(o, gid[pix])
    g = rng.normal(size=(pix.size, 3)) * inner[:, None]
    return o, g, inner


def _set_upstream(b, k, pix, g):
    sc, v, _ = b.cases[k]
    n = v.W * v.H
    full = np.zeros((3, n), np.float32)
    full[:, pix] = g.T
    b.gin[k].copy_(_dev(full.reshape(-1)))


def _check_grads(oracle, b, k, pix, o, g):
    sc, v, _ = b.cases[k]
    oc, op, ov = oracle.grad(v, sc.pos, sc.vel, sc.col, sc.tri, o["id"], g, pix=pix)
    for name, gpu, ref in zip(("col", "pos", "vel"), b.gout[k], (oc, op, ov)):
        if name == "vel" and v.mode in (S.MODE_CLASSIC, S.MODE_FOVEATED):
            assert float(gpu.abs().max()) == 0.0    # t = 0: velocities do not act
            continue
        err = _grad_rel_err(gpu, ref)
        assert err <= 1e-3, (k, name, err)


def test_mixed_batch_frame_and_graph_match_oracle(pr, oracle):
    """pr_frame_batch and a replay of the training-frame graph on the mixed
    batch: every pixel of every view against the oracle, and the adjoint
    against the oracle gradient of the interior pixels."""
    import torch
    cases = _views_mixed()
    b = Batch(pr, cases)
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(7)
    try:
        with torch.cuda.stream(stream):
            pr.pr_frame_batch(ws, b.entries, b.grads)          # zero upstream gradients: forward only
            stream.synchronize()
            eager = [tuple(x.clone() for x in o) for o in b.out]
            for k in range(len(cases)):
                _check_forward(oracle, b, k)
            sub = []
            for k, (sc, v, _) in enumerate(cases):
                pix = np.arange(v.W * v.H)
                o, g, inner = _grad_subset(oracle, b, k, pix, rng)
                assert inner.mean() > 0.02, k
                _set_upstream(b, k, pix, g)
                sub.append((pix, o, g))
            graph = pr.pr_graph_capture_frame(ws, b.entries, b.grads)   # runs the frame once eagerly too
            for rep in range(2):
                b.zero_grads()
                for o in b.out:
                    for x in o:
                        x.fill_(5)
                pr.pr_graph_launch(graph)
                stream.synchronize()
                for o, r in zip(b.out, eager):
                    assert all(torch.equal(x, y) for x, y in zip(o, r))
                for k, (pix, o, g) in enumerate(sub):
                    _check_grads(oracle, b, k, pix, o, g)
            pr.pr_graph_free(graph)
    finally:
        pr.pr_workspace_free(ws)
        b.close()


def _span_sample(v, T, k):
    if T > 100_000:
        return S.sample_pixels(v.W, v.H, 1 << 14, 4, 32, 900 + k)
    return S.sample_pixels(v.W, v.H, 1 << 16, 4, 64, 900 + k)


@pytest.mark.parametrize("fp64", [0, 1])
def test_workload_shaped_batch_graph_matches_oracle(pr, oracle, fp64):
    """The captured training-frame graph (forward + adjoint in one replay,
    the benchmark's step) on a batch spanning the 64-view workload's
    extremes, against the oracle on seeded samples of every view; fp64 = 1
    runs the precision form and holds it to the strict rule."""
    import torch
    cases = S.config_batched_span(seed=4)
    assert {v.mode for _, v, _ in cases} == {0, 1, 2, 3} and {t for _, _, t in cases} == {8, 16, 32}
    assert min(sc.T for sc, _, _ in cases) == 1000 and max(sc.T for sc, _, _ in cases) == 500_000
    b = Batch(pr, cases)
    ws = pr.pr_workspace_create()
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(17)
    params = pr.make_params("zenon", 16, fp64)
    try:
        with torch.cuda.stream(stream):
            graph = pr.pr_graph_capture_frame(ws, b.entries, b.grads, params)
            for o in b.out:
                for x in o:
                    x.fill_(5)
            b.zero_grads()
            pr.pr_graph_launch(graph)                          # upstream gradients still zero
            stream.synchronize()
            if fp64:
                assert pr.pr_workspace_stats(ws)["flagged"] > 0
            sub = []
            for k, (sc, v, _) in enumerate(cases):
                pix = _span_sample(v, sc.T, k)
                rep = _check_forward(oracle, b, k, pix=pix, fp64=bool(fp64))
                assert rep["hit_frac"] > 0.01, (k, rep)
                gpix = np.sort(rng.choice(pix, size=min(2048, pix.size), replace=False))
                o, g, inner = _grad_subset(oracle, b, k, gpix, rng)
                assert inner.sum() > 20, k
                _set_upstream(b, k, gpix, g)
                sub.append((gpix, o, g))
            b.zero_grads()
            pr.pr_graph_launch(graph)
            stream.synchronize()
            for k, (gpix, o, g) in enumerate(sub):
                _check_grads(oracle, b, k, gpix, o, g)
            pr.pr_graph_free(graph)
    finally:
        pr.pr_workspace_free(ws)
        b.close()


@pytest.mark.parametrize("fp64", [0, 1])
def test_differentiable_frame_loss_gradient_matches_oracle(pr, oracle, fp64):
    """The differentiable workload at full size (512 x 512, 10k small
    triangles, joint mode): every pixel of the forward against the oracle,
    then the training frame's adjoint of the L2 loss against a target
    rendered by the oracle from parameters perturbed by N(0, 0.01): the
    upstream gradient 2 (rgb - target) of the oracle's own image on the
    interior pixels (zero elsewhere), the gradient against the oracle's."""
    import torch
    sc, view, tgt = S.config_diff(seed=5)
    n = view.W * view.H
    target = oracle.render(view, tgt.pos, tgt.vel, tgt.col, tgt.tri)["rgb"]
    b = Batch(pr, [(sc, view, 16)])
    ws = pr.pr_workspace_create()
    try:
        params = pr.make_params("zenon", 16, fp64)
        pr.pr_rasterize_batch(ws, b.entries, params)
        rep = _check_forward(oracle, b, 0, fp64=bool(fp64))
        assert rep["hit_frac"] > 0.3
        gid = b.host(0)[0]
        o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri, near=True)
        inner = _interior(o, gid)
        assert inner.mean() > 0.1
        g = 2.0 * (o["rgb"] - target) * inner[:, None]
        assert np.abs(g).max() > 1e-3
        _set_upstream(b, 0, np.arange(n), g)
        pr.pr_frame_batch(ws, b.entries, b.grads, params)
        torch.cuda.synchronize()
        _check_grads(oracle, b, 0, np.arange(n), o, g)
    finally:
        pr.pr_workspace_free(ws)
        b.close()


def test_large_frame_precision_form_strict(pr, oracle):
    """The 1M-triangle stereo frame in the precision form, under the strict
    rule, on a seeded sample of each eye."""
    sc, views = S.config_large(seed=3)
    for k, v in enumerate(views):
        g = gpu_frame(pr, sc, v, tile=32, fp64=1)
        pix = S.sample_pixels(v.W, v.H, 400, 1, 16, 700 + k)
        o = oracle.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix)
        rep = compare(oracle, v, sc, o, g["id"], g["depth"], g["rgb"], pix=pix, fp64=True)
        assert rep["hit_frac"] > 0.01 and g["stats"]["flagged"] > 0
