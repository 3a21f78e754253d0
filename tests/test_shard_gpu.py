"""The view-sharded training frame on the GPU: two processes (gloo ranks)
each run the library's training frame on their share of the views of two
shared scenes, on their own buffers; after the one all-reduce of the flat
per-vertex gradient buffer both hold what a single process gets from all
views, up to the order of the float atomics.  No kernel of one rank waits
on the other: the collective runs on host copies."""
import os

import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S
from paper_1806_05385_gb300 import shard

pytestmark = pytest.mark.gpu


def _cases():
    """Two scenes, six views (four of scene 0, two of scene 1), mixed modes
    and sizes; upstream gradients seeded per view."""
    sc = [S.random_triangles(600, 61, offset=0.4), S.random_triangles(300, 62)]
    out = []
    for k, (s, mode, W, H) in enumerate([(0, S.MODE_BOTH, 96, 80), (0, S.MODE_ROLLING, 120, 64),
                                         (1, S.MODE_CLASSIC, 64, 64), (0, S.MODE_FOVEATED, 80, 96),
                                         (1, S.MODE_BOTH, 100, 72), (0, S.MODE_ROLLING, 72, 72)]):
        p0, p1 = S.head_poses(1.0 + 0.5 * k, 0.2 * k)
        out.append((s, S.View(W=W, H=H, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=mode,
                              fovea=(0.4 + 0.03 * k, 0.5))))
    return sc, out


def _run(rank, world, dist=None):
    import torch
    from paper_1806_05385_gb300 import binding as B
    B.load()
    scenes, cases = _cases()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    handles = [B.pr_scene_upload(dev(s.pos), dev(s.vel), dev(s.col), dev(s.tri)) for s in scenes]
    views = [v for _, v in cases]
    outs = [(torch.empty(v.W * v.H, dtype=torch.int32, device="cuda"), torch.empty(v.W * v.H, device="cuda"),
             torch.empty(3 * v.W * v.H, device="cuda")) for v in views]
    rng = np.random.default_rng(5)
    upstream = [dev(rng.normal(size=3 * v.W * v.H).astype(np.float32)) for v in views]
    ws = B.pr_workspace_create()
    try:
        sf = shard.ShardedFrame([s.V for s in scenes], [s for s, _ in cases], [v.W * v.H for v in views], rank,
                                world, device="cuda")
        frame = shard.library_frame(B, ws, [handles[s] for s, _ in cases], views, outs, upstream,
                                    [16, 8, 32, 16, 8, 16])
        g = sf.step(frame, dist)
        torch.cuda.synchronize()
        return sf.mine, g.cpu().numpy()
    finally:
        B.pr_workspace_free(ws)
        for h in handles:
            B.pr_scene_free(h)


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = _run(rank, world, dist)
    dist.destroy_process_group()


def test_two_ranks_sum_to_the_single_process_gradient(pr):
    import torch.multiprocessing as mp
    _, want = _run(0, 1)
    port = 29800 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as m:   # no fork of a process that may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert sorted(res[0][0] + res[1][0]) == list(range(6)) and res[0][0] and res[1][0]
    scale = float(np.abs(want).max())
    assert scale > 0
    for r in (0, 1):
        assert np.allclose(res[r][1], want, rtol=1e-4, atol=1e-5 * scale)
    assert np.array_equal(res[0][1], res[1][1])
