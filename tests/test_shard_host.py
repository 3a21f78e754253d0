"""Host logic of the view-sharded training frame (paper_1806_05385_gb300.shard)
on CPU: the pixel-balanced partition of the views, and two gloo ranks whose
one all-reduce of the flat per-vertex gradient buffer gives every rank the
single-process sum.  The per-view work here is a stand-in that adds a fixed
pattern per view into its scene's gradient slices (the library's training
frame runs on the GPU: tests/test_shard_gpu.py)."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1806_05385_gb300 import shard

SCENES = [5, 7, 3]
SCENE_OF = [0, 1, 0, 2, 1]
PIXELS = [100, 300, 50, 200, 80]


def _standin(mine, grads):
    """Adds (k + 1) * (index + 1) * 10^a to array a of view k's scene."""
    for k, (dc, dp, dv) in zip(mine, grads):
        for a, x in enumerate((dc, dp, dv)):
            x += (k + 1) * (torch.arange(x.numel(), dtype=torch.float32) + 1) * 10.0 ** a


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sf = shard.ShardedFrame(SCENES, SCENE_OF, PIXELS, rank, world)
    g = sf.step(_standin, dist)
    out[rank] = (sf.mine, g.numpy().copy())
    dist.destroy_process_group()


def test_partition_covers_every_view_once_and_balances_pixels():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 4, 8):
        w = rng.integers(1, 1000, size=23)
        parts = shard.partition(w, world)
        assert sorted(sum(parts, [])) == list(range(23))
        assert all(p == sorted(p) for p in parts)
        loads = [w[p].sum() for p in parts]
        assert max(loads) - w.sum() / world <= w.max()        # within one view of the even share
    assert sorted(sum(shard.partition([5, 5], 4), [])) == [0, 1]   # fewer views than ranks
    assert shard.partition([], 3) == [[], [], []]


def test_two_gloo_ranks_sum_to_the_single_process_gradient():
    port = 29700 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as m:   # no fork of a process that may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    ref = shard.ShardedFrame(SCENES, SCENE_OF, PIXELS, 0, 1)
    want = ref.step(_standin).numpy()
    assert sorted(res[0][0] + res[1][0]) == list(range(len(SCENE_OF)))
    assert res[0][0] and res[1][0]
    for r in (0, 1):
        assert np.array_equal(res[r][1], want)
    # the layout: scene s's dcol, dpos, dvel are consecutive [3 V] slices
    dc, dp, dv = ref.scene_grads(1)
    assert dc.numel() == dp.numel() == dv.numel() == 3 * SCENES[1]
    assert float(dp[0]) == pytest.approx(10.0 * (2 + 5))      # views 1 and 4 see scene 1
