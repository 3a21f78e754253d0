"""View-sharded training frame over several processes (one per GPU).

Every pixel's result depends only on its own time, ray and the scene
(Sec. 3.2, "Intersection": each pixel's hit is comparable because it has a
unique time and ray), so the views of a training frame split across ranks
with no exchange in the forward.  The adjoint of each rank's views adds
into per-vertex gradients of scenes that other ranks' views may also see;
one all-reduce (sum) of every scene's 9 FP32 values per vertex (colour,
position, velocity gradients) makes the full gradient on every rank.

Layout: one flat FP32 buffer holds, scene after scene, dcol [V][3], dpos
[V][3], dvel [V][3]; a single collective reduces all of it.  With NCCL it
is reduced in place on the device; with gloo through a host copy.

The per-rank work is a callable, so the partition and the reduction are
plain host logic: ``ShardedFrame.step`` takes ``frame(views, grads)``, which
must ADD the gradients of the listed views into the given per-scene slices
(``library_frame`` builds the one that runs the library's training frame).
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def partition(weights: Sequence[float], world: int) -> list[list[int]]:
    """Contiguous split of the items (views) over ``world`` ranks with
    balanced total weight (pixel count): rank r gets the items whose weight
    midpoint falls in its share [r, r + 1) * total / world.  Every item goes
    to exactly one rank; a rank may get none when there are fewer items than
    ranks."""
    w = np.asarray(weights, dtype=np.float64)
    if w.size == 0:
        return [[] for _ in range(world)]
    total = float(w.sum())
    mid = np.cumsum(w) - 0.5 * w
    owner = np.minimum((mid * world / max(total, 1e-300)).astype(np.int64), world - 1)
    return [np.nonzero(owner == r)[0].tolist() for r in range(world)]


class ShardedFrame:
    """The gradient buffer of a set of scenes and the view partition of one
    rank.  scene_sizes: V of every scene; scene_of[k]: scene of view k;
    pixels[k]: its pixel count (the partition's weight)."""

    def __init__(self, scene_sizes: Sequence[int], scene_of: Sequence[int], pixels: Sequence[int], rank: int,
                 world: int, device="cpu"):
        import torch
        self.rank, self.world = rank, world
        self.scene_of = list(scene_of)
        self.parts = partition(pixels, world)
        self.mine = self.parts[rank]
        self.offsets = np.concatenate([[0], np.cumsum([9 * int(v) for v in scene_sizes])]).astype(np.int64)
        self.grad = torch.zeros(int(self.offsets[-1]), dtype=torch.float32, device=device)
        self.sizes = [int(v) for v in scene_sizes]

    def scene_grads(self, s: int):
        """(dcol, dpos, dvel) of scene s: [3 V] views into the flat buffer."""
        o, V = int(self.offsets[s]), self.sizes[s]
        g = self.grad
        return g[o:o + 3 * V], g[o + 3 * V:o + 6 * V], g[o + 6 * V:o + 9 * V]

    def step(self, frame: Callable, dist=None):
        """Zero the gradients, run ``frame`` on this rank's views, and sum
        the gradients over the ranks (one all-reduce).  Returns the flat
        gradient buffer, equal on every rank."""
        self.grad.zero_()
        if self.mine:
            frame(self.mine, [self.scene_grads(self.scene_of[k]) for k in self.mine])
        if dist is not None and self.world > 1:
            if dist.get_backend() == "nccl" or self.grad.device.type == "cpu":
                dist.all_reduce(self.grad, op=dist.ReduceOp.SUM)
            else:  # gloo: through the host
                h = self.grad.cpu()
                dist.all_reduce(h, op=dist.ReduceOp.SUM)
                self.grad.copy_(h)
        return self.grad


def library_frame(B, ws, handles, views, outputs, upstream, tiles, params=None):
    """The per-rank work of a sharded step through the library: one
    pr_frame_batch over the listed views (batched forward, then the adjoint
    of each view's upstream image gradient, accumulated into the given
    gradient slices).  handles[k], views[k], outputs[k] = (id, depth, rgb),
    upstream[k] = dL/drgb [3][H][W] and tiles[k] describe view k of the
    whole frame."""
    def frame(mine, grads):
        entries = [(handles[k], views[k], *outputs[k], tiles[k]) for k in mine]
        g = [dict(grad_rgb=upstream[k], dcol=d[0], dpos=d[1], dvel=d[2]) for k, d in zip(mine, grads)]
        B.pr_frame_batch(ws, entries, g, params)
    return frame
