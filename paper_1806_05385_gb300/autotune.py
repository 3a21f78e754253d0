"""Tile-size autotuner of the batched form.

For each view class -- mode, resolution bucket and triangle-count bucket --
it times the view's frame through the C ABI (pr_rasterize, CUDA events on the
current stream) for each bin tile size in {8, 16, 32}; the timings are cached
in a JSON file so that later runs reuse them.  A batch then takes one tile
size for all its views -- the one with the least summed time over them --
and a view class leaves it only for a tile that is faster by more than
`margin`: every tile size of a batch is a fragment launch of its own, whose
start and tail the per-view timings do not see, so near-ties are not worth
a split (on the 64-view workload, per-class fastest tiles gave a fragment
stage of 0.96-1.03 ms against 0.85 ms for 16 throughout).  Bin and
work-item capacities need no tuning: the library sizes them from the counts
a frame reports and regrows on overflow.
"""
from __future__ import annotations

import json
import math
import os

from . import binding as B

TILES = (8, 16, 32)


def default_cache_path() -> str:
    base = os.environ.get("PR_AUTOTUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                                 "paper_1806_05385_gb300")
    return base if base.endswith(".json") else os.path.join(base, "tiles.json")


def view_class(view, T: int) -> str:
    """Views that share mode, resolution bucket (x1.5 steps) and triangle
    bucket (x4 steps) share a tile size."""
    px = max(1, int(view.W) * int(view.H))
    return f"m{int(view.mode)}_p{int(math.log(px, 1.5))}_t{int(math.log(max(T, 1), 4))}"


def _load(path):
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    # Anything but a mapping of class -> {"tile": ...} is discarded.
    if not isinstance(data, dict):
        return {}
    return {k: e for k, e in data.items() if isinstance(e, dict) and e.get("tile") in TILES}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_tile(scene, view, tile: int, reps: int = 10, params=None) -> float:
    """Least device time (ms) of pr_rasterize for one view at one tile size
    over `reps` runs (the least is the run that other work disturbed least)."""
    import torch
    n = int(view.W) * int(view.H)
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    p = B.make_params(params.bound if params is not None else "zenon", tile,
                      params.fp64_retest if params is not None else 0, params.seg if params is not None else 0)
    st = torch.cuda.current_stream()
    B.pr_rasterize(scene, view, p, ids, None)  # warm-up (sizes the scratch)
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.pr_rasterize(scene, view, p, ids, None)
        e1.record(st)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return min(out)


def _times(entry):
    """The cached per-tile times of a class, or None if incomplete."""
    ms = entry.get("ms")
    if not isinstance(ms, dict):
        return None
    try:
        out = {t: float(ms[str(t)] if str(t) in ms else ms[t]) for t in TILES}
    except (KeyError, TypeError, ValueError):
        return None
    return out


def tune(cases, cache_path: str | None = None, reps: int = 10, refresh: bool = False, margin: float = 0.10):
    """cases: list of (scene_handle, view, T).  Returns one tile size per
    case: the batch's tile (least summed time over the cases), or a class's
    own fastest where that beats the batch's by more than `margin` (a
    fraction).  Cached classes are not re-timed unless refresh."""
    path = cache_path or default_cache_path()
    cache = {} if refresh else _load(path)
    changed = False
    per_case = []
    for scene, view, T in cases:
        key = view_class(view, T)
        times = _times(cache[key]) if key in cache else None
        if times is None:
            times = {t: time_tile(scene, view, t, reps) for t in TILES}
            cache[key] = {"tile": min(times, key=times.get), "ms": times}
            changed = True
        per_case.append(times)
    if changed:
        _save(path, cache)
    if not per_case:
        return []
    total = {t: sum(ms[t] for ms in per_case) for t in TILES}
    base = min(TILES, key=lambda t: (total[t], t != 16))
    tiles = []
    for ms in per_case:
        best = min(TILES, key=lambda t: ms[t])
        tiles.append(best if ms[best] < (1.0 - margin) * ms[base] else base)
    return tiles
