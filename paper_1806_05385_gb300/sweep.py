"""Bound-variant and scalability sweeps of the rasterizer (the evaluation of
Sec. 6: Tables 1-2 and the scalability plots), on the seeded synthetic HMD
scene instead of the paper's named scenes.

For every configuration it renders one view through the C ABI and reports
the raster time (stages a-c: bound, binning, fragment; median of CUDA-event
timings on the current stream), the stage times, the number of bin entries
and ray-triangle tests, and the sample test efficiency STE = hits / tests
(Sec. 6, "Sample Test Efficiency": the share of tested pixels that belong
to the primitive).  Sweeps:

* ``bounds``: Trivial / Quad / Hull / Adaptive / Zenon (Sec. 4.2) in rolling
  and joint mode, and the foveation bounds Sector / Simple / Recursive
  (Sec. 4.1) in foveated and joint mode, on a 720x800 eye with 50 objects
  (the Trivial bound puts every triangle in every tile);
* ``resolution``: framebuffer size, classic vs rolling vs joint;
* ``rotation``: head yaw during the frame (the transformation during
  scan-out), classic vs rolling;
* ``alpha``: foveation strength of p(d) = D (d/D)^alpha.

    python -m paper_1806_05385_gb300.sweep [--sweeps bounds,resolution,...] [--reps N] [--out file.md]
"""
from __future__ import annotations

import argparse
import json
import statistics

from . import binding as B
from . import scenes as S

MODE_NAMES = {S.MODE_CLASSIC: "classic", S.MODE_ROLLING: "rolling", S.MODE_FOVEATED: "foveated",
              S.MODE_BOTH: "joint"}


class Bench:
    """One uploaded scene; renders views and times them."""

    def __init__(self, sc, reps: int = 7):
        import torch
        self.torch = torch
        dev = lambda a: torch.from_numpy(a).cuda()
        self.sc = sc
        self.h = B.pr_scene_upload(dev(sc.pos), dev(sc.vel), dev(sc.col), dev(sc.tri))
        self.reps = reps

    def run(self, view, bound="zenon", tile=16, fov_bound="sector"):
        try:
            return self._run(view, bound, tile, fov_bound)
        except B.PrError as e:  # e.g. more bin entries than one frame may hold
            return {"ms": None, "error": str(e)}

    def _run(self, view, bound, tile, fov_bound):
        torch = self.torch
        n = view.W * view.H
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        depth = torch.empty(n, dtype=torch.float32, device="cuda")
        p = B.make_params(bound, tile, 0, 0, fov_bound=fov_bound)
        st = torch.cuda.current_stream()
        B.pr_rasterize(self.h, view, p, ids, depth)  # sizes the scratch
        times, stages = [], []
        for _ in range(self.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            B.pr_rasterize(self.h, view, p, ids, depth)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stages.append(B.pr_scene_stats(self.h)["stage_ms"])
        s = B.pr_scene_stats(self.h)
        med = lambda k: statistics.median(x[k] for x in stages)
        return {"ms": statistics.median(times), "bound_ms": med(0), "bin_ms": med(1), "fragment_ms": med(2),
                "pairs": s["pairs"], "tests": s["tests"], "hits": s["hits"],
                "ste": s["hits"] / s["tests"] if s["tests"] else None, "pixels": n}

    def close(self):
        B.pr_scene_free(self.h)


def one_eye(W=1440, H=1600, yaw=3.0, pitch=1.0, mode=S.MODE_BOTH, alpha=2.0, seed=2, objects=200):
    """The first eye of the stereo HMD scene (scenes.config_hmd) with its
    resolution, head motion, mode or foveation strength replaced."""
    sc, views = S.config_hmd(seed=seed, W=W, H=H, n_objects=objects)
    v = views[0]
    p0, p1 = S.head_poses(yaw, pitch, -0.032)
    return sc, S.View(W=W, H=H, tan_x=v.tan_x, tan_y=v.tan_y, pose0=p0, pose1=p1, mode=mode, fovea=v.fovea,
                      alpha=alpha)


BOUNDS_VIEW = dict(W=720, H=800, objects=50)  # small enough for the Trivial bound's every-tile bins


def sweep_bounds(reps):
    sc, _ = one_eye(**BOUNDS_VIEW)
    b = Bench(sc, reps)
    rows = []
    for mode in (S.MODE_ROLLING, S.MODE_BOTH):
        _, view = one_eye(mode=mode, **BOUNDS_VIEW)
        for kind in ("trivial", "quad", "hull", "adaptive", "zenon"):
            rows.append(dict(sweep="bounds", mode=MODE_NAMES[mode], bound=kind, fov_bound="sector",
                             **b.run(view, kind)))
    for mode in (S.MODE_FOVEATED, S.MODE_BOTH):
        _, view = one_eye(mode=mode, **BOUNDS_VIEW)
        for fb in ("sector", "simple", "recursive"):
            rows.append(dict(sweep="bounds", mode=MODE_NAMES[mode], bound="zenon", fov_bound=fb,
                             **b.run(view, "zenon", fov_bound=fb)))
    b.close()
    return rows


def sweep_resolution(reps):
    rows = []
    sc, _ = one_eye()
    b = Bench(sc, reps)
    for side in (512, 1024, 1440, 2048, 2880):
        for mode in (S.MODE_CLASSIC, S.MODE_ROLLING, S.MODE_BOTH):
            _, view = one_eye(W=side, H=side, mode=mode)
            rows.append(dict(sweep="resolution", side=side, mode=MODE_NAMES[mode], **b.run(view)))
    b.close()
    return rows


def sweep_rotation(reps):
    rows = []
    sc, _ = one_eye()
    b = Bench(sc, reps)
    for yaw in (0.0, 1.0, 2.0, 4.0, 8.0, 16.0):
        for mode in (S.MODE_CLASSIC, S.MODE_ROLLING):
            _, view = one_eye(yaw=yaw, pitch=0.0, mode=mode)
            rows.append(dict(sweep="rotation", yaw_deg=yaw, mode=MODE_NAMES[mode], **b.run(view)))
    b.close()
    return rows


def sweep_alpha(reps):
    rows = []
    sc, _ = one_eye()
    b = Bench(sc, reps)
    for alpha in (1.0, 1.5, 2.0, 2.5, 3.0, 4.0):
        _, view = one_eye(mode=S.MODE_FOVEATED, alpha=alpha)
        rows.append(dict(sweep="alpha", alpha=alpha, mode="foveated", **b.run(view)))
    b.close()
    return rows


SWEEPS = {"bounds": sweep_bounds, "resolution": sweep_resolution, "rotation": sweep_rotation, "alpha": sweep_alpha}


def to_markdown(rows):
    out = []
    for name in SWEEPS:
        rs = [r for r in rows if r["sweep"] == name]
        if not rs:
            continue
        keys = []
        for r in rs:
            keys += [k for k in r if k not in ("sweep", "pixels", "hits") and k not in keys]
        out.append(f"### {name}\n")
        out.append("| " + " | ".join(keys) + " |")
        out.append("|" + "---|" * len(keys))
        for r in rs:
            cells = []
            for k in keys:
                x = r.get(k, "")
                if x is None:
                    cells.append("-")
                elif isinstance(x, float):
                    cells.append(f"{100 * x:.1f} %" if k == "ste" else f"{x:.3f}")
                else:
                    cells.append(str(x))
            out.append("| " + " | ".join(cells) + " |")
        out.append("")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--sweeps", default=",".join(SWEEPS))
    ap.add_argument("--reps", type=int, default=7)
    ap.add_argument("--out", default=None, help="also write the tables as markdown")
    args = ap.parse_args(argv)
    names = [n for n in args.sweeps.split(",") if n]
    unknown = [n for n in names if n not in SWEEPS]
    if unknown or not names:
        ap.error(f"--sweeps: unknown {unknown}; choose from {', '.join(SWEEPS)}")
    import torch
    torch.cuda.set_device(0)
    B.load()
    rows = []
    for name in names:
        for r in SWEEPS[name](args.reps):
            print(json.dumps(r), flush=True)
            rows.append(r)
    if args.out:
        with open(args.out, "w") as f:
            f.write(to_markdown(rows))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
