#!/usr/bin/env python
"""Benchmark of the perceptual-rasterization hot path on GB300.

One step = one stereo HMD frame through every stage of the path: the
batched, graph-captured forward (a) bounds -> (b) binning -> (c) per-fragment
ray casting -> (d) shading for both eyes, then (e) the adjoint of the shaded
image for both eyes.  value = framebuffer pixels / step time (Mpix/s).

Prints ONE JSON line (rank 0).  Default workload: 1440x1600 per eye x 2
eyes, 266k triangles (200 subdivision-3 icospheres + a 10k ground plane),
joint foveated + rolling, seeded synthetic scene already resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1806_05385_gb300 import scenes as S  # noqa: E402

# FP32 operations of one watertight test in k_fragment's ray_test, counted
# from the source: 15 FMA (vertex interpolation to the pixel time: 9, shear:
# 6) = 30 FLOP, plus 6 multiplies and 3 subtractions for the edge functions.
FLOP_PER_TEST = 39
SMS = 152
FP32_LANES = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload():
    sc, views = S.config_hmd(seed=2)
    name = (f"hmd-stereo {views[0].W}x{views[0].H}x2 eyes, {sc.T} tris (200 ico-sub3 + 10k ground), "
            f"foveated+rolling (alpha 2, d=(1,0)), yaw 3deg pitch 1deg, zenon bound, tile 16")
    return sc, views, name


# ---------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])
        self.th = threading.Thread(target=rd, daemon=True)
        self.th.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nme in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- reference arm

def cpu_oracle_sample(sc, views, seconds: float, seed: int = 11):
    """Time the FP64 oracle (forward render + shade + gradient) on a seeded
    pixel sample of the stereo frame, sized to about `seconds` of work."""
    from oracle import oracle as O
    O.build()
    rng = np.random.default_rng(seed)

    def run(n):
        t0 = time.perf_counter()
        tests = 0
        for v in views:
            pix = np.sort(rng.choice(v.W * v.H, size=n // len(views), replace=False))
            o = O.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix)
            g = np.ones((pix.size, 3))
            O.grad(v, sc.pos, sc.vel, sc.col, sc.tri, o["id"], g, pix=pix)
            tests += pix.size * sc.T
        return time.perf_counter() - t0, tests

    dt, _ = run(256)
    n = int(max(256, min(1 << 16, 256 * seconds / max(dt, 1e-3))))
    n -= n % len(views)
    dt, tests = run(n)
    return {"pixels": n, "seconds": dt, "tests": tests, "cores": O.num_threads()}


def reference_arm(args, rank, world):
    sc, views, name = workload()
    if rank != 0:
        return 0
    cpu_s = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(sc, views, cpu_s / 4)
    runs = [cpu_oracle_sample(sc, views, cpu_s) for _ in range(args.steps)]
    px = sum(r["pixels"] for r in runs)
    sec = sum(r["seconds"] for r in runs)
    val = px / sec / 1e6
    line = {"metric": "Mpix/s & ray-tri tests/s at 1 GB300 (batched vs plain); fwd+bwd ms/frame",
            "value": val, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": name, "sample": f"{runs[0]['pixels']} pixels per step, all triangles each"},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": runs[0]["cores"], "kind": "oracle",
                             "sample": f"{runs[0]['pixels']} seeded pixels of the stereo frame per step, "
                                       f"forward + gradient, every triangle tested"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "tests_per_s": sum(r["tests"] for r in runs) / sec}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- our arm

def source_hash():
    p = os.path.join(ROOT, "paper_1806_05385_gb300", "csrc", "pr_stage_c.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per fragment launch from the committed ncu summary, only
    if it was taken on the current fragment-kernel source."""
    p = os.path.join(ROOT, "profiles", "fragment_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("source_sha256_16") != source_hash():
        return None
    return d.get("dram_bytes_per_launch")


def our_arm(args, rank, world):
    import torch
    from paper_1806_05385_gb300 import binding as B

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.load()
    sc, views, name = workload()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    stream = torch.cuda.Stream()          # a capturable stream for the forward graph
    torch.cuda.set_stream(stream)
    h = B.pr_scene_upload(dev(sc.pos), dev(sc.vel), dev(sc.col), dev(sc.tri))
    ws = B.pr_workspace_create()
    npx = [v.W * v.H for v in views]
    ids = [torch.empty(n, dtype=torch.int32, device="cuda") for n in npx]
    depth = [torch.empty(n, dtype=torch.float32, device="cuda") for n in npx]
    rgb = [torch.empty(3 * n, dtype=torch.float32, device="cuda") for n in npx]
    gen = torch.Generator(device="cuda").manual_seed(1234)
    grad = [torch.randn(3 * n, device="cuda", generator=gen) for n in npx]
    V = sc.V
    dcol, dpos, dvel = (torch.zeros(3 * V, device="cuda") for _ in range(3))
    params = B.make_params("zenon", 16, 0, 0)
    entries = [(h, v, ids[k], depth[k], rgb[k]) for k, v in enumerate(views)]
    graph = B.pr_graph_capture_batch(ws, entries, params)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def backward():
        for k, v in enumerate(views):
            B.pr_backward(h, v, ids[k], grad[k], dcol, dpos, dvel)

    def step():
        B.pr_graph_launch(graph)
        backward()

    def timed(fn, k, flush_l2=True):
        ms = []
        for _ in range(k):
            if flush_l2:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    step_ms = timed(step, args.steps)
    clocks = clk.stop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = B.pr_workspace_stats(ws)
    frag_ms = st["stage_ms"][2]

    # forward only: batched graph vs plain per-view calls
    fwd_batched = timed(lambda: B.pr_graph_launch(graph), args.steps)

    def plain():
        for k, v in enumerate(views):
            B.pr_rasterize(h, v, params, ids[k], depth[k])
            B.pr_shade(h, v, ids[k], rgb[k])
    for _ in range(3):
        plain()
    fwd_plain = timed(plain, args.steps)
    bwd_ms = timed(backward, args.steps)

    total_ms = sum(step_ms)
    mean_ms = total_ms / len(step_ms)
    if dist:
        t = torch.tensor([mean_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = float(t.item())
    pix = sum(npx)
    value = world * pix / (mean_ms * 1e-3) / 1e6

    # end to end through the C ABI with host buffers: scene arrays in from
    # pinned host memory, shaded images and gradients back to pinned host
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hpos, hvel, hcol = pin(sc.pos), pin(sc.vel), pin(sc.col)
        hrgb = [torch.empty(3 * n, dtype=torch.float32).pin_memory() for n in npx]
        hg = [g.cpu().pin_memory() for g in grad]
        hd = [torch.zeros(3 * V).pin_memory() for _ in range(3)]
        ent_h = [(h, v, ids[k], None, hrgb[k]) for k, v in enumerate(views)]

        def e2e_step():
            B.pr_scene_update(h, hpos, hvel, hcol)
            B.pr_rasterize_batch(ws, ent_h, params)
            for k, v in enumerate(views):
                B.pr_backward(h, v, ids[k], hg[k], hd[0], hd[1], hd[2])
        for _ in range(2):
            e2e_step()
        ems = timed(e2e_step, max(3, args.steps // 2))
        h2d = 3 * V * 12 + sum(g.numel() * 4 for g in hg) + 3 * (3 * V * 4)
        d2h = sum(x.numel() * 4 for x in hrgb) + 3 * (3 * V * 4)
        e2e = {"value": world * pix / (statistics.mean(ems) * 1e-3) / 1e6, "unit": "Mpix/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # roofline of the dominant kernel (stage c, FP32 ALU bound)
    sm_mhz = clocks.get("sm_mhz") or 1470.0
    peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    achieved = st["tests"] * FLOP_PER_TEST / (frag_ms * 1e-3) / 1e12 if frag_ms > 0 else 0.0
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "traffic": ncu_traffic(),
            "kernel": "k_fragment<16>", "flop_per_test": FLOP_PER_TEST,
            "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 FLOP x median SM clock {sm_mhz:.0f} MHz "
                          f"sampled during the timed region"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r = cpu_oracle_sample(sc, views, args.cpu_seconds)
        cpu = {"value": r["pixels"] / r["seconds"] / 1e6, "unit": "Mpix/s", "cores": r["cores"], "kind": "oracle",
               "sample": f"{r['pixels']} seeded pixels of the stereo frame, FP64 forward + gradient, "
                         f"every triangle tested ({r['tests']:.3g} tests in {r['seconds']:.1f} s)",
               "tests_per_s": r["tests"] / r["seconds"]}

    kernels_per_step = 11 + len(views)   # forward graph (11 kernels) + one adjoint per eye
    line = {
        "metric": "Mpix/s & ray-tri tests/s at 1 GB300 (batched vs plain); fwd+bwd ms/frame",
        "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": name, "views": len(views), "pixels_per_step": pix, "triangles": sc.T,
                   "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": kernels_per_step * args.steps,
        "tests_per_s": st["tests"] / (frag_ms * 1e-3) if frag_ms > 0 else None,
        "ste": st["hits"] / st["tests"] if st["tests"] else None,
        "stats": {k: st[k] for k in ("tests", "hits", "pairs", "items", "culled", "pixels")},
        "stage_ms": {"bound": st["stage_ms"][0], "bin": st["stage_ms"][1], "fragment": frag_ms,
                     "resolve": st["stage_ms"][4], "shade": st["stage_ms"][5]},
        "fwd_mpix_s": {"batched_graph": world * pix / (statistics.mean(fwd_batched) * 1e-3) / 1e6,
                       "plain_per_view": world * pix / (statistics.mean(fwd_plain) * 1e-3) / 1e6},
        "fwd_bwd_ms_per_frame": mean_ms, "bwd_ms_per_frame": statistics.mean(bwd_ms),
    }
    B.pr_graph_free(graph)
    B.pr_workspace_free(ws)
    B.pr_scene_free(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    return our_arm(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
