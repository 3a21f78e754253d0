#!/usr/bin/env python
"""Benchmark of the perceptual-rasterization hot path on GB300.

One step = one training frame of the workload through every stage of the
path, captured as one CUDA graph: (a) bounds -> (b) binning and the depth
sort of every work item's run -> (c) per-fragment ray casting -> (d)
shading for all views, with (e) the adjoint of an upstream image gradient
for every view in the same kernel.  value = framebuffer pixels / step time
(Mpix/s).

Prints ONE JSON line (rank 0).  Default workload: 1440x1600 per eye x 2
eyes, 266k triangles (200 subdivision-3 icospheres + a 10k ground plane),
joint foveated + rolling, seeded synthetic scene already resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload hmd|large|batched|diff]
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
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["hmd", "large", "batched", "diff"], default="hmd",
                    help="hmd: stereo 1440x1600, 266k tris (default); large: stereo 2160^2, 1M tris, FP64 "
                         "re-test; batched: 64 views of 1k-500k tris; diff: 512^2, 10k tris")
    return ap.parse_args()


class Workload:
    """Scenes, views (each naming its scene), the FP64 re-test switch and a name."""

    def __init__(self, scenes, views, scene_of, fp64, name):
        self.scenes, self.views, self.scene_of, self.fp64, self.name = scenes, views, scene_of, fp64, name


def workload(kind: str = "hmd") -> Workload:
    if kind == "hmd":
        sc, views = S.config_hmd(seed=2)
        name = (f"hmd-stereo {views[0].W}x{views[0].H}x2 eyes, {sc.T} tris (200 ico-sub3 + 10k ground), "
                f"foveated+rolling (alpha 2, d=(1,0)), yaw 3deg pitch 1deg, zenon bound, tile 16")
        return Workload([sc], views, [0, 0], 0, name)
    if kind == "large":
        sc, views = S.config_large(seed=3)
        name = (f"large-stereo {views[0].W}x{views[0].H}x2 eyes, {sc.T} tris (ico-sub2/box instances, sizes "
                f"1e-3..1, half moving), foveated+rolling, FP64 re-test of flagged fragments")
        return Workload([sc], views, [0, 0], 1, name)
    if kind == "batched":
        pairs = S.config_batched(seed=4)
        scenes = [p[0] for p in pairs]
        views = [p[1] for p in pairs]
        name = (f"batched {len(views)} views, {sum(x.T for x in scenes)} tris (1k..500k log-uniform), "
                f"{sum(v.W * v.H for v in views) / 1e6:.1f} Mpx (512^2..2160^2), mixed modes, autotuned tiles")
        return Workload(scenes, views, list(range(len(views))), 0, name)
    sc, view, _ = S.config_diff(seed=5)
    name = f"diff {view.W}x{view.H}, {sc.T} small tris, foveated+rolling, fwd + bwd (colours, positions, velocities)"
    return Workload([sc], [view], [0], 0, name)


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

def cpu_oracle_sample(wl: Workload, seconds: float, seed: int = 11, pixels: int = 0):
    """Time the FP64 oracle (forward render + shade + gradient, every
    triangle of the view's scene tested per pixel) on a seeded pixel sample
    spread over the workload's views, sized to about `seconds` of work (or
    of `pixels` pixels when given, without the sizing runs)."""
    from oracle import oracle as O
    O.build()
    rng = np.random.default_rng(seed)

    def run(n):
        t0 = time.perf_counter()
        tests = 0
        per = max(1, n // len(wl.views))
        for v, si in zip(wl.views, wl.scene_of):
            sc = wl.scenes[si]
            pix = np.sort(rng.choice(v.W * v.H, size=min(per, v.W * v.H), replace=False))
            o = O.render(v, sc.pos, sc.vel, sc.col, sc.tri, pix=pix)
            O.grad(v, sc.pos, sc.vel, sc.col, sc.tri, o["id"], np.ones((pix.size, 3)), pix=pix)
            tests += pix.size * sc.T
        return time.perf_counter() - t0, tests, per * len(wl.views)

    if pixels > 0:
        dt, tests, n = run(pixels)
        return {"pixels": n, "seconds": dt, "tests": tests, "cores": O.num_threads()}
    # calibrate on growing samples until one takes a tenth of the budget (a
    # tiny first sample is dominated by per-call setup and overstates the cost)
    n = max(64, 4 * len(wl.views))
    while True:
        dt, _, n = run(n)
        if dt >= seconds / 10 or n >= 1 << 18:
            break
        n = int(min(1 << 18, n * min(8.0, max(2.0, seconds / 10 / max(dt, 1e-3)))))
    n = int(max(n, min(1 << 18, n * seconds / max(dt, 1e-3))))
    dt, tests, n = run(n)
    return {"pixels": n, "seconds": dt, "tests": tests, "cores": O.num_threads()}


def reference_arm(args, rank, world):
    wl = workload(args.workload)
    if rank != 0:
        return 0
    cpu_s = max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps + args.warmup)))
    # size the per-step sample once, then every step renders that many pixels
    n = cpu_oracle_sample(wl, cpu_s)["pixels"]
    for _ in range(args.warmup):
        cpu_oracle_sample(wl, cpu_s, pixels=max(1, n // 4))
    runs = [cpu_oracle_sample(wl, cpu_s, pixels=n) for _ in range(args.steps)]
    px = sum(r["pixels"] for r in runs)
    sec = sum(r["seconds"] for r in runs)
    val = px / sec / 1e6
    sample = (f"{runs[0]['pixels']} seeded pixels over the workload's views per step, FP64 forward + gradient, "
              f"every triangle tested")
    line = {"metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "sample": sample},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": runs[0]["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "tests_per_s": sum(r["tests"] for r in runs) / sec}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- our arm

METRIC = "Mpix/s & ray-tri tests/s at 1 GB300 (batched vs plain); fwd+bwd ms/frame"


def source_hash(name: str = "pr_stage_c.cu"):
    p = os.path.join(ROOT, "paper_1806_05385_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def measured_peak(key: str):
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0 if key == "hbm_gbs" else None  # the recipe's fallback


KERNEL_SOURCES = {"k_fragment": "pr_stage_c.cu", "k_shade<1>": "pr_stage_de.cu"}


def ncu_traffic(workload_kind: str, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, only
    if it was taken on this workload and on the kernel's current source."""
    p = os.path.join(ROOT, "profiles", "traffic_hmd.json")
    try:
        d = json.load(open(p))[kernel]
    except (OSError, ValueError, KeyError):
        return None
    if d.get("source_sha256_16") != source_hash(KERNEL_SOURCES[kernel]) or d.get("workload") != workload_kind:
        return None
    return d.get("dram_bytes_per_launch")


def aggregate(local_ms: float, local_pixels: int, dist=None, device="cpu"):
    """Whole-job throughput of weakly scaled replicas: the pixels all ranks
    rendered per step over the slowest rank's step time.  Returns (Mpix/s,
    max ms per step); without a process group, the local values."""
    if dist is None:
        return local_pixels / (local_ms * 1e-3) / 1e6, local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    p = torch.tensor([float(local_pixels)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return float(p.item()) / (ms * 1e-3) / 1e6, ms


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
    wl = workload(args.workload)
    views = wl.views
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    stream = torch.cuda.Stream()          # a capturable stream for the forward graph
    torch.cuda.set_stream(stream)
    handles = [B.pr_scene_upload(dev(sc.pos), dev(sc.vel), dev(sc.col), dev(sc.tri)) for sc in wl.scenes]
    hv = [handles[si] for si in wl.scene_of]
    ws = B.pr_workspace_create()
    npx = [v.W * v.H for v in views]
    ids = [torch.empty(n, dtype=torch.int32, device="cuda") for n in npx]
    depth = [torch.empty(n, dtype=torch.float32, device="cuda") for n in npx]
    rgb = [torch.empty(3 * n, dtype=torch.float32, device="cuda") for n in npx]
    gen = torch.Generator(device="cuda").manual_seed(1234)
    grad = [torch.randn(3 * n, device="cuda", generator=gen) for n in npx]
    grads = [tuple(torch.zeros(3 * sc.V, device="cuda") for _ in range(3)) for sc in wl.scenes]
    if args.workload == "batched":
        from paper_1806_05385_gb300 import autotune
        tiles = autotune.tune([(hv[k], v, wl.scenes[wl.scene_of[k]].T) for k, v in enumerate(views)])
    else:
        tiles = [16] * len(views)
    params = B.make_params("zenon", 16, wl.fp64, 0)
    entries = [(hv[k], v, ids[k], depth[k], rgb[k], tiles[k]) for k, v in enumerate(views)]
    # one training frame = one graph: forward (a)-(d) with the adjoint (e)
    # of an upstream image gradient, reading the frame's own records
    fgrads = [dict(grad_rgb=grad[k], dcol=grads[wl.scene_of[k]][0], dpos=grads[wl.scene_of[k]][1],
                   dvel=grads[wl.scene_of[k]][2]) for k in range(len(views))]
    graph = B.pr_graph_capture_frame(ws, entries, fgrads, params)
    # the same frame with CUDA events between the stages as graph nodes: the
    # stage (kernel) times of the rooflines come from its replays, run right
    # after the timed ones under the same conditions (the event nodes cost
    # tens of microseconds per replay, so the timed graph carries none)
    graph_t = B.pr_graph_capture_frame(ws, entries, fgrads,
                                       B.make_params("zenon", 16, wl.fp64, 0, graph_stage_times=1))
    ws_f = B.pr_workspace_create()
    graph_fwd = B.pr_graph_capture_batch(ws_f, entries, params)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    bwd_entries = [(hv[k], v, ids[k], grad[k], *grads[wl.scene_of[k]]) for k, v in enumerate(views)]
    ws_b = B.pr_workspace_create()

    def backward():
        B.pr_backward_batch(ws_b, bwd_entries)

    def step():
        B.pr_graph_enqueue(graph)

    def timed(fn, k, flush_l2=True, check=None):
        """Per call, device time between events recorded before and after
        fn's work on the stream; check() then reads the call's status."""
        ms = []
        for _ in range(k):
            if flush_l2:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if check:
                check()
            ms.append(e0.elapsed_time(e1))
        return ms

    for _ in range(max(3, args.warmup)):
        B.pr_graph_launch(graph)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    step_ms = timed(step, args.steps, check=lambda: B.pr_graph_status(graph))
    clocks = clk.stop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    st = B.pr_workspace_stats(ws)
    # stage times: CUDA events on the launching stream inside replays of the
    # instrumented graph, L2 flushed before each, averaged
    stage_runs = []

    def stage_check():
        B.pr_graph_status(graph_t)
        stage_runs.append(list(B.pr_workspace_stats(ws)["stage_ms"]))
    timed(lambda: B.pr_graph_enqueue(graph_t), args.steps, check=stage_check)
    stage_ms = [statistics.mean(r[k] for r in stage_runs) for k in range(8)]
    frag_ms = stage_ms[2]

    # forward only: batched graph vs plain per-view calls
    fwd_batched = timed(lambda: B.pr_graph_enqueue(graph_fwd), args.steps, check=lambda: B.pr_graph_status(graph_fwd))

    def plain():
        for k, v in enumerate(views):
            p = B.make_params("zenon", tiles[k], wl.fp64, 0)
            B.pr_rasterize(hv[k], v, p, ids[k], depth[k])
            B.pr_shade(hv[k], v, ids[k], rgb[k])
    for _ in range(2):
        plain()
    fwd_plain = timed(plain, max(3, args.steps // 2))
    bwd_ms = timed(backward, max(3, args.steps // 2))

    # the display step after shading (Sec. 3.1.1, "Display"): every view's
    # framebuffer image unfoveated to a display of the same size, both methods
    disp_out = [torch.empty(3 * n, device="cuda") for n in npx]
    ws_d = B.pr_workspace_create()

    def display(method):
        for k, v in enumerate(views):
            B.pr_unfoveate(ws_d, v, rgb[k], disp_out[k], v.W, v.H, method, 0.5)
    display_ms = {}
    for m in ("mip", "projected"):
        for _ in range(2):
            display(m)
        display_ms[m] = statistics.mean(timed(lambda: display(m), max(3, args.steps // 2)))
    B.pr_workspace_free(ws_d)
    hbm = measured_peak("hbm_gbs")
    # algorithmic bytes: 12 B rgb in + 12 B rgb out per pixel; the pyramid adds
    # one read of the image and writes / reads a third of it
    disp_bytes = {"mip": sum(12 * n + 12 * n + 12 * n + 8 * n for n in npx), "projected": sum(24 * n for n in npx)}
    display_step = {m: {"ms": display_ms[m], "mpix_s": world * sum(npx) / (display_ms[m] * 1e-3) / 1e6,
                        "gbs": disp_bytes[m] / (display_ms[m] * 1e-3) / 1e9,
                        "hbm_frac": disp_bytes[m] / (display_ms[m] * 1e-3) / 1e9 / hbm if hbm else None}
                    for m in display_ms}

    pix = sum(npx)
    value, mean_ms = aggregate(sum(step_ms) / len(step_ms), pix, dist, "cuda")

    # end to end through the public API with host buffers, as a training
    # loop would run it: every step the scene arrays and the upstream image
    # gradient go up from pinned host memory, the scene is updated, the frame
    # graph (forward + adjoint) replays, and the shaded images and the
    # gradients come back to pinned host memory, with the replay's status read
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hsc = [(pin(sc.pos), pin(sc.vel), pin(sc.col)) for sc in wl.scenes]
        dsc = [tuple(torch.empty_like(x, device="cuda") for x in a) for a in hsc]
        hrgb = [torch.empty(3 * n, dtype=torch.float32).pin_memory() for n in npx]
        hg = [g.cpu().pin_memory() for g in grad]
        hd = [tuple(torch.zeros(3 * sc.V).pin_memory() for _ in range(3)) for sc in wl.scenes]

        side = torch.cuda.Stream()

        def e2e_step():
            # the upstream gradient goes up on a second stream while the
            # scene is copied and updated; the frame waits for both
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                for g, hgk in zip(grad, hg):
                    g.copy_(hgk, non_blocking=True)
            for a, d in zip(hsc, dsc):
                for x, y in zip(a, d):
                    y.copy_(x, non_blocking=True)
            for h, d in zip(handles, dsc):
                B.pr_scene_update(h, *d)
            stream.wait_stream(side)
            for gs in grads:
                for x in gs:
                    x.zero_()
            B.pr_graph_enqueue(graph)
            for r, hr in zip(rgb, hrgb):
                hr.copy_(r, non_blocking=True)
            for gs, hgs in zip(grads, hd):
                for x, y in zip(gs, hgs):
                    y.copy_(x, non_blocking=True)
            stream.synchronize()
            B.pr_graph_status(graph)
        for _ in range(2):
            e2e_step()
        ems = timed(e2e_step, max(3, args.steps // 2))

        # the same steps as a training loop that overlaps its copies with
        # the GPU work, double-buffered: two copies of the scene, gradient
        # input, images and gradient outputs, each with its own frame graph
        # on the one workspace (replays stay in order on `stream`).  While
        # frame k runs on one set, step k+1's inputs go up into the other
        # set and its scene is updated (second stream), and step k's results
        # come down after it (third stream).  Every step still copies its
        # own inputs from pinned host memory and its own images and
        # gradients back to it, flushes L2 before its frame, and the host
        # reads every frame's status before it enqueues the next frame
        # (pr_graph_status reads the last replay's counters).
        side_in, side_out = torch.cuda.Stream(), torch.cuda.Stream()
        handles2 = [B.pr_scene_upload(dev(sc.pos), dev(sc.vel), dev(sc.col), dev(sc.tri)) for sc in wl.scenes]
        hv2 = [handles2[si] for si in wl.scene_of]
        rgb2 = [torch.empty_like(r) for r in rgb]
        grad2 = [g.clone() for g in grad]
        grads2 = [tuple(torch.zeros_like(x) for x in gs) for gs in grads]
        dsc2 = [tuple(torch.empty_like(x) for x in d) for d in dsc]
        entries2 = [(hv2[k], v, ids[k], depth[k], rgb2[k], tiles[k]) for k, v in enumerate(views)]
        fgrads2 = [dict(grad_rgb=grad2[k], dcol=grads2[wl.scene_of[k]][0], dpos=grads2[wl.scene_of[k]][1],
                        dvel=grads2[wl.scene_of[k]][2]) for k in range(len(views))]
        graph2 = B.pr_graph_capture_frame(ws, entries2, fgrads2, params)
        sets = [dict(h=handles, grad=grad, rgb=rgb, grads=grads, dsc=dsc, graph=graph),
                dict(h=handles2, grad=grad2, rgb=rgb2, grads=grads2, dsc=dsc2, graph=graph2)]

        def upload_copies(bs):
            """Step inputs -> buffer set bs on side_in: the upstream gradient
            and the scene arrays from pinned host memory.  The caller has
            synchronised on the last frame that read bs."""
            with torch.cuda.stream(side_in):
                for g, hgk in zip(bs["grad"], hg):
                    g.copy_(hgk, non_blocking=True)
                for a, d in zip(hsc, bs["dsc"]):
                    for x, y in zip(a, d):
                        y.copy_(x, non_blocking=True)

        def upload_update(bs):
            """pr_scene_update of set bs from its uploaded arrays, on side_in
            after the copies (it waits for side_in); returns the event the
            set's frame waits for."""
            with torch.cuda.stream(side_in):
                for h, d in zip(bs["h"], bs["dsc"]):
                    B.pr_scene_update(h, *d)
                ev = torch.cuda.Event()
                ev.record(side_in)
            return ev

        def e2e_pipelined(k_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            side_in.wait_event(e0)
            upload_copies(sets[0])
            ready = upload_update(sets[0])
            out_free = [None, None]
            for it in range(k_steps):
                bs = sets[it % 2]
                if it + 1 < k_steps:
                    # the other set's last frame (step it-1) has completed:
                    # the host synchronised on it at the end of that step
                    upload_copies(sets[(it + 1) % 2])
                stream.wait_event(ready)
                if out_free[it % 2] is not None:
                    stream.wait_event(out_free[it % 2])  # step it-2's results have left this set
                flush.zero_()
                for gs in bs["grads"]:
                    for x in gs:
                        x.zero_()
                B.pr_graph_enqueue(bs["graph"])
                done = torch.cuda.Event()
                done.record(stream)
                with torch.cuda.stream(side_out):
                    side_out.wait_event(done)
                    for r, hr in zip(bs["rgb"], hrgb):
                        hr.copy_(r, non_blocking=True)
                    for gs, hgs in zip(bs["grads"], hd):
                        for x, y in zip(gs, hgs):
                            y.copy_(x, non_blocking=True)
                    out_free[it % 2] = torch.cuda.Event()
                    out_free[it % 2].record(side_out)
                if it + 1 < k_steps:
                    ready = upload_update(sets[(it + 1) % 2])
                done.synchronize()
                B.pr_graph_status(bs["graph"])
            for ev in out_free:
                if ev is not None:
                    stream.wait_event(ev)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / k_steps

        e2e_pipelined(3)
        pms = e2e_pipelined(max(3, args.steps))
        # the loop's last results reached the host: they equal the images of
        # its last frame, and both buffer sets rendered the same images
        last = sets[(max(3, args.steps) - 1) % 2]
        for r, r2, hr in zip(last["rgb"], rgb2, hrgb):
            assert torch.equal(r.cpu(), hr), "pipelined end-to-end images differ from the device's"
            assert torch.equal(r2.cpu(), hr), "the two buffer sets rendered different images"
        B.pr_graph_free(graph2)
        for h in handles2:
            B.pr_scene_free(h)
        sv = sum(sc.V for sc in wl.scenes)
        h2d = 3 * sv * 12 + sum(g.numel() * 4 for g in hg)
        d2h = sum(x.numel() * 4 for x in hrgb) + 3 * sv * 12
        e2e = {"value": world * pix / (pms * 1e-3) / 1e6, "unit": "Mpix/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": pms,
               "path": "training loop through the public API with two buffer sets (scene copy, upstream "
                       "gradient, images, gradients; one frame graph each) used in turn: while frame k runs, step "
                       "k+1's scene arrays and upstream gradient go up from pinned host memory into the other set "
                       "and pr_scene_update runs there (second stream), and frame k's images and gradients go back "
                       "to pinned host memory after it (third stream); L2 flushed before every frame; the host "
                       "synchronises on every frame and reads its pr_graph_status before enqueuing the next; K "
                       "steps timed as a whole with CUDA events, from the first upload to the last download",
               "serial": {"value": world * pix / (statistics.mean(ems) * 1e-3) / 1e6,
                          "ms_per_step": statistics.mean(ems),
                          "path": "the same copies and calls with no overlap across steps (upload, update, frame, "
                                  "download, synchronise, status; L2 flushed before each step, outside the "
                                  "timed region)"}}

    # rooflines: stage (c) k_fragment (FP32 ALU) and the training frame's
    # shading + adjoint kernel k_shade<1> (HBM); the bench line's "roofline"
    # is the one of the two that takes longer per frame
    sm_mhz = clocks.get("sm_mhz") or 1470.0
    peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    ffma = B.pr_measure_fp32_peak()  # on-box cross-check of the derived peak (independent FMA chains)
    achieved = st["tests"] * FLOP_PER_TEST / (frag_ms * 1e-3) / 1e12 if frag_ms > 0 else 0.0
    roof_frag = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": achieved / peak if peak else None, "traffic": ncu_traffic(args.workload, "k_fragment"),
                 "kernel": "k_fragment", "time_ms": frag_ms, "flop_per_test": FLOP_PER_TEST,
                 "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 FLOP x median SM clock {sm_mhz:.0f} MHz "
                               f"sampled during the timed region (no FP32 figure in MEASURED_PEAKS.json)",
                 "peak_measured_ffma": ffma,
                 "achieved_basis": "ray-triangle tests of one frame x 39 FLOP / fragment-stage time of that frame "
                                   "(CUDA events on the launching stream, inside replays of the frame graph captured with "
                                   "stage events, one per timed step)"}
    # k_shade<1>: per pixel 8 B key in, 4 B id + 4 B depth + 12 B rgb out, 12 B
    # upstream gradient in; per visible triangle 108 B vertex data in (3 x
    # position, velocity, colour) and 108 B gradients out (3 x dcol, dpos, dvel)
    shade_ms = stage_ms[5]
    visible = sum(int(torch.unique(x[x >= 0]).numel()) for x in ids)
    shade_bytes = 40 * pix + 216 * visible
    hbm_peak = measured_peak("hbm_gbs")
    shade_gbs = shade_bytes / (shade_ms * 1e-3) / 1e9 if shade_ms > 0 else 0.0
    roof_shade = {"bound": "hbm", "achieved": shade_gbs, "peak": hbm_peak, "unit": "GB/s",
                  "frac": shade_gbs / hbm_peak if hbm_peak else None,
                  "traffic": ncu_traffic(args.workload, "k_shade<1>"), "kernel": "k_shade<1>", "time_ms": shade_ms,
                  "algorithmic_bytes": shade_bytes, "visible_triangles": visible,
                  "peak_basis": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                  "achieved_basis": "40 B per pixel + 216 B per visible triangle / shading + adjoint stage time "
                                    "(CUDA events on the launching stream, inside replays of the frame graph captured "
                                    "with stage events, one per timed step)"}
    roof, roof2 = (roof_shade, roof_frag) if shade_ms > frag_ms else (roof_frag, roof_shade)
    # stage (a) with the frame init, HBM: per triangle-view at least 84 B in
    # (three vertices' positions and velocities, indices) and 120 B out
    # (record, pixel box, candidate count); per pixel the 8 B key set to
    # ~0; per tile 16 B display box + 20 B counts and cursors
    ttot = sum(wl.scenes[wl.scene_of[k]].T for k in range(len(views)))
    ntiles = sum(((v.W + tiles[k] - 1) // tiles[k]) * ((v.H + tiles[k] - 1) // tiles[k]) for k, v in enumerate(views))
    a_bytes = 204 * ttot + 8 * pix + 36 * ntiles
    a_gbs = a_bytes / (stage_ms[0] * 1e-3) / 1e9 if stage_ms[0] > 0 else 0.0
    roof_a = {"bound": "hbm", "achieved": a_gbs, "peak": hbm_peak, "unit": "GB/s",
              "frac": a_gbs / hbm_peak if hbm_peak else None, "traffic": None,
              "kernel": "k_frame_init + k_bound (stage a)", "time_ms": stage_ms[0], "algorithmic_bytes": a_bytes,
              "achieved_basis": "204 B per triangle-view + 8 B per pixel + 36 B per tile (lower bound: the "
                                "half-planes of kept triangles not counted) / stage (a) event time"}
    roof = dict(roof, secondary=roof2, stage_a=roof_a)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r = cpu_oracle_sample(wl, args.cpu_seconds)
        cpu = {"value": r["pixels"] / r["seconds"] / 1e6, "unit": "Mpix/s", "cores": r["cores"], "kind": "oracle",
               "sample": f"{r['pixels']} seeded pixels over the workload's views, FP64 forward + gradient, "
                         f"every triangle tested ({r['tests']:.3g} tests in {r['seconds']:.1f} s)",
               "tests_per_s": r["tests"] / r["seconds"]}

    n_classes = len({(t, wl.fp64) for t in tiles})
    # frame init (with the tile boxes), bound, candidate scan, bin count, tile scan (with the work
    # items), bin scatter, run sort, one fragment launch per (tile, precision) class, [FP64 re-test],
    # resolve + shade + adjoint
    kernels_step = 8 + n_classes + (1 if wl.fp64 else 0)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if not wl.fp64 else "f32+f64-retest", "data": "synthetic",
        "config": {"workload": wl.name, "views": len(views), "pixels_per_step": pix,
                   "triangles": sum(sc.T for sc in wl.scenes),
                   "step": "one graph per frame: init + tile boxes, bound, bin, run sort, fragment, [FP64 re-test], "
                           "resolve + shade + adjoint (one kernel)",
                   "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": kernels_step * args.steps,
        "tests_per_s": st["tests"] / (frag_ms * 1e-3) if frag_ms > 0 else None,
        "ste": st["hits"] / st["tests"] if st["tests"] else None,
        "stats": {k: st[k] for k in ("tests", "hits", "pairs", "items", "culled", "pixels", "flagged", "changed",
                                     "fp64_depth_err")},
        "stage_ms": {"bound": stage_ms[0], "bin": stage_ms[1], "fragment": frag_ms,
                     "fp64_retest": stage_ms[3], "resolve_shade_adjoint": stage_ms[5],
                     "basis": "CUDA events between the stages, inside replays of the same frame graph "
                              "captured with them (graph_stage_times), one per timed step, L2 flushed"},
        "fwd_mpix_s": {"batched_graph": world * pix / (statistics.mean(fwd_batched) * 1e-3) / 1e6,
                       "plain_per_view": world * pix / (statistics.mean(fwd_plain) * 1e-3) / 1e6},
        "fwd_bwd_ms_per_frame": mean_ms, "bwd_ms_separate_call": statistics.mean(bwd_ms),
        "display_step": display_step,
        "tiles": sorted(set(tiles)),
    }
    B.pr_graph_free(graph)
    B.pr_graph_free(graph_t)
    B.pr_graph_free(graph_fwd)
    B.pr_workspace_free(ws)
    B.pr_workspace_free(ws_f)
    B.pr_workspace_free(ws_b)
    for h in handles:
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
