#!/usr/bin/env python
"""Benchmark of the perceptual-rasterization hot path on GB300.

A training frame of the workload runs every stage of the path as one CUDA
graph: (a) bounds -> (b) binning and the depth sort of every work item's run
-> (c) per-fragment ray casting -> (d) shading for all views, with (e) the
adjoint of an upstream image gradient for every view in the same kernel.  A
timed step is R consecutive training frames (graph replays), R chosen from a
warm-up measurement so that the K timed steps span at least --target-seconds
(the clock record then covers the timed region).  value = framebuffer pixels
x R / step time (Mpix/s).

Prints ONE JSON line (rank 0).  Default workload: the batched 64-view
workload -- 64 independent scenes of 1k..500k triangles (log-uniform), square
views of side 512..2160 (log-uniform), modes uniform over classic, rolling,
foveated and joint, tile sizes autotuned -- seeded synthetic scenes already
resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|hmd|large|diff] [--target-seconds S]
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# more hardware work queues than the default 8, so that the training loop's
# streams (frames, uploads, downloads) do not share one and wait on each
# other's work (a process setting, read when CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

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
    ap.add_argument("--target-seconds", type=float, default=2.5,
                    help="the K timed steps span at least this long (frames per step sized to it)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["batched", "hmd", "large", "diff"], default="batched",
                    help="batched: 64 views of 1k-500k tris (default); hmd: stereo 1440x1600, 266k tris; large: "
                         "stereo 2160^2, 1M tris, FP64 re-test; diff: 512^2, 10k tris")
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
    p = os.path.join(ROOT, "profiles", f"traffic_{workload_kind}.json")
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
    # the training targets: one 8-bit RGB image per view (seeded synthetic),
    # slices of one flat buffer; the gradients of every scene ([V][3] dcol,
    # dpos, dvel) slices of one flat buffer too, so a training loop moves
    # each with one copy
    pix_off = np.concatenate([[0], np.cumsum([3 * n for n in npx])]).astype(np.int64)
    tflat = torch.randint(0, 256, (int(pix_off[-1]),), dtype=torch.uint8, device="cuda", generator=gen)
    tgt8 = [tflat[int(pix_off[k]):int(pix_off[k + 1])] for k in range(len(views))]
    loss = torch.zeros(len(views), device="cuda")
    v_off = np.concatenate([[0], np.cumsum([9 * sc.V for sc in wl.scenes])]).astype(np.int64)
    gflat = torch.zeros(int(v_off[-1]), device="cuda")

    def scene_slices(flat, s):
        o, V = int(v_off[s]), wl.scenes[s].V
        return flat[o:o + 3 * V], flat[o + 3 * V:o + 6 * V], flat[o + 6 * V:o + 9 * V]
    grads = [scene_slices(gflat, s) for s in range(len(wl.scenes))]
    if args.workload == "batched":
        from paper_1806_05385_gb300 import autotune
        tiles = autotune.tune([(hv[k], v, wl.scenes[wl.scene_of[k]].T) for k, v in enumerate(views)])
    else:
        tiles = [16] * len(views)
    params = B.make_params("zenon", 16, wl.fp64, 0)
    entries = [(hv[k], v, ids[k], depth[k], rgb[k], tiles[k]) for k, v in enumerate(views)]
    # one training frame = one graph: forward (a)-(d), the L2 loss of every
    # view against its 8-bit target image and the adjoint (e) of that loss,
    # reading the frame's own records
    fgrads = [dict(target_u8=tgt8[k], loss=loss[k:k + 1], dcol=grads[wl.scene_of[k]][0],
                   dpos=grads[wl.scene_of[k]][1], dvel=grads[wl.scene_of[k]][2]) for k in range(len(views))]
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

    frames = [1]  # training frames (graph replays) per timed step, sized after the warm-up

    def step():
        for _ in range(frames[0]):
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
    # frames per step: the K timed steps span at least target_seconds, so the
    # clock sampler sees the timed region many times (every rank takes the
    # largest R, so all ranks time the same work)
    frame_ms = statistics.median(timed(step, 5, check=lambda: B.pr_graph_status(graph)))
    frames[0] = max(1, int(np.ceil(args.target_seconds * 1e3 / (max(1, args.steps) * frame_ms))))
    if dist:
        fr = torch.tensor([frames[0]], dtype=torch.int64, device="cuda")
        dist.all_reduce(fr, op=dist.ReduceOp.MAX)
        frames[0] = int(fr.item())
    R = frames[0]
    k2 = max(3, min(args.steps, 10))  # repetitions of the secondary measurements
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
    timed(lambda: B.pr_graph_enqueue(graph_t), k2, check=stage_check)
    stage_ms = [statistics.mean(r[k] for r in stage_runs) for k in range(8)]
    frag_ms = stage_ms[2]

    # forward only: batched graph vs plain per-view calls
    fwd_batched = timed(lambda: B.pr_graph_enqueue(graph_fwd), k2, check=lambda: B.pr_graph_status(graph_fwd))

    def plain():
        for k, v in enumerate(views):
            p = B.make_params("zenon", tiles[k], wl.fp64, 0)
            B.pr_rasterize(hv[k], v, p, ids[k], depth[k])
            B.pr_shade(hv[k], v, ids[k], rgb[k])
    for _ in range(2):
        plain()
    fwd_plain = timed(plain, k2)
    bwd_ms = timed(backward, k2)

    # the display step after shading (Sec. 3.1.1, "Display"): every view's
    # framebuffer image unfoveated to a display of the same size, both methods
    disp_out = [torch.empty(3 * n, device="cuda") for n in npx]
    ws_d = B.pr_workspace_create()

    # every view's framebuffer image unfoveated in one batched call, and the
    # same with one call per view for comparison
    # (the ABI view structs are built once, as a caller that displays every
    # frame would keep them)
    pviews = [B.make_view(v) for v in views]
    disp_entries = [(pviews[k], rgb[k], disp_out[k], v.W, v.H) for k, v in enumerate(views)]

    def display(method):
        B.pr_unfoveate_batch(ws_d, disp_entries, method, 0.5)

    def display_per_view(method):
        for k, v in enumerate(views):
            B.pr_unfoveate(ws_d, pviews[k], rgb[k], disp_out[k], v.W, v.H, method, 0.5)
    display_ms, display_pv_ms = {}, {}
    for m in ("mip", "projected"):
        for _ in range(2):
            display(m)
            display_per_view(m)
        # the two forms alternate, so that both see the same conditions
        tb, tv = [], []
        for _ in range(k2):
            tb += timed(lambda: display(m), 1)
            tv += timed(lambda: display_per_view(m), 1)
        display_ms[m] = statistics.median(tb)
        display_pv_ms[m] = statistics.median(tv)
    B.pr_workspace_free(ws_d)
    hbm = measured_peak("hbm_gbs")
    # algorithmic bytes: 12 B rgb in + 12 B rgb out per pixel; the pyramid adds
    # one read of the image and writes / reads a third of it
    disp_bytes = {"mip": sum(12 * n + 12 * n + 12 * n + 8 * n for n in npx), "projected": sum(24 * n for n in npx)}
    display_step = {m: {"ms": display_ms[m], "mpix_s": world * sum(npx) / (display_ms[m] * 1e-3) / 1e6,
                        "gbs": disp_bytes[m] / (display_ms[m] * 1e-3) / 1e9,
                        "hbm_frac": disp_bytes[m] / (display_ms[m] * 1e-3) / 1e9 / hbm if hbm else None,
                        "per_view_call_ms": display_pv_ms[m],
                        "basis": "all views in one pr_unfoveate_batch call (per_view_call_ms: one pr_unfoveate "
                                 "call per view), CUDA events around the call on an idle stream (the "
                                 "call's host-side checks included), L2 flushed before each, the two "
                                 "forms alternating, median"}
                    for m in display_ms}

    pix = sum(npx)
    value, mean_ms = aggregate(sum(step_ms) / len(step_ms), pix * R, dist, "cuda")

    # end to end through the public API, as a training loop runs it: every
    # step the current scene parameters (positions, velocities, colours of
    # every scene: the host's copy, as an optimiser on the host keeps them)
    # and the step's 8-bit target images go up from pinned host memory, one
    # copy each, pr_scene_update_batch steps every scene from them, the
    # training-frame graph replays (forward, L2 loss, adjoint), and the
    # per-view losses and the per-vertex gradients come back to pinned host
    # memory, one copy each, with every replay's status read on the host.
    # No image comes back: a training step returns its loss and gradients.
    e2e = None
    if not args.no_e2e:
        hpar = torch.cat([torch.from_numpy(np.concatenate([sc.pos.ravel(), sc.vel.ravel(), sc.col.ravel()]))
                          for sc in wl.scenes]).pin_memory()
        htf = tflat.cpu().pin_memory()
        hloss = torch.zeros(len(views)).pin_memory()
        hgrad = torch.zeros(int(v_off[-1])).pin_memory()
        side_in, side_out = torch.cuda.Stream(), torch.cuda.Stream()
        # two buffer sets (scenes, parameters, targets, loss, gradients; one
        # frame graph each) used in turn, so one step's uploads and the
        # previous step's downloads overlap the current frame; replays stay
        # in order on `stream` (they share the workspace)
        handles2 = [B.pr_scene_upload(dev(sc.pos), dev(sc.vel), dev(sc.col), dev(sc.tri)) for sc in wl.scenes]
        hv2 = [handles2[si] for si in wl.scene_of]
        tflat2 = torch.empty_like(tflat)
        tgt2 = [tflat2[int(pix_off[k]):int(pix_off[k + 1])] for k in range(len(views))]
        loss2 = torch.zeros_like(loss)
        gflat2 = torch.zeros_like(gflat)
        grads2 = [scene_slices(gflat2, s) for s in range(len(wl.scenes))]
        rgb2 = [torch.empty_like(r) for r in rgb]
        entries2 = [(hv2[k], v, ids[k], depth[k], rgb2[k], tiles[k]) for k, v in enumerate(views)]
        fgrads2 = [dict(target_u8=tgt2[k], loss=loss2[k:k + 1], dcol=grads2[wl.scene_of[k]][0],
                        dpos=grads2[wl.scene_of[k]][1], dvel=grads2[wl.scene_of[k]][2]) for k in range(len(views))]
        graph2 = B.pr_graph_capture_frame(ws, entries2, fgrads2, params)
        sets = [dict(h=handles, par=torch.empty(hpar.numel(), device="cuda"), tf=tflat, loss=loss, g=gflat,
                     graph=graph),
                dict(h=handles2, par=torch.empty(hpar.numel(), device="cuda"), tf=tflat2, loss=loss2, g=gflat2,
                     graph=graph2)]
        for bs in sets:
            bs["pv"] = [scene_slices(bs["par"], s) for s in range(len(wl.scenes))]

        def upload(bs, after=None):
            """Step inputs -> buffer set bs on side_in, once the event `after`
            (the last frame that read bs) has passed: parameters and targets,
            one copy each, then every scene updated from the parameters;
            returns the event the set's frame waits for."""
            with torch.cuda.stream(side_in):
                if after is not None:
                    side_in.wait_event(after)
                bs["par"].copy_(hpar, non_blocking=True)
                bs["tf"].copy_(htf, non_blocking=True)
                B.pr_scene_update_batch(bs["h"], [p[0] for p in bs["pv"]], [p[1] for p in bs["pv"]],
                                        [p[2] for p in bs["pv"]])
                ev = torch.cuda.Event()
                ev.record(side_in)
            return ev

        marks = []  # (frame start, frame end) events of the timed loop's steps
        host_t = []  # host clock when each of them was enqueued

        def frame(bs):
            f0 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            bs["loss"].zero_()
            bs["g"].zero_()
            B.pr_graph_enqueue(bs["graph"])
            done = torch.cuda.Event(enable_timing=True)
            done.record(stream)
            marks.append((f0, done))
            host_t.append(time.perf_counter())
            return done

        def download(bs, done):
            with torch.cuda.stream(side_out):
                side_out.wait_event(done)
                hloss.copy_(bs["loss"], non_blocking=True)
                hgrad.copy_(bs["g"], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(side_out)
            return ev

        def e2e_loop(k_steps, overlap=True):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            side_in.wait_event(e0)
            ready = upload(sets[0])
            out_free = [None, None]
            prev = None  # (done event, graph) of the step whose status the host reads next
            for it in range(k_steps):
                bs = sets[it % 2 if overlap else 0]
                stream.wait_event(ready)
                if out_free[it % 2] is not None:
                    stream.wait_event(out_free[it % 2])  # step it-2's results have left this set
                flush.zero_()
                done = frame(bs)
                if overlap:
                    if it + 1 < k_steps:
                        # the other set's inputs change once its last frame
                        # (step it-1) has finished: a wait on the device
                        ready = upload(sets[(it + 1) % 2], prev[0] if prev is not None else None)
                    out_free[it % 2] = download(bs, done)
                    if prev is not None:
                        # step it-1's status, read while step it runs (each
                        # graph has its own copy of its status words)
                        prev[0].synchronize()
                        B.pr_graph_status(prev[1])
                    prev = (done, bs["graph"])
                else:
                    out_free[0] = download(bs, done)
                    done.synchronize()
                    B.pr_graph_status(bs["graph"])
                    if it + 1 < k_steps:
                        out_free[0].synchronize()
                        ready = upload(sets[0])
            if prev is not None:
                prev[0].synchronize()
                B.pr_graph_status(prev[1])
            for ev in out_free:
                if ev is not None:
                    stream.wait_event(ev)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / k_steps

        e2e_loop(3)
        # the step's transfers alone, for reading the overlap: one upload
        # (copies + scene updates) and one download, each timed by itself
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(side_in)
        upload(sets[0])
        a1.record(side_in)
        a1.synchronize()
        up_ms = a0.elapsed_time(a1)
        ev0 = torch.cuda.Event()
        ev0.record(stream)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(side_out)
        download(sets[0], ev0)
        b1.record(side_out)
        b1.synchronize()
        down_ms = b0.elapsed_time(b1)
        marks.clear()
        host_t.clear()
        # the timed steps of the overlapped loop: the bench's step count (its
        # first upload and last download, which nothing overlaps, are spread
        # over them)
        ke = max(3, args.steps)
        # the host waits for a frame every step, so a pause of this Python
        # process idles the GPU (one run saw a 16 ms stall between two
        # enqueues); the cyclic garbage collector, the pause the harness
        # itself can cause, runs before the timed loops and not during them,
        # as timeit does
        gc.collect()
        gc.disable()
        try:
            pms = e2e_loop(ke)
        finally:
            gc.enable()
        # how the steps lay on the compute stream: each frame's own time, and
        # the wait before it (its inputs' upload, when that did not overlap)
        frames_in_loop = [a.elapsed_time(b) for a, b in marks]
        gaps_in_loop = [marks[k - 1][1].elapsed_time(marks[k][0]) for k in range(1, len(marks))]
        frame_in_loop, gap_in_loop = statistics.median(frames_in_loop), statistics.median(gaps_in_loop)
        host_gap_max = 1e3 * max(b - a for a, b in zip(host_t, host_t[1:]))
        # the loop's last results reached the host: they equal the last
        # frame's losses and gradients on the device
        last = sets[(ke - 1) % 2]
        assert torch.equal(last["loss"].cpu(), hloss), "end-to-end losses differ from the device's"
        assert torch.equal(last["g"].cpu(), hgrad), "end-to-end gradients differ from the device's"
        gc.collect()
        gc.disable()
        try:
            sms = e2e_loop(k2, overlap=False)
        finally:
            gc.enable()
        B.pr_graph_free(graph2)
        for h in handles2:
            B.pr_scene_free(h)
        h2d = hpar.numel() * 4 + htf.numel()
        d2h = hgrad.numel() * 4 + hloss.numel() * 4
        e2e = {"value": world * pix / (pms * 1e-3) / 1e6, "unit": "Mpix/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": pms,
               "upload_ms_alone": up_ms, "download_ms_alone": down_ms,
               "frame_ms_in_loop": frame_in_loop, "gap_ms_between_frames": gap_in_loop,
               "frame_ms_in_loop_max": max(frames_in_loop), "gap_ms_between_frames_max": max(gaps_in_loop),
               "gap_ms_between_frames_total": sum(gaps_in_loop),
               "host_ms_between_enqueues_max": host_gap_max,
               "path": "training loop through the public API: every step the parameters of every scene (positions, "
                       "velocities, colours: the host's copy) and the step's 8-bit target images go up from pinned "
                       "host memory (one copy each), pr_scene_update_batch steps every scene from them, the "
                       "training-frame graph replays (forward, L2 loss against the targets, adjoint), and the "
                       "per-view losses and per-vertex gradients come back to pinned host memory (one copy each); "
                       "the host reads every replay's pr_graph_status, each while the next replay runs (every "
                       "graph keeps its own status copy), all before the timed region ends; two buffer sets used "
                       "in turn, so the next step's uploads (second stream, after the set's last frame on the "
                       "device) and this step's downloads (third stream) overlap the frames; L2 flushed before "
                       "every frame; K steps timed as a whole with CUDA events from the first upload to the last "
                       "download, Python's cyclic garbage collector paused during the timed steps",
               "serial": {"value": world * pix / (sms * 1e-3) / 1e6, "ms_per_step": sms,
                          "path": "the same calls and copies on one buffer set with no overlap across steps: "
                                  "upload, frame, download, wait, status, then the next step's upload"}}

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
                                   "stage events, ten replays)"}
    # k_shade<1>: per pixel 8 B key in, 4 B id + 4 B depth + 12 B rgb out, 3 B
    # 8-bit target in; per visible triangle 108 B vertex data in (3 x
    # position, velocity, colour) and 108 B gradients out (3 x dcol, dpos, dvel)
    shade_ms = stage_ms[5]
    visible = sum(int(torch.unique(x[x >= 0]).numel()) for x in ids)
    # a frame with more than 96 MB of keys has the shading set each covered
    # pixel's key back to ~0 for the next frame (8 B more per covered pixel)
    covered = sum(int((x >= 0).sum()) for x in ids)
    reset_bytes = 8 * covered if 8 * pix > (96 << 20) else 0
    shade_bytes = 31 * pix + 216 * visible + reset_bytes
    hbm_peak = measured_peak("hbm_gbs")
    shade_gbs = shade_bytes / (shade_ms * 1e-3) / 1e9 if shade_ms > 0 else 0.0
    roof_shade = {"bound": "hbm", "achieved": shade_gbs, "peak": hbm_peak, "unit": "GB/s",
                  "frac": shade_gbs / hbm_peak if hbm_peak else None,
                  "traffic": ncu_traffic(args.workload, "k_shade<1>"), "kernel": "k_shade<1>", "time_ms": shade_ms,
                  "algorithmic_bytes": shade_bytes, "visible_triangles": visible,
                  "peak_basis": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                  "covered_pixels": covered, "key_reset_bytes": reset_bytes,
                  "achieved_basis": "31 B per pixel + 216 B per visible triangle (+ 8 B per covered pixel where "
                                    "the shading sets the keys back) / shading + adjoint stage time "
                                    "(CUDA events on the launching stream, inside replays of the frame graph captured "
                                    "with stage events, ten replays)"}
    roof, roof2 = (roof_shade, roof_frag) if shade_ms > frag_ms else (roof_frag, roof_shade)
    # stage (a) with the frame init, HBM: per triangle-view at least 84 B in
    # (three vertices' positions and velocities, indices) and 120 B out
    # (record, pixel box, candidate count); per pixel the 8 B key set to
    # ~0; per tile 16 B display box + 20 B counts and cursors
    ttot = sum(wl.scenes[wl.scene_of[k]].T for k in range(len(views)))
    ntiles = sum(((v.W + tiles[k] - 1) // tiles[k]) * ((v.H + tiles[k] - 1) // tiles[k]) for k, v in enumerate(views))
    # (the key clear, 8 B per pixel, only where the frame's keys fit in L2:
    # a larger frame's keys are set back by the previous frame's shading)
    a_bytes = 204 * ttot + (8 * pix if 8 * pix <= (96 << 20) else 0) + 36 * ntiles
    a_gbs = a_bytes / (stage_ms[0] * 1e-3) / 1e9 if stage_ms[0] > 0 else 0.0
    roof_a = {"bound": "hbm", "achieved": a_gbs, "peak": hbm_peak, "unit": "GB/s",
              "frac": a_gbs / hbm_peak if hbm_peak else None, "traffic": None,
              "kernel": "k_frame_init + k_bound (stage a)", "time_ms": stage_ms[0], "algorithmic_bytes": a_bytes,
              "achieved_basis": "204 B per triangle-view + 8 B per pixel (frames with keys within 96 MB) + "
                                "36 B per tile (lower bound: the "
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
    # resolve + shade + loss + adjoint, the losses' partial sums
    kernels_step = 9 + n_classes + (1 if wl.fp64 else 0)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if not wl.fp64 else "f32+f64-retest", "data": "synthetic",
        "config": {"workload": wl.name, "views": len(views), "frames_per_step": R, "pixels_per_frame": pix,
                   "pixels_per_step": pix * R, "triangles": sum(sc.T for sc in wl.scenes),
                   "step": f"{R} training frames, each one replay of the frame graph: init + tile boxes, bound, bin, "
                           "run sort, fragment, [FP64 re-test], resolve + shade + L2 loss against each view's 8-bit "
                           "target image + adjoint (one kernel); the status of the step's last replay is read after it",
                   "l2": f"flushed before every timed step (256 MB write); between the frames of a step, inputs larger "
                         f"than L2: each frame reads {96 * ttot / 1e6:.0f} MB of stage (a) records and writes "
                         f"{20 * pix / 1e6:.0f} MB of images", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": kernels_step * R * args.steps,
        "tests_per_s": st["tests"] / (frag_ms * 1e-3) if frag_ms > 0 else None,
        "ste": st["hits"] / st["tests"] if st["tests"] else None,
        "stats": {k: st[k] for k in ("tests", "hits", "pairs", "items", "culled", "pixels", "flagged", "changed",
                                     "fp64_depth_err")},
        "stage_ms": {"bound": stage_ms[0], "bin": stage_ms[1], "fragment": frag_ms,
                     "fp64_retest": stage_ms[3], "resolve_shade_adjoint": stage_ms[5],
                     "basis": "CUDA events between the stages, inside replays of the same frame graph "
                              "captured with them (graph_stage_times), ten replays, L2 flushed before each"},
        "fwd_mpix_s": {"batched_graph": world * pix / (statistics.mean(fwd_batched) * 1e-3) / 1e6,
                       "plain_per_view": world * pix / (statistics.mean(fwd_plain) * 1e-3) / 1e6},
        "fwd_bwd_ms_per_frame": mean_ms / R, "bwd_ms_separate_call": statistics.mean(bwd_ms),
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
