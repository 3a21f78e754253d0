"""Host-side checks of the C ABI that need no GPU: the library builds and
exports every entry point include/pr.h declares, the ctypes records match the
C layouts, statuses come back without a device, and the stage (a) catch-up
interval (evaluated on the host) contains every time at which the rolling
scan meets the triangle, found here by brute force."""
import ctypes as C
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1806_05385_gb300 import binding as B
from paper_1806_05385_gb300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pr.h")


@pytest.fixture(scope="module")
def lib():
    return B.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pr_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", B.lib_path()], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_struct_layouts_match_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pr_view), offsetof(pr_view, pose0),
         offsetof(pr_view, light_w), sizeof(pr_params), sizeof(pr_stats), sizeof(pr_batch_view),
         offsetof(pr_batch_view, id_out), offsetof(pr_batch_view, tile), sizeof(pr_frame_grad),
         offsetof(pr_frame_grad, dvel), sizeof(pr_backward_view), offsetof(pr_backward_view, dvel),
         offsetof(pr_frame_grad, target_u8), offsetof(pr_frame_grad, loss), sizeof(pr_unfoveate_entry),
         offsetof(pr_unfoveate_entry, Hd));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(B.PrView), B.PrView.pose0.offset, B.PrView.light_w.offset, C.sizeof(B.PrParams),
            C.sizeof(B.PrStats), C.sizeof(B.PrBatchView), B.PrBatchView.id_out.offset, B.PrBatchView.tile.offset,
            C.sizeof(B.PrFrameGrad), B.PrFrameGrad.dvel.offset, C.sizeof(B.PrBackwardView),
            B.PrBackwardView.dvel.offset, B.PrFrameGrad.target_u8.offset, B.PrFrameGrad.loss.offset,
            C.sizeof(B.PrUnfoveateEntry), B.PrUnfoveateEntry.Hd.offset]
    assert got == want


def test_status_strings_and_version(lib):
    assert B.pr_version() >= 1
    assert B.pr_status_string(0) == "ok"
    assert "overflow" in B.pr_status_string(B.PR_ERR_OVERFLOW)
    assert B.pr_status_string(99) == "unknown status"


def test_invalid_arguments_are_statuses_not_crashes(lib):
    h = C.c_void_p()
    # null pointers are rejected before any device work
    assert lib.pr_scene_upload(None, None, None, None, 3, 1, None, C.byref(h)) == B.PR_ERR_INVALID_ARG
    assert lib.pr_rasterize(None, None, None, None, None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_shade(None, None, None, None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_backward(None, None, None, None, None, None, None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_rasterize_batch(None, None, 0, None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_frame_batch(None, None, 0, None, None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_graph_capture_frame(None, None, 0, None, None, None, C.byref(h)) == B.PR_ERR_INVALID_ARG
    assert lib.pr_graph_launch(None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_graph_enqueue(None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_graph_status(None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_measure_fp32_peak(None, None) == B.PR_ERR_INVALID_ARG
    assert lib.pr_unfoveate_batch(None, None, 0, None, None) == B.PR_ERR_INVALID_ARG


def test_no_device_is_reported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    pos = np.zeros((3, 3), np.float32)
    tri = np.array([[0, 1, 2]], np.int32)
    h = C.c_void_p()
    s = lib.pr_scene_upload(B._ptr(pos), B._ptr(pos), B._ptr(pos), B._ptr(tri), 3, 1, None, C.byref(h))
    assert s == B.PR_ERR_NO_CUDA


# --------------------------------------------------------------------------
# stage (a) catch-up interval (Zenon, Sec. 4.2.4) vs brute force
# --------------------------------------------------------------------------

def _met_times(view, S3, D3, n=4001):
    """Times in [0, 1] at which the scan meets some point of the triangle:
    dense sampling of t, and of barycentrics on a fine grid."""
    ts = np.linspace(0.0, 1.0, n)
    g = np.linspace(0, 1, 41)
    bb = np.array([(a, b, 1 - a - b) for a in g for b in g if a + b <= 1 + 1e-12])
    met = []
    for t in ts:
        P = S3 + t * D3                      # [3,3]
        X = bb @ P                            # [m,3]
        x = (X[:, 0] / (X[:, 2] * view.tan_x) + 1) / 2
        y = (X[:, 1] / (X[:, 2] * view.tan_y) + 1) / 2
        r = x * view.d[0] + y * view.d[1]
        if (r.min() - t) <= 0 <= (r.max() - t):
            met.append(t)
    return np.array(met)


@pytest.mark.parametrize("seed", range(6))
def test_catch_interval_contains_every_meeting_time(lib, seed):
    rng = np.random.default_rng(seed)
    view = S.View(W=64, H=64, tan_x=0.6, tan_y=0.5, pose0=np.eye(4), pose1=np.eye(4), mode=S.MODE_ROLLING,
                  d=(1.0, 0.0) if seed % 3 else (0.7, 0.3))
    checked = 0
    for _ in range(60):
        c = rng.uniform([-1.5, -1, 2], [1.5, 1, 8])
        S3 = c + rng.uniform(-0.6, 0.6, (3, 3))
        D3 = rng.normal(0, 0.6, (3, 3))
        D3[:, 2] = rng.normal(0, 0.5, 3)
        if (S3[:, 2].min() < 0.5) or ((S3 + D3)[:, 2].min() < 0.5):
            continue
        S3 = S3.astype(np.float32).astype(np.float64)
        E3 = (S3 + D3).astype(np.float32).astype(np.float64)
        D3 = E3 - S3
        ok, (lo, hi) = B.pr_debug_catch_interval(view, S3, E3)
        met = _met_times(view, S3, D3, n=801)
        if met.size == 0:
            continue
        checked += 1
        assert ok, "scan meets the triangle but the interval is empty"
        assert lo <= met.min() + 1e-6 and met.max() <= hi + 1e-6
        # and it is tight: no wider than the sampled set plus the sampling step and margin
        assert hi - lo <= (met.max() - met.min()) + 2 * (1.0 / 800) + 3e-4
    assert checked > 10


def test_catch_interval_linear_mover_closed_form(lib):
    """Static camera, fronto-parallel triangle moving along x: each vertex is
    met at t = x0 / (1 - V) (Sec. 4.2.4, the linear case)."""
    view = S.View(W=64, H=64, tan_x=0.5, tan_y=0.5, pose0=np.eye(4), pose1=np.eye(4), mode=S.MODE_ROLLING)
    z, vx = 4.0, 0.3
    S3 = np.array([[-0.6, -0.5, z], [0.5, -0.3, z], [-0.1, 0.6, z]])
    E3 = S3 + np.array([vx, 0.0, 0.0])
    ok, (lo, hi) = B.pr_debug_catch_interval(view, S3, E3)
    V = vx / (2 * z * 0.5)
    x0 = (S3[:, 0] / z / 0.5 + 1) / 2
    tc = x0 / (1 - V)
    assert ok
    assert lo == pytest.approx(tc.min(), abs=2e-4) and hi == pytest.approx(tc.max(), abs=2e-4)


def test_catch_interval_never_met(lib):
    """A triangle that stays ahead of the scan for the whole frame (moving
    right faster than the scan, starting right of it) is never met."""
    view = S.View(W=64, H=64, tan_x=0.5, tan_y=0.5, pose0=np.eye(4), pose1=np.eye(4), mode=S.MODE_ROLLING)
    z = 4.0
    S3 = np.array([[0.4, -0.2, z], [0.8, -0.1, z], [0.6, 0.3, z]])   # display x ~ 0.6 .. 0.7
    E3 = S3 + np.array([20.0, 0.0, 0.0])
    ok, _ = B.pr_debug_catch_interval(view, S3, E3)
    assert not ok
