import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def pr():
    """The CUDA library through its Python binding; the GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_05385_gb300 import binding
    binding.load()
    return binding


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Every GPU-vs-oracle comparison of the session with the rule it was
    held to and what the FP32 windows forgave beyond the strict rule:
    mismatches excused only by them, and agreeing pixels over the flat 1e-5
    depth bound (tests/parity_util.py)."""
    try:
        from tests.parity_util import REPORTS
    except ImportError:
        return
    if not REPORTS:
        return
    tr = terminalreporter
    tr.section("GPU vs oracle parity (rule, pixels, mismatches, excused only by the FP32 windows, "
               "pixels over the flat 1e-5 depth bound, pixels over the flat 1e-4 colour bound)")
    for tid, rule, npx, mism, loose, over, dmax, rover, rmax in REPORTS:
        tr.write_line(f"{rule:6s} {npx:9d} px {mism:6d} mism {loose:5d} fp32-only {over:6d} depth>1e-5 "
                      f"(max {dmax:.1e}) {rover:6d} rgb>1e-4 (max {rmax:.1e})  {tid}")
    tot = {r: [0, 0, 0, 0] for r in ("strict", "fp32")}
    for _, rule, npx, mism, loose, over, _, rover, _ in REPORTS:
        tot[rule][0] += npx
        tot[rule][1] += loose
        tot[rule][2] += over
        tot[rule][3] += rover
    for rule, (npx, loose, over, rover) in tot.items():
        tr.write_line(f"total {rule}: {npx} pixels compared, {loose} mismatches excused only by the FP32 "
                      f"windows, {over} pixels over the flat depth bound, {rover} over the flat colour bound")
