"""The multi-GPU (replica) path of bench.py on CPU: two gloo ranks with
different step times; the whole-job value is the pixels of both ranks over
the slower rank's time, identical on every rank."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 2.0 if rank == 0 else 3.0
    value, ms = bench.aggregate(local_ms, 1_000_000, dist, "cpu")
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_rank_aggregate():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, ms = res[r]
        assert ms == pytest.approx(3.0)
        assert value == pytest.approx(2_000_000 / 3e-3 / 1e6)


def test_single_process_aggregate():
    import bench
    assert bench.aggregate(4.0, 2_000_000) == pytest.approx((500.0, 4.0))


def test_reference_arm_prints_one_json_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints
    one JSON line with the contract's keys, on a short sample."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cpu-seconds", "1", "--workload", "diff"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "impl", "cpu_baseline", "e2e"):
        assert k in d
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
