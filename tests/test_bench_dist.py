"""Host logic of bench.py on CPU.  The multi-GPU (replica) path: two gloo
ranks with different step times; the whole-job value is the pixels of both
ranks over the slower rank's time, identical on every rank.  Also the
reference arm's JSON line, the gate on reported ncu traffic and the peak
fallback."""
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


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    """The ncu DRAM traffic of a kernel is reported only while the kernel's
    source is the one the counters were taken on, and only for the workload
    they were taken on; otherwise it is null."""
    import json
    import bench
    src = tmp_path / "paper_1806_05385_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "pr_stage_c.cu").write_text("// kernel source\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"workload": "hmd", "source_sha256_16": bench.source_hash("pr_stage_c.cu"),
             "dram_bytes_per_launch": 1234.0}
    (tmp_path / "profiles" / "traffic_hmd.json").write_text(json.dumps({"k_fragment": entry}))
    assert bench.ncu_traffic("hmd", "k_fragment") == 1234.0
    assert bench.ncu_traffic("large", "k_fragment") is None
    assert bench.ncu_traffic("hmd", "k_shade<1>") is None  # never captured
    (src / "pr_stage_c.cu").write_text("// kernel source, changed\n")
    assert bench.ncu_traffic("hmd", "k_fragment") is None


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    import json
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak("hbm_gbs") == 6800.0  # no file: the stated fallback
    assert bench.measured_peak("bf16_tflops") is None
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6674.2}))
    assert bench.measured_peak("hbm_gbs") == 6674.2
