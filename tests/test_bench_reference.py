"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the contract's keys and the same workload description as
the GPU arm; no GPU is needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    import bench
    from paper_2103_14990_gb300 import instances as I
    assert d["config"] == bench.bench_config(I.chain1024(), 1)
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT


def test_all_cores_baseline_aggregates_processes():
    """The all-cores oracle baseline runs one single-threaded oracle process
    per core on the same bounded sample and adds their rates."""
    import types
    import bench
    args = types.SimpleNamespace(workload="chain10", sample_seconds=0.2, steps=4)
    out = bench.cpu_baseline_all_cores(args, [10, 10, 10, 10], cores=2)
    assert out["cores"] == 2 and out["kind"] == "oracle"
    assert out["value"] is not None and out["value"] > 0
    assert out["oracle_admm_iters_per_s"] > 0
    # four steps of ten iterations at the aggregate rate (plus the u/dynamics tail)
    assert out["value"] <= 4 / (40 / out["oracle_admm_iters_per_s"]) + 1e-9
