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


def test_ncu_record_is_gated_by_the_kernel_source(tmp_path, monkeypatch):
    """`traffic` and the on-chip counters are reported only while the kernel
    source hashes to the captured one (the template and the device helpers
    it inlines); any edit of either file, another inner QP or lost messages
    turn them into nulls."""
    import bench
    monkeypatch.setattr(bench, "kernel_sha", lambda: bench.NCU["src_sha256"])  # as if captured on this source
    rec = bench.ncu_record("chain1024", "box", 0.0)
    w = bench.NCU["workloads"]["chain1024"]
    assert rec["traffic"] == w["dram_bytes_per_launch"] and rec["traffic_launch_iters"] == w["iters_per_launch"]
    assert bench.ncu_record("batch256", "box", 0.0)["traffic_scaled_from"]
    assert bench.ncu_record("chain1024", "block", 0.0) == {"traffic": None, "onchip": None}
    assert bench.ncu_record("chain1024", "box", 0.1) == {"traffic": None, "onchip": None}
    assert bench.ncu_record("chain10", "box", 0.0) == {"traffic": None, "onchip": None}
    edited = []
    for i, path in enumerate(bench.KERNEL_SRC):
        f = tmp_path / f"src{i}"
        f.write_bytes(open(path, "rb").read() + (b"// edited\n" if i == 1 else b""))
        edited.append(str(f))
    monkeypatch.undo()
    sha = bench.kernel_sha()
    monkeypatch.setattr(bench, "KERNEL_SRC", edited)
    assert bench.kernel_sha() != sha
    assert bench.ncu_record("chain1024", "box", 0.0) == {"traffic": None, "onchip": None}


def test_roofline_counts_algorithmic_bytes_over_kernel_time():
    """achieved = algorithmic bytes per iteration x iterations of the launches
    (the longest instance of each) / summed sweep-kernel event time; frac
    against the given peak."""
    import bench
    info = {"iter_bytes_min": 46_532_272, "iter_bytes": 82_839_712}
    rec = {"iters": [[1000], [1000], [58]], "kms": [10.0, 10.0, 0.58]}
    r = bench.alg_roofline(info, rec, 6651.7, "measured")
    expect = 46_532_272 * 2058 / (20.58e-3) / 1e9
    assert abs(r["achieved"] - round(expect, 1)) < 1e-6
    assert r["frac"] == round(expect / 6651.7, 4) and r["bound"] == "hbm"
    assert r["mean_launch_ms"] == round(20.58 / 3, 4)
    assert r["algorithmic_bytes_per_iter"] == 46_532_272 and r["kernel_load_bytes_per_iter"] == 82_839_712
