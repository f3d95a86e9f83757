#!/usr/bin/env python
"""DLMPC benchmark on GB300: closed-loop MPC steps/s of the N=1024 chain.

One "step" is one MPC step of Alg. 1 (per-step precompute, the whole ADMM of
Alg. 2 to convergence, u(tau), x(tau+1)) for the chain of 1024 subsystems,
T=10, d=3, |x| <= 1, |u| <= 2, x(0) ~ U[-0.9, 0.9] (seed 0), FP32 sweeps.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

Our arm: W warm-up steps, then the state is reset to x(0) and K closed-loop
steps are timed with CUDA events recorded by the library on its stream (the
L2 is flushed between steps by a 256 MiB write outside the timed events).
Headline: warm-started (previous step's Psi/Lambda) steps; the same K steps
with cold starts ("plain") and through the host-buffer C-ABI call ("e2e")
are reported beside it.  N > 1: one independent replica per GPU, no
communication (weak scaling).  The reference arm times the FP64 oracle on
the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPC steps/s & ADMM iters/s, batched+warm-start vs plain at 1e-4 rel; HBM GB/s"
UNIT = "MPC steps/s"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SRC = os.path.join(ROOT, "paper_2103_14990_gb300", "csrc", "dlmpc_sweep.cu")
# DRAM bytes (read + write) of one sweep_kernel launch of a workload from an
# ncu capture, and the sha256 of the kernel source it was taken on; reported
# as null for other workloads and when the source has changed since.
NCU_TRAFFIC = {"workload": "chain1024", "src_sha256": "82fb4a1ebcf2a59f25bf54a70c1e95e4fb0e1907e249160eb066d13d18dfed25",
               "bytes_per_launch": 158949632,  # profiles/sweep_kernel_chain1024.md
               # the same kernel's on-chip load from the full capture (50 fixed
               # iterations, same launch shape): where the loop's bytes are served
               "onchip": {"lts_throughput_pct_of_peak": 21.9, "l2_hit_rate_pct": 93.6,
                          "issue_active_pct": 38.3, "dram_throughput_pct_of_peak": 1.6}}


INNER_QP = {"box": "diagonal Q, R with boxes (closed-form row Phi-step)",
            "block": "full SPD Q_i, R_i with boxes (slot box-QP)",
            "coupled": "full SPD Q_i, R_i, boxes and 2 coupled state rows per slot (explicit slot-QP solution)"}


def workload(name: str, inner_qp: str = "box"):
    from paper_2103_14990_gb300 import instances as I
    p = {"chain1024": I.chain1024, "chain10": I.chain10, "grid64": I.grid64}[name]()
    if inner_qp == "block":
        p = I.with_block_costs(p, seed=101)
    elif inner_qp == "coupled":
        p = I.with_coupled_constraints(p, seed=102, n_cx=2, n_cu=0, g_range=(0.8, 1.2))
    return p


def bench_config(prob, world: int, inner_qp: str = "box", stale_prob: float = 0.0) -> dict:
    """The workload description shared by both arms."""
    return {"workload": prob.name, "inner_qp": INNER_QP[inner_qp], "message_loss": stale_prob,
            "n_sub": prob.n_sub, "T": prob.T, "d": prob.d, "boxes": "|x|<=1, |u|<=2",
            "warm_start": "previous MPC step's Psi/Lambda (step 0 cold)", "max_iter": prob.max_iter,
            "eps": prob.eps_p, "l2": "flushed between steps (256 MiB write outside the events)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def kernel_sha() -> str:
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def replica_throughput(t_local: float, steps: int, world: int, dist=None, device: str = "cpu"):
    """Whole-job MPC steps/s of `world` independent replicas that each ran
    `steps` steps: all ranks' units over the slowest rank's time (max over
    ranks).  Returns (value, max time)."""
    t = t_local
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * steps / t, t


def run_ours(args):
    import numpy as np
    import torch
    import paper_2103_14990_gb300 as pkg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prob = workload(args.workload, args.inner_qp)
    t_setup = time.time()
    solver = pkg.Solver([prob])
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    if args.stale_prob > 0:  # simulated lost messages (the distributed setting)
        solver.set_option(pkg.OPT_STALE_PROB, args.stale_prob)
        solver.set_option(pkg.OPT_STALE_SEED, 2021)
    n, nx, nu = prob.n_sub, prob.nx, prob.nu
    x0 = torch.tensor(prob.x0.astype(np.float32), device="cuda")
    tune = []
    if not args.no_autotune:
        t_tune = time.time()
        tune = solver.autotune(x0, iters=args.tune_iters)
        t_tune = time.time() - t_tune
    solver.set_option(pkg.OPT_TIMING, 1)
    info = solver.info()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def loop(K, warm):
        x = x0.clone()
        xn = torch.empty_like(x)
        u = torch.empty(n, nu, device="cuda")
        kms, sms, iters, status = [], [], [], []
        for tau in range(K):
            flush.zero_()
            rc, st = solver.step(x, u, xn, warm=(pkg.WARM_COLD if tau == 0 else warm), stats=True)
            a, b = solver.timing()
            kms.append(a)
            sms.append(b)
            iters.append(st[0]["iters"])
            status.append(st[0]["status"])
            x, xn = xn, x
        return kms, sms, iters, status, x

    def sync_all():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # warm-up (discarded), then the timed closed loops from x(0)
    loop(args.warmup, pkg.WARM_PREVIOUS)
    sync_all()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        kms, sms, iters, status, xK = loop(args.steps, pkg.WARM_PREVIOUS)
        sync_all()
        wall = time.perf_counter() - wall0
    value, t_dev = replica_throughput(sum(sms) / 1e3, args.steps, world, dist, device="cuda")
    kern_s = sum(kms) / 1e3
    tot_iters = sum(iters)

    # the same closed loop replayed from captured CUDA graphs (whole-step events)
    solver.set_option(pkg.OPT_GRAPH, 1)
    loop(2, pkg.WARM_PREVIOUS)
    gk, gs, git, gst, _ = loop(args.steps, pkg.WARM_PREVIOUS)
    solver.set_option(pkg.OPT_GRAPH, 0)
    graph = {"value": args.steps / (sum(gs) / 1e3), "unit": UNIT, "iters_per_step": sum(git) / len(git)}

    # plain: cold start at every step, same kernel
    pk, ps, pit, pst, _ = loop(args.steps, pkg.WARM_COLD)
    plain = {"value": args.steps / (sum(ps) / 1e3), "unit": UNIT,
             "admm_iters_per_s": sum(pit) / (sum(pk) / 1e3), "iters_per_step": sum(pit) / len(pit)}

    # ablation of the paper's GPU mappings (Sec. III): ADMM iterations/s from x(0)
    ablation = {}
    if not args.no_ablation and args.inner_qp == "box" and args.stale_prob == 0:  # the paper's mappings
        names = {0: "naive (Sec. III-A)", 1: "combined (Sec. III-C)", 2: "persistent column patch (this library)"}
        for v, it_n in ((0, args.ablation_iters), (1, args.ablation_iters), (2, 10 * args.ablation_iters)):
            solver.run_variant(v, x0, 2)  # warm-up
            ms = solver.run_variant(v, x0, it_n)
            ablation[names[v]] = {"admm_iters_per_s": round(1e3 * it_n / ms, 1), "iters": it_n}
        base = ablation[names[0]]["admm_iters_per_s"]
        for v in ablation.values():
            v["speedup_vs_naive"] = round(v["admm_iters_per_s"] / base, 2)

    learned = (learned_line(prob, args)
               if (not args.no_learned and rank == 0 and world == 1 and args.inner_qp == "box"
                   and args.stale_prob == 0) else None)
    batched = (batched_line(prob, args, flush)
               if (args.batch > 1 and args.stale_prob == 0 and rank == 0 and world == 1) else None)

    # e2e: host (pinned) buffers through the C ABI, H2D and D2H inside the timed region
    xh = torch.empty(n, nx, dtype=torch.float32, pin_memory=True)
    xnh = torch.empty(n, nx, dtype=torch.float32, pin_memory=True)
    uh = torch.empty(n, nu, dtype=torch.float32, pin_memory=True)
    xh.copy_(x0.cpu())
    sync_all()
    e0 = time.perf_counter()
    for tau in range(args.steps):
        solver.step_host_ptr(xh.data_ptr(), uh.data_ptr(), xnh.data_ptr(),
                             warm=(pkg.WARM_COLD if tau == 0 else pkg.WARM_PREVIOUS))
        xh, xnh = xnh, xh
    e_wall = time.perf_counter() - e0
    e2e = {"value": args.steps / e_wall, "unit": UNIT, "h2d_bytes_per_step": n * nx * 4,
           "d2h_bytes_per_step": n * (nu + nx) * 4 + 32 + 16}

    # roofline of the sweep kernel: algorithmic bytes / CUDA-event kernel time
    peak, peak_src = measured_peaks()
    achieved = info["iter_bytes"] * tot_iters / kern_s / 1e9
    ncu_current = (NCU_TRAFFIC["src_sha256"] == kernel_sha() and NCU_TRAFFIC["workload"] == args.workload
                   and args.inner_qp == "box" and args.stale_prob == 0)
    traffic = NCU_TRAFFIC["bytes_per_launch"] if ncu_current else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_src, "kernel": "sweep_kernel",
                "algorithmic_bytes_per_iter": info["iter_bytes"],
                "mean_launch_ms": round(sum(kms) / len(kms), 4),
                "note": "the operators stay in shared memory and L2: DRAM moves `traffic` bytes per launch, "
                        "far below the algorithmic bytes; the loop is bound by on-chip latency (onchip)",
                "onchip": NCU_TRAFFIC["onchip"] if ncu_current else None}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_dev / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded chain plant, x0 ~ U[-0.9,0.9])",
        "config": bench_config(prob, world, args.inner_qp, args.stale_prob),
        "admm_iters_per_s": round(tot_iters / kern_s, 1),
        "iters_per_step": round(tot_iters / args.steps, 2),
        "steps_at_max_iter": int(sum(1 for s in status if s != 0)),
        "plain": plain,
        "e2e": e2e,
        "roofline": roofline,
        "graph": graph,
        "ablation": ablation,
        "learned": learned,
        "batched": batched,
        "sweep": {"group_threads": info["group_threads"], "groups_per_cta": info["groups_per_cta"],
                  "wave": info["wave"], "grid_ctas": info["grid_ctas"], "smem_bytes": info["smem_bytes"],
                  "resident_n_items": info["resident_n_items"],
                  "resident_state_items": info["resident_state_items"],
                  "autotuned_shapes": len(tune), "autotune_s": round(t_tune, 3) if tune else None},
        "gpu_launches": 2 * args.steps,
        "setup_precompute_s": round(t_setup, 3),
        "wall_s_timed_region": round(wall, 4),
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.inner_qp == "box" and args.stale_prob == 0:
        out["cpu_baseline"] = cpu_baseline(args, iters)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args, iters)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def batched_line(prob, args, flush):
    """Several instances of the workload (the same plant, different x(0)) in
    one context: one launch per MPC step advances every instance's closed
    loop, an instance at rest once its ADMM has converged.  Instance-steps per
    second against the single-instance line."""
    import numpy as np
    import torch
    import dataclasses
    import paper_2103_14990_gb300 as pkg
    from paper_2103_14990_gb300 import instances as I
    B = args.batch
    x0s = I.random_x0(prob.n_sub, B, seed=3000)
    probs = [dataclasses.replace(prob, x0=x0s[b]) for b in range(B)]
    s = pkg.Solver(probs)
    x = torch.tensor(np.concatenate([p.x0 for p in probs]).astype(np.float32), device="cuda")
    s.autotune(x, iters=args.tune_iters)
    s.set_option(pkg.OPT_TIMING, 1)
    xn = torch.empty_like(x)
    u = torch.empty(x.shape[0], prob.nu, device="cuda")
    steps = max(3, args.steps // 5)
    ms, iters = 0.0, []
    for tau in range(args.warmup + steps):
        flush.zero_()
        rc, st = s.step(x, u, xn, warm=(pkg.WARM_COLD if tau == 0 else pkg.WARM_PREVIOUS), stats=True)
        if tau >= args.warmup:
            ms += s.timing()[1]
            iters.append([d["iters"] for d in st])
        x, xn = xn, x
    info = s.info()
    s.close()
    it = np.array(iters)
    return {"instances": B, "steps": steps, "value": round(B * steps / (ms / 1e3), 3), "unit": "instance MPC steps/s",
            "ms_per_step": round(ms / steps, 4), "launch_iters_per_step": round(float(it.max(axis=1).mean()), 2),
            "instance_admm_iters_per_s": round(float(it.sum()) / (ms / 1e3), 1),
            "instance_iters_per_step": round(float(it.mean()), 2),
            "sweep": {"group_threads": info["group_threads"], "groups_per_cta": info["groups_per_cta"],
                      "wave": info["wave"], "resident_n_items": info["resident_n_items"]},
            "x0": "U[-0.9, 0.9] per instance (seed 3000); closed loops from x(0), warm start from the previous step"}


def learned_line(prob, args):
    """Learned warm start on the benchmark chain: training pairs from closed
    loops of the batched solver (random x(0), cold-start solutions), BF16
    training on the GPU, then held-out visited states solved from the same
    state with a cold and with a learned start to the same epsilon: ADMM
    iterations and MPC steps/s (whole step, network inference included)."""
    import numpy as np
    import torch
    import paper_2103_14990_gb300 as pkg
    from paper_2103_14990_gb300 import instances as I
    from paper_2103_14990_gb300 import warmstart as W
    t0 = time.time()
    # the first steps of a loop from x(0) ~ U[-0.9, 0.9] often cannot meet the
    # state box on some subsystem and stop at max_iter; pairs come from the
    # converged steps that follow
    pairs = W.closed_loop_pairs(prob, I.random_x0(prob.n_sub, args.learn_replicas, seed=1000),
                                steps=args.learn_steps, skip_first=args.learn_steps // 3)
    t_data = time.time() - t0
    t0 = time.time()
    mlp = W.train(pairs, hidden=256, epochs=args.learn_epochs, batch=2048, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    err = W.prediction_error(mlp, pairs)
    states, status = W.heldout_states(prob, seed=2000, trajectories=4, steps=args.learn_steps)
    keep = np.nonzero(status == 0)[0][::2]
    ic, il, sc, sl, _, _ = W.compare_starts(prob, mlp, states[keep])
    # MPC steps/s over the same held-out states, one instance, whole step timed
    s = pkg.Solver([prob])
    s.set_option(pkg.OPT_LEARN_PLANT, 1)
    s.attach_mlp(mlp)
    s.autotune(torch.tensor(prob.x0.astype(np.float32), device="cuda"), iters=0)
    xs = [torch.tensor(states[k].astype(np.float32), device="cuda") for k in keep]
    u = torch.empty(prob.n_sub, prob.nu, device="cuda")
    rates = {}
    for name, warm in (("cold", pkg.WARM_COLD), ("learned", pkg.WARM_LEARNED)):
        s.step(xs[0], u, None, warm=warm)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for x in xs:
            s.step(x, u, None, warm=warm)
        torch.cuda.synchronize()
        rates[name] = len(xs) / (time.perf_counter() - w0)
    s.close()
    return {"workload": prob.name, "train_pairs": int(pairs.feats.shape[0]), "train_steps_used": pairs.steps_used,
            "train_steps_skipped": pairs.steps_skipped,
            "epochs": args.learn_epochs, "data_s": round(t_data, 2), "train_s": round(t_train, 2),
            "train_rel_err": round(err, 4), "heldout_states": int(len(keep)),
            "iters_cold": round(float(ic.mean()), 2), "iters_learned": round(float(il.mean()), 2),
            "all_converged": bool(np.all(sc == 0) and np.all(sl == 0)),
            "steps_per_s_cold": round(rates["cold"], 2), "steps_per_s_learned": round(rates["learned"], 2),
            "note": "each held-out state solved twice from scratch (cold vs network start), eps 1e-4; "
                    "steps/s with host-side synchronisation per step"}


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_iters_table(workload_name: str):
    path = os.path.join(ROOT, "tests", "golden", "chain1024_oracle_iters.json")
    if workload_name != "chain1024" or not os.path.exists(path):
        return None
    return json.load(open(path))


def oracle_sample(workload_name: str, seconds: float, min_iters: int):
    """Times oracle ADMM iterations from x(0) for about `seconds`; returns
    (seconds per iteration, iterations timed, seconds per u+dynamics)."""
    import numpy as np
    from oracle import dlmpc_oracle as O
    prob = workload(workload_name)
    o = O.Oracle(prob)
    res = O.admm(o.lay, o.blocks, prob.x0, fixed_iters=1)  # warm the code path
    done, t0 = 0, time.perf_counter()
    Psi, Lam = res.Psi, res.Lam
    while done < min_iters or time.perf_counter() - t0 < seconds:
        r = O.admm(o.lay, o.blocks, prob.x0, Psi0=Psi, Lam0=Lam, fixed_iters=1)
        Psi, Lam = r.Psi, r.Lam
        done += 1
    t_iter = (time.perf_counter() - t0) / done
    t1 = time.perf_counter()
    u = o.control(r)
    o.dynamics(prob.x0, u)
    return t_iter, done, time.perf_counter() - t1


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _single_thread_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    return env


def cpu_baseline(args, gpu_iters):
    """The oracle on one host core, on a bounded sample of the same workload."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", args.workload,
           "--sample-seconds", str(args.sample_seconds)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=_single_thread_env(), timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    s = json.loads(r.stdout.strip().splitlines()[-1])
    table = oracle_iters_table(args.workload)
    if table is not None:
        its = table["previous"]["iters"][:args.steps]
        src = "oracle's own per-step iteration counts (tests/golden/chain1024_oracle_iters.json)"
    else:
        its = gpu_iters
        src = "the GPU run's per-step iteration counts"
    t = sum(i * s["t_iter"] + s["t_tail"] for i in its)
    return {"value": round(len(its) / t, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{s['iters']} FP64 oracle ADMM iterations from x(0) ({s['t_iter'] * 1e3:.1f} ms each, "
                      f"one thread), scaled by {src} over the {len(its)} timed steps; one-time precompute excluded",
            "oracle_admm_iters_per_s": round(1.0 / s["t_iter"], 3)}


def cpu_baseline_all_cores(args, gpu_iters, cores=None):
    """The oracle on every host core: one single-threaded oracle process per
    core, all timing the same bounded sample at once (the oracle's loops are
    serial numpy, so the host's cores are used by independent copies)."""
    cores = cores or min(os.cpu_count() or 1, 64)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", args.workload,
           "--sample-seconds", str(args.sample_seconds)]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=_single_thread_env()) for _ in range(cores)]
    rates, tails = [], []
    for pr in procs:
        out, err = pr.communicate(timeout=900)
        if pr.returncode != 0:
            return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": "failed: " + err[-300:]}
        r = json.loads(out.strip().splitlines()[-1])
        rates.append(1.0 / r["t_iter"])
        tails.append(r["t_tail"])
    table = oracle_iters_table(args.workload)
    its = table["previous"]["iters"][:args.steps] if table is not None else gpu_iters
    agg = sum(rates)                       # oracle ADMM iterations per second over all cores
    t = sum(i / agg + max(tails) / cores for i in its)
    return {"value": round(len(its) / t, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{cores} single-threaded oracle processes at once, each timing FP64 ADMM iterations from "
                      f"x(0) for {args.sample_seconds:g} s; aggregate {agg:.1f} iterations/s scaled by the same "
                      f"per-step iteration counts as cpu_baseline",
            "oracle_admm_iters_per_s": round(agg, 3)}


def run_oracle_sample(args):
    t_iter, done, t_tail = oracle_sample(args.workload, args.sample_seconds, 3)
    print(json.dumps({"t_iter": t_iter, "iters": done, "t_tail": t_tail}))


def reference_worker(args):
    """One single-threaded oracle process of the reference arm: warm-up, then
    the timed steps, each step 2 FP64 oracle ADMM iterations (+u, dynamics)
    from x(0) on its own state, scaled to that step's oracle iteration count.
    Prints the estimated seconds of the timed steps."""
    from oracle import dlmpc_oracle as O
    prob = workload(args.workload)
    o = O.Oracle(prob)
    its = oracle_iters_table(args.workload)["previous"]["iters"]
    per_step_sample = 2
    Psi = Lam = None

    def sample_step(tau):
        nonlocal Psi, Lam
        t0 = time.perf_counter()
        r = O.admm(o.lay, o.blocks, prob.x0, Psi0=Psi, Lam0=Lam, fixed_iters=per_step_sample)
        o.dynamics(prob.x0, o.control(r))
        Psi, Lam = r.Psi, r.Lam
        dt = time.perf_counter() - t0
        return dt / per_step_sample * its[tau % len(its)]

    for tau in range(args.warmup):
        sample_step(tau)
    total = sum(sample_step(tau) for tau in range(args.steps))
    print(json.dumps({"total": total}), flush=True)


def run_reference(args):
    """The oracle on the host cores: one single-threaded oracle process per
    core, each running the whole closed loop's steps as independent replicas
    (the oracle's loops are serial numpy), so the value is the MPC steps per
    second of all cores together."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = workload(args.workload)
    table = oracle_iters_table(args.workload) if (args.inner_qp == "box" and args.stale_prob == 0) else None
    if table is None:
        print(json.dumps({"impl": "reference", "unavailable": "no oracle iteration table for this workload"}))
        return
    cores = min(os.cpu_count() or 1, 64)
    cmd = [sys.executable, os.path.abspath(__file__), "--reference-worker", "--workload", args.workload,
           "--steps", str(args.steps), "--warmup", str(args.warmup)]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=_single_thread_env()) for _ in range(cores)]
    totals = []
    for pr in procs:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            print(json.dumps({"impl": "reference", "unavailable": "oracle worker failed: " + err[-200:]}))
            return
        totals.append(json.loads(out.strip().splitlines()[-1])["total"])
    value = sum(args.steps / t for t in totals)
    sample = (f"{cores} single-threaded oracle processes at once, each running the {args.steps} steps as an "
              f"independent replica; each step: 2 FP64 oracle ADMM iterations (+u, dynamics) from x(0), scaled "
              f"to that step's oracle iteration count from tests/golden/chain1024_oracle_iters.json")
    print(json.dumps({
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 / value, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded chain plant, x0 ~ U[-0.9,0.9])", "impl": "reference",
        "config": bench_config(prob, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="chain1024")
    ap.add_argument("--stale-prob", type=float, default=0.0,
                    help="probability that an exchange message is lost (the receiver keeps its value)")
    ap.add_argument("--inner-qp", choices=sorted(INNER_QP), default="box",
                    help="Phi-step cost/constraint form: box (default), block, coupled")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--batch", type=int, default=8, help="instances of the batched line (1: none)")
    ap.add_argument("--learn-replicas", type=int, default=8)
    ap.add_argument("--learn-steps", type=int, default=36)
    ap.add_argument("--learn-epochs", type=int, default=40)
    ap.add_argument("--ablation-iters", type=int, default=20)
    # the autotuner's fixed iteration count: near the steps' own (about 350 on
    # the chain) so that a plan's one-time prologue (bulk copies of resident
    # N) weighs as it does in the timed loop
    ap.add_argument("--tune-iters", type=int, default=200)
    ap.add_argument("--sample-seconds", type=float, default=15.0)
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--reference-worker", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not (args.oracle_sample or args.reference_worker):
        ap.error("--warmup must be >= 3")
    if args.oracle_sample:
        run_oracle_sample(args)
    elif args.reference_worker:
        reference_worker(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
