#!/usr/bin/env python
"""DLMPC benchmark on GB300: closed-loop MPC steps/s of the N=1024 chain.

One "step" is one MPC step of Alg. 1 (per-step precompute, the whole ADMM of
Alg. 2 to convergence, u(tau), x(tau+1)) for the chain of 1024 subsystems,
T=10, d=3, |x| <= 1, |u| <= 2, x(0) ~ U[-0.9, 0.9] (seed 0), FP32 sweeps.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

Our arm: W warm-up steps, then the state is reset to x(0) and K closed-loop
steps are timed with CUDA events recorded by the library on its stream (the
L2 is flushed between steps by a 256 MiB write outside the timed events).
Headline: warm-started steps (the previous step's Psi/Lambda where that step
met Conv, zeros after a step stopped at max_iter); the same K steps with cold
starts ("plain"), with the previous step's state whatever its status
("warm_previous") and through the host-buffer C-ABI call ("e2e") are
reported beside it, with the mixed 256-instance batch (batched against one
context per instance) and the other workloads' closed loops.  N > 1: one independent replica per GPU, no
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
# the sweep kernel's source: its template and the device helpers it inlines
KERNEL_SRC = [os.path.join(ROOT, "paper_2103_14990_gb300", "csrc", f) for f in ("dlmpc_sweep.cuh", "dlmpc_common.cuh")]
# Counters of one sweep_kernel launch per workload from ncu captures of the
# kernel source whose sha256 is given (the capture commands are recorded with
# the profile summaries): DRAM bytes read + written, the iterations that
# launch ran, and the on-chip figures of the same kernel.  A workload without
# a capture of the current source reports null.
NCU = {
    "src_sha256": "3f742c50df985204ab7d47e1c040b0602b1ea05ab514b9a5c4d87eb0c043c5b3",
    "workloads": {
        # one bench-plan launch (7 groups of 96, 80-register tier) of 200
        # fixed iterations after an L2 flush: the operators come from DRAM
        # once per launch, the loop is served by shared memory and L2 (full
        # capture of 50 iterations, same plan)
        "chain1024": {"dram_bytes_per_launch": 63611136 + 765952, "iters_per_launch": 200,
                      "onchip": {"dram_throughput_pct": 1.43, "lts_throughput_pct": 19.86,
                                 "l2_hit_rate_pct": 92.66, "issue_active_pct": 41.3, "warps_active_pct": 32.8}},
        # 20 fixed iterations of the bench's plan (15 groups of 64, 64-register
        # tier): N and N^T streamed from DRAM every iteration
        "grid64": {"dram_bytes_per_launch": 13411877632 + 214867712, "iters_per_launch": 20,
                   "onchip": {"dram_throughput_pct": 45.3, "lts_throughput_pct": 29.0,
                              "l2_hit_rate_pct": 22.3, "issue_active_pct": 18.7, "warps_active_pct": 46.9}},
        # 64 of the 256 instances (a few GB on the device), 10 fixed
        # iterations of the bench's plan (8 groups of 128, 64-register tier);
        # scaled to the 256-instance launch by the algorithmic bytes (DRAM /
        # algorithmic = 1.89 on the 64-instance capture)
        "batch256": {"dram_bytes_per_launch": int(1.888 * 9889012444 * 20), "iters_per_launch": 20,
                     "scaled_from": "64-instance capture: 49100904960 B per 10 iterations, 2.60 GB algorithmic each",
                     "onchip": {"dram_throughput_pct": 39.2, "lts_throughput_pct": 25.1,
                                "l2_hit_rate_pct": 22.3, "issue_active_pct": 14.0, "warps_active_pct": 49.9}},
    },
}


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
            "warm_start": "previous MPC step's Psi/Lambda where that step met Conv, else zeros (step 0 cold)",
            "max_iter": prob.max_iter,
            "eps": prob.eps_p, "l2": "flushed between steps (256 MiB write outside the events)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def kernel_sha() -> str:
    """sha256 of the kernel source files, concatenated in order."""
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        h.update(open(path, "rb").read())
    return h.hexdigest()


def ncu_record(workload_name: str, inner_qp: str, stale_prob: float) -> dict:
    """`traffic` (DRAM bytes per launch, with the iterations of the captured
    launch) and the on-chip counters from the ncu capture of this workload, if
    it was taken on the current kernel source; null otherwise."""
    w = NCU["workloads"].get(workload_name)
    if w is None or NCU["src_sha256"] != kernel_sha() or inner_qp != "box" or stale_prob != 0:
        return {"traffic": None, "onchip": None}
    out = {"traffic": w["dram_bytes_per_launch"], "traffic_launch_iters": w["iters_per_launch"],
           "onchip": w.get("onchip")}
    if "scaled_from" in w:
        out["traffic_scaled_from"] = w["scaled_from"]
    return out


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


def closed_loop(solver, x0, K, warm, flush):
    """K closed-loop MPC steps of every instance of `solver` from x0 (step 0
    cold, the others `warm`): per step the library's CUDA-event times (sweep
    kernel, whole step; the L2 flushed before each step outside the events)
    and every instance's iterations and status."""
    import torch
    import paper_2103_14990_gb300 as pkg
    x = x0.clone()
    xn = torch.empty_like(x)
    u = torch.empty(x.shape[0], solver.nu, device="cuda")
    rec = {"kms": [], "sms": [], "iters": [], "status": []}
    for tau in range(K):
        if flush is not None:
            flush.zero_()
        rc, st = solver.step(x, u, xn, warm=(pkg.WARM_COLD if tau == 0 else warm), stats=True)
        a, b = solver.timing()
        rec["kms"].append(a)
        rec["sms"].append(b)
        rec["iters"].append([d["iters"] for d in st])
        rec["status"].append([d["status"] for d in st])
        x, xn = xn, x
    rec["x_final"] = x
    return rec


def merge_records(recs):
    """Records of several one-instance loops as one record of instance-steps
    (times add up; iterations and status side by side)."""
    out = {"kms": [], "sms": [], "iters": [], "status": []}
    K = len(recs[0]["sms"])
    for tau in range(K):
        out["kms"].append(sum(r["kms"][tau] for r in recs))
        out["sms"].append(sum(r["sms"][tau] for r in recs))
        out["iters"].append([r["iters"][tau][0] for r in recs])
        out["status"].append([r["status"][tau][0] for r in recs])
    return out


def summarise(rec, unit=UNIT):
    """MPC steps/s (instance-steps over the summed whole-step event time),
    ADMM iterations/s (instance iterations over the summed sweep-kernel time),
    iterations per instance-step, steps stopped at max_iter, and the same
    rates over the steps that converged."""
    import numpy as np
    K = len(rec["sms"])
    it = np.array(rec["iters"], dtype=np.float64)
    stt = np.array(rec["status"])
    n_inst = it.shape[1]
    s_step, s_kern = sum(rec["sms"]) / 1e3, sum(rec["kms"]) / 1e3
    out = {"value": round(n_inst * K / s_step, 3), "unit": unit, "steps": K,
           "ms_per_step": round(1e3 * s_step / K, 4),
           "admm_iters_per_s": round(float(it.sum()) / s_kern, 1),
           "iters_per_step": round(float(it.mean()), 2),
           "steps_at_max_iter": int((stt != 0).sum())}
    if n_inst > 1:
        out["launch_iters_per_step"] = round(float(it.max(axis=1).mean()), 2)
        # per MPC step: whole-step ms, mean iterations, instances at the cap
        out["by_step"] = [[round(rec["sms"][t], 3), round(float(it[t].mean()), 1), int((stt[t] != 0).sum())]
                          for t in range(K)]
    else:
        conv = [t for t in range(K) if rec["status"][t][0] == 0]
        if conv:
            cs = sum(rec["sms"][t] for t in conv) / 1e3
            ck = sum(rec["kms"][t] for t in conv) / 1e3
            ci = sum(rec["iters"][t][0] for t in conv)
            out["converged_steps"] = {"steps": len(conv), "value": round(len(conv) / cs, 3), "unit": unit,
                                      "admm_iters_per_s": round(ci / ck, 1),
                                      "iters_per_step": round(ci / len(conv), 2)}
    return out


def alg_roofline(info, rec, peak, peak_src):
    """HBM roofline of the sweep kernel by algorithmic bytes (every N_j once
    per iteration, the exchanged row sums and the compact iterate): bytes of
    the iterations run / sweep-kernel event time."""
    iters = sum(max(i) for i in rec["iters"])
    kern_s = sum(rec["kms"]) / 1e3
    achieved = info["iter_bytes_min"] * iters / kern_s / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_src,
            "algorithmic_bytes_per_iter": info["iter_bytes_min"],
            "kernel_load_bytes_per_iter": info["iter_bytes"],
            "mean_launch_ms": round(1e3 * kern_s / len(rec["kms"]), 4)}


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
        r = closed_loop(solver, x0, K, warm, flush)
        return r["kms"], r["sms"], [i[0] for i in r["iters"]], [s[0] for s in r["status"]], r["x_final"]

    def sync_all():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # warm-up (discarded), then the timed closed loops from x(0)
    loop(args.warmup, pkg.WARM_CONVERGED)
    sync_all()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        rec = closed_loop(solver, x0, args.steps, pkg.WARM_CONVERGED, flush)
        sync_all()
        wall = time.perf_counter() - wall0
    kms, sms = rec["kms"], rec["sms"]
    iters, status = [i[0] for i in rec["iters"]], [s[0] for s in rec["status"]]
    value, t_dev = replica_throughput(sum(sms) / 1e3, args.steps, world, dist, device="cuda")
    kern_s = sum(kms) / 1e3
    tot_iters = sum(iters)
    warm_summary = summarise(rec)

    # the same closed loop replayed from captured CUDA graphs (whole-step events)
    solver.set_option(pkg.OPT_GRAPH, 1)
    loop(2, pkg.WARM_CONVERGED)
    gk, gs, git, gst, _ = loop(args.steps, pkg.WARM_CONVERGED)
    solver.set_option(pkg.OPT_GRAPH, 0)
    graph = {"value": args.steps / (sum(gs) / 1e3), "unit": UNIT, "iters_per_step": sum(git) / len(git)}

    # plain: cold start at every step, same kernel
    plain = summarise(closed_loop(solver, x0, args.steps, pkg.WARM_COLD, flush))
    plain["start"] = "cold (zeros) at every step, one instance per launch"
    # the previous step's state whatever that step's status (also after a
    # step stopped at max_iter)
    warm_previous = summarise(closed_loop(solver, x0, args.steps, pkg.WARM_PREVIOUS, flush))

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
    other = rank == 0 and world == 1 and args.inner_qp == "box" and args.stale_prob == 0
    batched = batch_line(args, flush) if (other and not args.no_batch) else None
    configs = ({name: config_line(name, args, flush) for name in ("chain10", "grid64") if name != args.workload}
               if (other and not args.no_configs) else None)

    # e2e: host (pinned) buffers through the C ABI, H2D and D2H inside the timed region
    xh = torch.empty(n, nx, dtype=torch.float32, pin_memory=True)
    xnh = torch.empty(n, nx, dtype=torch.float32, pin_memory=True)
    uh = torch.empty(n, nu, dtype=torch.float32, pin_memory=True)
    xh.copy_(x0.cpu())
    sync_all()
    e0 = time.perf_counter()
    for tau in range(args.steps):
        solver.step_host_ptr(xh.data_ptr(), uh.data_ptr(), xnh.data_ptr(),
                             warm=(pkg.WARM_COLD if tau == 0 else pkg.WARM_CONVERGED))
        xh, xnh = xnh, xh
    e_wall = time.perf_counter() - e0
    e2e = {"value": args.steps / e_wall, "unit": UNIT, "h2d_bytes_per_step": n * nx * 4,
           "d2h_bytes_per_step": n * (nu + nx) * 4 + 32 + 16}

    # roofline of the sweep kernel: algorithmic bytes / CUDA-event kernel time
    peak, peak_src = measured_peaks()
    roofline = alg_roofline(info, rec, peak, peak_src)
    roofline["kernel"] = "sweep_kernel"
    roofline.update(ncu_record(args.workload, args.inner_qp, args.stale_prob))
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_dev / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded chain plant, x0 ~ U[-0.9,0.9])",
        "config": bench_config(prob, world, args.inner_qp, args.stale_prob),
        "admm_iters_per_s": round(tot_iters / kern_s, 1),
        "iters_per_step": round(tot_iters / args.steps, 2),
        "steps_at_max_iter": int(sum(1 for s in status if s != 0)),
        "converged_steps": warm_summary.get("converged_steps"),
        "plain": plain,
        "warm_previous": warm_previous,
        "e2e": e2e,
        "roofline": roofline,
        "graph": graph,
        "ablation": ablation,
        "learned": learned,
        "batched": batched,
        "configs": configs,
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


def config_line(name, args, flush):
    """Another workload's closed loop on its own: the autotuned launch, warm
    (previous step) against plain (cold) starts, the same number of steps."""
    import numpy as np
    import torch
    import paper_2103_14990_gb300 as pkg
    prob = workload(name)
    s = pkg.Solver([prob])
    x0 = torch.tensor(prob.x0.astype(np.float32), device="cuda")
    s.autotune(x0, iters=args.tune_iters)
    s.set_option(pkg.OPT_TIMING, 1)
    K = prob.mpc_steps
    closed_loop(s, x0, args.warmup, pkg.WARM_CONVERGED, flush)
    warm = closed_loop(s, x0, K, pkg.WARM_CONVERGED, flush)
    plain = closed_loop(s, x0, K, pkg.WARM_COLD, flush)
    info = s.info()
    peak, peak_src = measured_peaks()
    out = {"workload": prob.name, "steps": K, "warm": summarise(warm), "plain": summarise(plain),
           "roofline": {**alg_roofline(info, warm, peak, peak_src), **ncu_record(name, "box", 0.0)},
           "sweep": {"group_threads": info["group_threads"], "groups_per_cta": info["groups_per_cta"],
                     "wave": info["wave"], "resident_n_items": info["resident_n_items"]}}
    s.close()
    return out


def batch_line(args, flush):
    """The mixed batch of independent instances (chain or grid per seed, N in
    16..512, T in 5..15, d in 1..3, boxes): every instance's closed loop from
    its x(0) for the same steps, at the same eps --
    batched_warm: all instances in one context, one launch per MPC step (an
    instance rests once its ADMM has converged), previous-step warm starts;
    plain: one context per instance, one launch per instance per MPC step,
    cold starts (the plain one-instance form); with --batch-all-arms also the
    batched cold-start and the one-context warm-start forms.
    Rates are instance MPC steps per second of summed whole-step event time.
    A fixed-iteration launch of the batch (all instances active) gives the
    HBM roofline per ADMM iteration."""
    import numpy as np
    import torch
    import paper_2103_14990_gb300 as pkg
    from paper_2103_14990_gb300 import instances as I
    probs = I.batch256(args.batch_count)
    K = args.batch_steps
    t0 = time.time()
    sb = pkg.Solver(probs)
    torch.cuda.synchronize()
    t_setup_b = time.time() - t0
    xb = torch.tensor(np.concatenate([p.x0 for p in probs]).astype(np.float32), device="cuda")
    sb.autotune(xb, iters=20)
    sb.set_option(pkg.OPT_TIMING, 1)
    closed_loop(sb, xb, 1, pkg.WARM_COLD, flush)                   # warm-up
    w0 = time.perf_counter()
    bw = closed_loop(sb, xb, K, pkg.WARM_CONVERGED, flush)
    wall_bw = time.perf_counter() - w0
    bc = closed_loop(sb, xb, K, pkg.WARM_COLD, flush) if args.batch_all_arms else None
    # per-iteration roofline: fixed iterations from x(0), every instance active
    sb.set_option(pkg.OPT_FIXED_ITERS, 20)
    fixed = closed_loop(sb, xb, 2, pkg.WARM_COLD, flush)
    fixed = {k: v[1:] for k, v in fixed.items() if k != "x_final"}
    sb.set_option(pkg.OPT_FIXED_ITERS, 0)
    info = sb.info()
    sb.close()
    t0 = time.time()
    singles = [pkg.Solver([p]) for p in probs]
    torch.cuda.synchronize()
    t_setup_s = time.time() - t0
    for s in singles:
        s.set_option(pkg.OPT_TIMING, 1)
    xs = [torch.tensor(p.x0.astype(np.float32), device="cuda") for p in probs]
    for s, x in zip(singles, xs):
        closed_loop(s, x, 1, pkg.WARM_COLD, flush)                  # warm-up
    w0 = time.perf_counter()
    sc = merge_records([closed_loop(s, x, K, pkg.WARM_COLD, flush) for s, x in zip(singles, xs)])
    wall_sc = time.perf_counter() - w0
    sw = (merge_records([closed_loop(s, x, K, pkg.WARM_CONVERGED, flush) for s, x in zip(singles, xs)])
          if args.batch_all_arms else None)
    for s in singles:
        s.close()
    unit = "instance MPC steps/s"
    out = {"instances": len(probs), "steps": K, "n_sub_total": info["n_sub_total"],
           "batched_warm": summarise(bw, unit), "plain": summarise(sc, unit),
           "wall_s": {"batched_warm": round(wall_bw, 3), "plain": round(wall_sc, 3)},
           "setup_precompute_s": {"batched": round(t_setup_b, 2), "single_contexts": round(t_setup_s, 2)}}
    if args.batch_all_arms:
        out["batched_cold"] = summarise(bc, unit)
        out["single_warm"] = summarise(sw, unit)
        out["speedup_batched_cold_vs_plain"] = round(out["batched_cold"]["value"] / out["plain"]["value"], 3)
    out["speedup_batched_warm_vs_plain"] = round(out["batched_warm"]["value"] / out["plain"]["value"], 3)
    peak, peak_src = measured_peaks()
    out["roofline"] = {**alg_roofline(info, fixed, peak, peak_src), "iters_per_launch": 20,
                       **ncu_record("batch256", "box", 0.0)}
    out["sweep"] = {"group_threads": info["group_threads"], "groups_per_cta": info["groups_per_cta"],
                    "wave": info["wave"], "resident_n_items": info["resident_n_items"]}
    out["note"] = ("plain = one context per instance, one launch per instance per MPC step, cold starts; "
                   "every form stops on the same Conv at eps 1e-4 (max_iter 1000); x(0) ~ U[-0.9, 0.9] per "
                   "instance (seed = index)")
    return out


def learned_line(prob, args):
    """Learned warm start on the benchmark chain: training pairs from closed
    loops of the batched solver (random x(0), cold-start solutions), BF16
    training on the GPU, then the visited states of held-out closed loops
    solved from a cold, a learned and a previous-step start to the same
    epsilon: ADMM iterations and MPC steps/s (whole step, network inference
    included)."""
    import torch
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
    trajs, tstat = W.heldout_trajectories(prob, seed=2000, trajectories=args.learn_heldout, steps=args.learn_steps)
    ev = W.evaluate_starts(prob, mlp, trajs, tstat)
    starts = {}
    for name, d in ev.items():
        starts[name] = {"iters_per_step": round(float(d["iters"].mean()), 2),
                        "converged": int((d["status"] == 0).sum()),
                        "steps_per_s": round(len(d["ms"]) / (float(d["ms"].sum()) / 1e3), 2)}
    return {"workload": prob.name, "train_pairs": int(pairs.feats.shape[0]), "train_steps_used": pairs.steps_used,
            "train_steps_skipped": pairs.steps_skipped,
            "epochs": args.learn_epochs, "data_s": round(t_data, 2), "train_s": round(t_train, 2),
            "train_rel_err": round(err, 4), "heldout_states": int(len(ev["cold"]["iters"])),
            "heldout_trajectories": args.learn_heldout, "starts": starts,
            "iters_saved_vs_cold": round(1.0 - starts["learned"]["iters_per_step"] / starts["cold"]["iters_per_step"], 4),
            "note": "every visited state of held-out closed loops (x(0) ~ U[-0.9,0.9], seed 2000) whose cold solve "
                    "converges, solved to eps 1e-4 from a cold, a learned and a previous-step start on one "
                    "single-instance context; steps/s from whole-step CUDA events (network inference included)"}


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
        its = table["converged"]["iters"][:args.steps]
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
    its = table["converged"]["iters"][:args.steps] if table is not None else gpu_iters
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
    its = oracle_iters_table(args.workload)["converged"]["iters"]
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
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-batch comparison")
    ap.add_argument("--batch-count", type=int, default=256, help="instances of the mixed batch")
    ap.add_argument("--batch-steps", type=int, default=3, help="closed-loop MPC steps of the mixed batch")
    ap.add_argument("--batch-all-arms", action="store_true",
                    help="also the batched cold-start and one-context warm-start forms")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' lines")
    ap.add_argument("--learn-replicas", type=int, default=8)
    ap.add_argument("--learn-steps", type=int, default=36)
    ap.add_argument("--learn-epochs", type=int, default=40)
    ap.add_argument("--learn-heldout", type=int, default=6, help="held-out closed loops of the learned line")
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
