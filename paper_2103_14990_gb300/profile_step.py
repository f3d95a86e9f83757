"""Runs a few MPC steps of one workload with a fixed sweep launch, for
profilers (ncu) and phase traces.

    python -m paper_2103_14990_gb300.profile_step --workload chain1024 \
        --iters 50 --shape 960701 --residency 2 --steps 3 [--trace] [--flush] [--inner-qp coupled]

--shape is threads per group * 10000 + groups per CTA * 100 + wave (0 keeps
the default plan); --iters runs exactly that many ADMM iterations per step
from a cold start.  Prints the plan, the kernel time of every step and, with
--trace, the median phase durations of the sweep over the CTAs.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="chain1024", choices=["chain1024", "chain10", "grid64", "batch256"])
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--shape", type=int, default=0)
    ap.add_argument("--residency", type=int, default=-1)
    ap.add_argument("--compact", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--trace", action="store_true")
    ap.add_argument("--flush", action="store_true", help="write 256 MiB before every step (L2 flushed, as in the benchmark)")
    ap.add_argument("--batch-count", type=int, default=256, help="instances of the mixed batch")
    ap.add_argument("--inner-qp", default="box", choices=["box", "block", "coupled"],
                    help="block: full SPD cost blocks; coupled: also 2 coupled state rows per slot")
    ap.add_argument("--network", action="store_true",
                    help="instead of sweeps: the learned start's network forward at the workload's sizes")
    a = ap.parse_args(argv)
    import torch
    import paper_2103_14990_gb300 as pkg
    from paper_2103_14990_gb300 import instances as I
    if a.network:
        return network_forward(a)
    probs = I.batch256(a.batch_count) if a.workload == "batch256" else \
        [{"chain1024": I.chain1024, "chain10": I.chain10, "grid64": I.grid64}[a.workload]()]
    if a.inner_qp == "block":
        probs = [I.with_block_costs(q, seed=101) for q in probs]
    elif a.inner_qp == "coupled":
        probs = [I.with_coupled_constraints(q, seed=102, n_cx=2, n_cu=0, g_range=(0.8, 1.2)) for q in probs]
    p = probs[0]
    s = pkg.Solver(probs)
    if a.shape > 0:
        s.set_option(pkg.OPT_SWEEP_SHAPE, a.shape)
    if a.residency >= 0:
        s.set_option(pkg.OPT_RESIDENCY, a.residency)
    s.set_option(pkg.OPT_COMPACT, a.compact)
    s.set_option(pkg.OPT_FIXED_ITERS, a.iters)
    s.set_option(pkg.OPT_TIMING, 1)
    if a.trace:
        s.set_option(pkg.OPT_TRACE, 1)
    info = s.info()
    print(json.dumps({k: info[k] for k in ("grid_ctas", "threads_per_cta", "group_threads", "groups_per_cta", "wave",
                                           "smem_bytes", "resident_n_items", "resident_state_items")}))
    x = torch.tensor(np.concatenate([q.x0 for q in probs]).astype(np.float32), device="cuda")
    u = torch.zeros(x.shape[0], p.nu, device="cuda")
    xn = torch.zeros_like(x)
    if a.shape == 0 and a.residency < 0:
        s.autotune(x, iters=5)
        info = s.info()
        print(json.dumps({"autotuned": {k: info[k] for k in ("group_threads", "groups_per_cta", "wave",
                                                              "resident_n_items", "iter_bytes_min")}}))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda") if a.flush else None
    for _ in range(a.steps):
        if flush is not None:
            flush.zero_()
        rc, st = s.step(x, u, xn, warm=pkg.WARM_COLD)
        ms = s.timing()[0]
        gbs = s.info()["iter_bytes_min"] * a.iters / (ms * 1e-3) / 1e9
        print(f"kernel {ms:.4f} ms  {1e3 * ms / a.iters:.2f} us/iteration  {gbs:.0f} GB/s algorithmic  "
              f"status {st[0]['status']}")
    if a.trace:
        tr = s.trace().astype(np.int64)
        # stamps: 0 top, 1 Phi-step, 7 pass 1 (+ y), 6 pass 2, 2 first patch done,
        # 3 all patches, 4 CTA synchronised, 5 grid barrier passed
        names = ["phi", "pass1", "pass2", "final", "rest", "cta_sync", "barrier"]
        pts = [(0, 1), (1, 7), (7, 6), (6, 2), (2, 3), (3, 4), (4, 5)]
        for it in range(1, tr.shape[1] - 1):
            ok = tr[:, it, 0] > 0
            row = [np.median((tr[ok, it, b] - tr[ok, it, a_]) / 1e3) for a_, b in pts]
            arr = (tr[ok, it, 4] - tr[ok, it, 0]) / 1e3
            tot = np.median((tr[ok, it + 1, 0] - tr[ok, it, 0]) / 1e3)
            print(f"iter {it}: " + " ".join(f"{n} {v:.2f}" for n, v in zip(names, row)) +
                  f" | arrival median {np.median(arr):.2f} max {np.max(arr):.2f} | total {tot:.2f} us")
    s.close()
    return 0


def network_forward(a) -> int:
    """The warm-start network (patch inputs -> 256 -> 256 -> Phi rows and
    Lambda) on one row per subsystem of the workload, `--steps` forward
    passes timed with CUDA events."""
    import torch
    import paper_2103_14990_gb300 as pkg
    from paper_2103_14990_gb300 import instances as I
    p = {"chain1024": I.chain1024, "chain10": I.chain10, "grid64": I.grid64}[a.workload]()
    s = pkg.Solver([p])
    s.set_option(pkg.OPT_LEARN_PLANT, 1)
    d_in, d_out = s.learned_dims()
    mlp = pkg.MLP(d_in, 256, d_out, seed=0)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    feats = s.learned_features(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.steps):
        e0.record()
        mlp.forward(feats)
        e1.record()
        torch.cuda.synchronize()
        print(f"network forward {p.n_sub} x {d_in} -> 256 -> 256 -> {d_out}: {1e3 * e0.elapsed_time(e1):.1f} us")
    mlp.close()
    s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
