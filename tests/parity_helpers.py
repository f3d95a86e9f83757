"""Shared parity helpers of the GPU tests (test infrastructure).

* rel / max_patch_rel: relative errors, over the whole array and per column
  patch (the nx columns owned by one subsystem, on their patch support);
* stopped_closed_loop: stopped-run parity of a closed loop at a matched
  iteration count;
* parallel_oracle: the FP64 oracle of a large instance, its column blocks
  (the oracle's own `column_block`, unchanged) computed by a pool of spawned
  processes so that the full-size tests finish in about a minute.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import dlmpc_oracle as O

REL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def patch_norms(lay, vals, offset=0):
    """||vals_j|| per column subsystem j (entries offset.. of a concatenation)."""
    nx = lay.prob.nx
    v = np.asarray(vals[offset:offset + lay.nnz], np.float64)
    sq = np.bincount(lay.col_sub, weights=v * v, minlength=lay.prob.n_sub)
    return np.sqrt(sq)


def max_patch_rel(lay, got, ref, floor=1e-7, floor_vals=None, offset=0):
    """max over column subsystems j of ||got_j - ref_j|| / max(||ref_j||, f_j),
    f_j = floor, or floor * ||floor_vals_j|| when floor_vals is given (a
    quantity accumulated from differences of floor_vals-sized terms is
    compared against that size).  `got` may be a concatenation of instances
    starting at `offset`; `ref` is the oracle's own array."""
    d = patch_norms(lay, np.asarray(got[offset:offset + lay.nnz], np.float64) - ref)
    scale = patch_norms(lay, ref)
    f = floor * (patch_norms(lay, floor_vals) if floor_vals is not None else 1.0)
    return float(np.max(d / np.maximum(scale, np.maximum(f, 1e-30))))


def stopped_closed_loop(p, torch, warm_name, steps, iter_tol=0.02, check_next=False, tune_iters=None,
                        oracle=None, max_iter=None):
    """Stopped-run parity (Conv on) of a closed loop, both sides solving from
    the oracle's x(tau) at every MPC step.  Per step:
      1. the GPU stops on its own Conv: status converged and an iteration
         count within max(3, iter_tol) of the oracle's;
      2. the same step again from the same start with exactly the oracle's
         iteration count (mode (i)): u, Psi and Lambda within 1e-4 relative of
         the oracle's stopped result (per column patch for Psi); this run's
         state is the next step's warm start, so the two sides start every
         step from matching states;
      3. where the two stop counts agree, the stopped u itself within 1e-4.
    Two runs stopped a few iterations apart differ by about eps / ||u|| in u
    (both meet the stopping test, neither is the exact optimum), which is why
    the comparison at 1e-4 is made at a matched count.  Returns a summary."""
    import paper_2103_14990_gb300 as pkg
    o = oracle if oracle is not None else O.Oracle(p)
    xs, us, its, stats = o.run_mpc(steps, warm=warm_name, max_iter=max_iter)
    s = pkg.Solver([p])
    if max_iter is not None:
        s.set_option(pkg.OPT_MAX_ITER, max_iter)
    if tune_iters is not None:
        s.autotune(torch.tensor(p.x0.astype(np.float32), device="cuda"), iters=tune_iters)
    saved = None
    out = {"matched_counts": 0, "iters_gpu": [], "iters_oracle": list(its), "worst_u": 0.0, "worst_psi_patch": 0.0}
    for tau in range(steps):
        x = torch.tensor(xs[tau].astype(np.float32), device="cuda")
        warm = pkg.WARM_PREVIOUS if (tau > 0 and (warm_name == "previous" or (
            warm_name == "converged" and stats[tau - 1].status == O.STATUS_CONVERGED))) else pkg.WARM_COLD
        u = torch.zeros(p.n_sub, p.nu, device="cuda")
        xn = torch.zeros(p.n_sub, p.nx, device="cuda")
        if warm == pkg.WARM_PREVIOUS:
            s.set_state(*saved)
        rc, st = s.step(x, u, xn, warm=warm)
        assert st[0]["status"] == stats[tau].status, (tau, st)
        assert abs(st[0]["iters"] - its[tau]) <= max(3, iter_tol * its[tau]), (tau, st[0]["iters"], its[tau])
        out["iters_gpu"].append(st[0]["iters"])
        ug = u.cpu().numpy()
        if check_next:
            assert np.max(np.abs(xn.cpu().numpy().reshape(-1) - o.dynamics(xs[tau], ug).reshape(-1))) < 1e-6
        if st[0]["iters"] == its[tau]:
            out["matched_counts"] += 1
            assert rel(ug, us[tau]) <= REL or np.max(np.abs(ug - us[tau])) < 1e-7, (tau, rel(ug, us[tau]))
        # mode (i) at the oracle's count from the same start
        if warm == pkg.WARM_PREVIOUS:
            s.set_state(*saved)
        s.set_option(pkg.OPT_FIXED_ITERS, its[tau])
        u2 = torch.zeros_like(u)
        s.step(x, u2, None, warm=warm)
        s.set_option(pkg.OPT_FIXED_ITERS, 0)
        _, psi, lam = s.get_state()
        saved = (psi.clone(), lam.clone())
        u2 = u2.cpu().numpy()
        eu = rel(u2, us[tau])
        assert eu <= REL or np.max(np.abs(u2 - us[tau])) < 1e-7, (tau, eu)
        psi_n, lam_n = psi.cpu().numpy(), lam.cpu().numpy()
        assert rel(psi_n, stats[tau].Psi) <= REL, tau
        assert rel(lam_n, stats[tau].Lam) <= REL or np.linalg.norm(stats[tau].Lam) < 1e-6, tau
        ep = max_patch_rel(o.lay, psi_n, stats[tau].Psi)
        assert ep <= REL, (tau, ep)
        out["worst_u"] = max(out["worst_u"], eu)
        out["worst_psi_patch"] = max(out["worst_psi_patch"], ep)
    s.close()
    return out


# ---------------------------------------------------------------------------
# the oracle of a large instance, column blocks in spawned processes
# ---------------------------------------------------------------------------

def _blocks_of(args):
    p, js = args
    out = []
    for j in js:
        b = O.column_block(p, j)
        b.Z = None            # the iteration needs P and q only
        out.append(b)
    return out


def parallel_oracle(p, procs=None, dynamics=True):
    """O.Oracle(p) with the column blocks computed in `procs` spawned
    processes (single-threaded BLAS each).  The pool is started with spawn,
    so it is safe after the GPU has been used."""
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    o = O.Oracle.__new__(O.Oracle)
    o.prob = p
    o.lay = O.Layout(p)
    chunks = [list(range(a, min(a + 32, p.n_sub))) for a in range(0, p.n_sub, 32)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            parts = pool.map(_blocks_of, [(p, c) for c in chunks])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    o.blocks = [b for part in parts for b in part]
    o.A = p.dense_A() if dynamics else None
    o.Bm = p.dense_B() if dynamics else None
    return o
