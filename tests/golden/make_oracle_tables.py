"""Writes tests/golden/chain1024_oracle_iters.json from the FP64 oracle alone.

Per-MPC-step ADMM iteration counts (and u norms) of the 50-step closed loop
of the N=1024 chain (T=10, d=3, boxes, seed 0), for a cold start at every step
for a start from the previous step's Psi and Lambda, and for that start only
after a step that met Conv (zeros otherwise), and the closed-loop states
x(tau) at tau = 16, 20, 30 of each loop.  The benchmark's CPU
baseline and reference arm time bounded samples of oracle iterations and scale
them by these counts; the full-size parity tests start from those states.  Run: python tests/golden/make_oracle_tables.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def run(warm):
    import numpy as np
    from oracle import dlmpc_oracle as O
    from paper_2103_14990_gb300 import instances as I
    p = I.chain1024()
    o = O.Oracle(p)
    t0 = time.time()
    xs, us, its, stats = o.run_mpc(p.mpc_steps, warm=warm)
    keep = [16, 20, 30]
    return warm, {"iters": [int(i) for i in its],
                  # closed-loop states x(tau) of this loop at a few steps after
                  # the steps that cannot meet the state box (parity inputs)
                  "x_at": {str(t): [float(v) for v in xs[t].reshape(-1)] for t in keep},
                  "status": [int(s.status) for s in stats],
                  "r_max": [float(s.r_max) for s in stats],
                  "u_norm": [float(np.linalg.norm(u)) for u in us],
                  "x_final_norm": float(np.linalg.norm(xs[-1])),
                  "seconds": time.time() - t0}


if __name__ == "__main__":
    with mp.get_context("spawn").Pool(3) as pool:
        res = dict(pool.map(run, ["previous", "cold", "converged"]))
    out = {"workload": "chain_N1024_T10_d3_box seed 0, 50 closed-loop MPC steps, max_iter 1000",
           "writer": "tests/golden/make_oracle_tables.py (FP64 oracle only)", **res}
    with open(os.path.join(HERE, "chain1024_oracle_iters.json"), "w") as f:
        json.dump(out, f, indent=1)
    print({k: (sum(v["iters"]), v["seconds"]) for k, v in res.items()})
