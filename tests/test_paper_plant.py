"""The paper's own evaluation plant (Sec. IV-A) run through the oracle.

The paper prints the plant but no numeric outputs; the checks are the
invariants of Sec. II-A on that plant (two inputs per node here, B = I) and
the centralised optimum of the same locality-constrained problem."""
import json
import os

import numpy as np

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_plant(n, T, d, seed=0):
    g = json.load(open(os.path.join(HERE, "golden", "paper_plant.json")))
    ptr, idx = I.chain_graph(n)
    rng = np.random.default_rng(seed)
    nnz = int(ptr[-1])
    x_lo = np.tile([g["x1_min"], -np.inf], (n, 1))
    x_hi = np.tile([g["x1_max"], np.inf], (n, 1))
    return I.Problem(n_sub=n, nx=2, nu=2, T=T, d=d, adj_ptr=ptr, adj_idx=idx,
                     A_diag=np.tile(np.array(g["A_ii"]), (n, 1, 1)),
                     A_off=np.tile(np.array(g["A_ij"]), (nnz, 1, 1)),
                     B=np.tile(np.array(g["B_ii"]), (n, 1, 1)),
                     q=np.ones((n, 2)), r=np.ones((n, 2)), x_lo=x_lo, x_hi=x_hi,
                     u_lo=None, u_hi=None, rho=1.0, eps_p=1e-9, eps_d=1e-9,
                     max_iter=20000, x0=rng.uniform(-0.2, 1.2, (n, 2)), mpc_steps=g["T_sim"])


def test_paper_plant_closed_loop_invariants():
    p = paper_plant(6, 5, 1)
    p.u_lo = np.full((6, 2), -np.inf)
    p.u_hi = np.full((6, 2), np.inf)
    o = O.Oracle(p)
    for b in o.blocks:
        assert b.feas < 1e-12
    xs, us, its, stats = o.run_mpc(3, warm="previous")
    assert all(s.status == O.STATUS_CONVERGED for s in stats)
    Z = O.global_Z_AB(p)
    rhs = np.zeros((Z.shape[0], 12)); rhs[:12] = np.eye(12)
    for s in stats:
        assert np.max(np.abs(Z @ o.lay.to_dense(s.Psi) - rhs)) < 1e-10
    # first-state bound holds on the planned trajectory
    y = o.lay.trajectory(stats[0].Phi, xs[0])
    Nx = 12
    for t in range(1, p.T):
        assert np.all(y[t * Nx:(t + 1) * Nx:2] >= -0.2 - 1e-7)
        assert np.all(y[t * Nx:(t + 1) * Nx:2] <= 1.2 + 1e-7)
