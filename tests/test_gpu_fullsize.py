"""Full-size workloads on the GPU, in the launch configuration the benchmark uses.

* chain N=1024, T=10, d=3, boxes: fixed-K parity of the whole state against
  the FP64 oracle (K = 40 iterations from x(0)).
* 64x64 grid, T=10, d=2: the precomputed operator of sampled patches (corner,
  edge, interior) against the oracle's projector.
* mixed batch of instances: sampled operators of several instances.
"""
import numpy as np
import pytest

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_chain1024_fixed_k_parity():
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.chain1024()
    s = pkg.Solver([p])
    K = 40
    s.set_option(pkg.OPT_FIXED_ITERS, K)
    s.set_option(pkg.OPT_EXPORT_PHI, 1)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    u = torch.zeros(p.n_sub, 1, device="cuda")
    xn = torch.zeros_like(x)
    rc, st = s.step(x, u, xn, warm=pkg.WARM_COLD)
    phi, psi, lam = [t.cpu().numpy() for t in s.get_state(phi=True)]
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    assert st[0]["iters"] == K
    assert rel(psi, ref.Psi) <= 1e-4
    assert rel(lam, ref.Lam) <= 1e-4
    assert rel(phi, ref.Phi) <= 1e-4
    u_ref = o.control(ref)
    assert rel(u.cpu().numpy(), u_ref) <= 1e-4
    s.close()


def _sampled_operator_check(p, js):
    import paper_2103_14990_gb300 as pkg
    s = pkg.Solver([p])
    for j in js:
        N, q = s.operator(j)
        blk = O.column_block(p, j)
        assert N.shape[1] == blk.P.shape[0] - blk.rank
        assert np.max(np.abs(N @ N.T - blk.P)) < 5e-6
        assert np.max(np.abs(q - blk.q)) < 5e-6
    s.close()


def test_grid64_sampled_operators():
    p = I.grid64()
    cols = 64
    js = [0, 63, 4095, 4032, 1, 64, 65, 2 * 64 + 2, 30 * 64 + 31, 64 * 10, 64 * 10 + 63, 4094]
    _sampled_operator_check(p, js)


def test_batch_sampled_operators():
    probs = [I.batch_instance(i) for i in range(6)]
    import paper_2103_14990_gb300 as pkg
    s = pkg.Solver(probs)
    off = 0
    for p in probs:
        for j in [0, p.n_sub // 2, p.n_sub - 1]:
            N, q = s.operator(off + j)
            blk = O.column_block(p, j)
            assert N.shape[1] == blk.P.shape[0] - blk.rank, p.name
            assert np.max(np.abs(N @ N.T - blk.P)) < 5e-6, p.name
            assert np.max(np.abs(q - blk.q)) < 5e-6, p.name
        off += p.n_sub
    s.close()
