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


def _one_iteration_check(s, probs, samples, torch, K=9):
    """K iterations from x(0), then one more from the state left behind, in
    the launch configuration the autotuner picks.  The last iteration is
    checked against the oracle's steps: the Phi-step on every row, the
    Psi-step on sampled column patches (projection of the GPU's own Phi +
    Lambda_prev), the Lambda-step everywhere."""
    import paper_2103_14990_gb300 as pkg
    x = torch.tensor(np.concatenate([p.x0 for p in probs]).astype(np.float32), device="cuda")
    u = torch.zeros(x.shape[0], probs[0].nu, device="cuda")
    s.autotune(x, iters=4)
    s.set_option(pkg.OPT_EXPORT_PHI, 1)
    s.set_option(pkg.OPT_FIXED_ITERS, K)
    s.step(x, u, None, warm=pkg.WARM_COLD)
    _, psi0, lam0 = (a.cpu().numpy().astype(np.float64) if a is not None else None for a in s.get_state())
    s.set_option(pkg.OPT_FIXED_ITERS, 1)
    s.step(x, u, None, warm=pkg.WARM_PREVIOUS)
    phi1, psi1, lam1 = (a.cpu().numpy().astype(np.float64) for a in s.get_state(phi=True))
    off = 0
    for b, p in enumerate(probs):
        lay = O.Layout(p)
        sl = slice(off, off + lay.nnz)
        ref_phi, _ = O.phi_step(lay, psi0[sl], lam0[sl], p.x0, p.rho)
        assert rel(phi1[sl], ref_phi) <= 1e-4, p.name
        assert rel(lam1[sl], lam0[sl] + phi1[sl] - psi1[sl]) <= 1e-5, p.name
        for j in samples(b, p):
            blk = O.column_block(p, j)
            for a in range(p.nx):
                c = slice(off + lay.col_off[j * p.nx + a], off + lay.col_off[j * p.nx + a + 1])
                v = phi1[c] + lam0[c]
                assert rel(psi1[c], blk.P @ v + blk.q[a]) <= 1e-4, (p.name, j, a)
        off += lay.nnz
    assert off == phi1.size


def _compact_matches_full(s, probs, torch, K=20):
    """K iterations on the compact iterate against K in the full form."""
    import paper_2103_14990_gb300 as pkg
    x = torch.tensor(np.concatenate([p.x0 for p in probs]).astype(np.float32), device="cuda")
    u = torch.zeros(sum(p.n_sub for p in probs), probs[0].nu, device="cuda")
    out = []
    for compact in (1, 0):
        s.set_option(pkg.OPT_EXPORT_PHI, 0)
        s.set_option(pkg.OPT_COMPACT, compact)
        s.set_option(pkg.OPT_FIXED_ITERS, K)
        s.step(x, u, None, warm=pkg.WARM_COLD)
        _, psi, lam = s.get_state()
        out.append((psi.cpu().numpy(), lam.cpu().numpy(), u.cpu().numpy().copy()))
    s.set_option(pkg.OPT_COMPACT, 1)
    for a, b in zip(out[0], out[1]):
        assert rel(a, b) <= 1e-4


def test_grid64_sampled_iteration():
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.grid64()
    s = pkg.Solver([p])
    corners_edges = [0, 63, 4032, 4095, 1, 64, 2 * 64 + 2, 30 * 64 + 31, 64 * 10 + 63, 4094]
    _one_iteration_check(s, [p], lambda b, q: corners_edges, torch)
    _compact_matches_full(s, [p], torch)
    s.close()


def test_batch256_sampled_iteration():
    import torch
    import paper_2103_14990_gb300 as pkg
    probs = I.batch256()
    s = pkg.Solver(probs)
    picked = [0, 1, 17, 128, 255]
    # the Phi- and Lambda-steps of every instance, the Psi-step of a few
    # patches (ends, middle) of a few instances
    _one_iteration_check(s, probs, lambda b, q: ([0, q.n_sub // 2, q.n_sub - 1] if b in picked else []), torch)
    _compact_matches_full(s, probs, torch)
    s.close()
