"""Plant update in place (dlmpc_update_plant) against a fresh context of the
new plant: only the patches that see a changed subsystem are re-factorised,
and the result must be the same bits as setting the new plant up from
scratch (operators, iterates, the dynamics of x(tau+1)); a change that alters
a patch's null-space dimension is refused and leaves the context as it was.
"""
import copy
import time

import numpy as np
import pytest

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I
from parity_helpers import REL, rel

pytestmark = pytest.mark.gpu


def _new_rows(p, subs, seed):
    """A copy of p whose listed subsystems get redrawn A_ii (the chain
    plant's k_i, d_i), couplings a_ij on their CSR rows and B_i scaled."""
    rng = np.random.default_rng(seed)
    q = copy.deepcopy(p)
    for i in subs:
        k, dd = rng.uniform(0.5, 1.5), rng.uniform(0.1, 0.5)
        q.A_diag[i] = [[1.0, 0.1], [-0.1 * k, 1.0 - 0.1 * dd]]
        for e in range(q.adj_ptr[i], q.adj_ptr[i + 1]):
            a = rng.uniform(-0.1, 0.1)
            q.A_off[e] = [[0.0, 0.0], [a, a]]
        q.B[i] = q.B[i] * rng.uniform(0.8, 1.2)
    A_diag = np.stack([q.A_diag[i] for i in subs])
    A_off = np.concatenate([q.A_off[q.adj_ptr[i]:q.adj_ptr[i + 1]] for i in subs])
    B = np.stack([q.B[i] for i in subs])
    return q, A_diag, A_off, B


def _fixed(s, torch, x0, K, warm=0):
    import paper_2103_14990_gb300 as pkg
    s.set_option(pkg.OPT_FIXED_ITERS, K)
    x = torch.tensor(x0.astype(np.float32), device="cuda")
    u = torch.zeros(x.shape[0], 1, device="cuda")
    xn = torch.zeros_like(x)
    s.step(x, u, xn, warm=warm)
    _, psi, lam = s.get_state()
    s.set_option(pkg.OPT_FIXED_ITERS, 0)
    return psi.cpu().numpy(), lam.cpu().numpy(), u.cpu().numpy(), xn.cpu().numpy()


def test_update_plant_equals_a_fresh_context():
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.make_instance(32, 10, 3, seed=4, boxes=True)
    subs = [5, 20]
    q, A_diag, A_off, B = _new_rows(p, subs, seed=9)
    s = pkg.Solver([p])
    before = {j: s.operator(j) for j in (0, 12, 31)}
    _fixed(s, torch, p.x0, 10)                       # some state in the context
    n = s.update_plant(subs, A_diag, A_off, B)
    seen = sorted({j for i in subs for j in range(32) if abs(i - j) <= p.d + 1})
    assert n == len(seen) == 18
    fresh = pkg.Solver([q])
    for j in range(32):
        Na, qa = s.operator(j)
        Nb, qb = fresh.operator(j)
        assert np.array_equal(Na, Nb) and np.array_equal(qa, qb), j
        if j in before:                              # untouched patches keep their operators
            assert np.array_equal(Na, before[j][0]) and np.array_equal(qa, before[j][1])
    a = _fixed(s, torch, q.x0, 30)
    b = _fixed(fresh, torch, q.x0, 30)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    o = O.Oracle(q)
    ref = O.admm(o.lay, o.blocks, q.x0, fixed_iters=30)
    assert rel(a[0], ref.Psi) <= REL
    assert rel(a[2], o.control(ref)) <= REL
    assert np.max(np.abs(a[3].reshape(-1) - o.dynamics(q.x0, a[2]).reshape(-1))) < 1e-6
    s.close()
    fresh.close()


def test_update_plant_refuses_a_nullity_change():
    """B_5 = 0 changes the null-space dimension of two patches of this chain
    (the oracle's ranks say so); the update is refused and the context keeps
    its operators and gives the same iterates as before."""
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.make_instance(16, 10, 3, seed=1, boxes=True)
    q = copy.deepcopy(p)
    q.B[5] = 0.0
    k_old = [O.column_block(p, j).P.shape[0] - O.column_block(p, j).rank for j in range(16)]
    k_new = [O.column_block(q, j).P.shape[0] - O.column_block(q, j).rank for j in range(16)]
    assert k_old != k_new
    s = pkg.Solver([p])
    ops = [s.operator(j) for j in range(16)]
    a = _fixed(s, torch, p.x0, 20)
    with pytest.raises(pkg.DlmpcError) as e:
        s.update_plant([5], q.A_diag[5:6], q.A_off[q.adj_ptr[5]:q.adj_ptr[6]], q.B[5:6])
    assert e.value.code == pkg.DLMPC_ERR_ARG
    for j in range(16):
        N, qq = s.operator(j)
        assert np.array_equal(N, ops[j][0]) and np.array_equal(qq, ops[j][1])
    b = _fixed(s, torch, p.x0, 20)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    s.close()


def test_update_plant_is_cheaper_than_the_precompute():
    """One changed subsystem of the N = 1024 chain re-factorises the 9
    patches within d + 1 = 4 hops instead of all 1024."""
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.chain1024()
    s = pkg.Solver([p], precompute=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.precompute()
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    q, A_diag, A_off, B = _new_rows(p, [500], seed=3)
    t0 = time.perf_counter()
    n = s.update_plant([500], A_diag, A_off, B)
    t_upd = time.perf_counter() - t0
    assert n == 9
    print(f"precompute {t_full * 1e3:.1f} ms, update of one subsystem {t_upd * 1e3:.1f} ms")
    assert t_upd < 0.5 * t_full
    s.close()
