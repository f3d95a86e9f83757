"""Pins of the FP64 oracle against facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: a brute-force
or library solver of the same optimisation problem, a closed form (Riccati,
Sherman-Morrison), an invariant of Sec. II-A (Z_AB Psi = I, Phi = Psi at
convergence, support inside L_d) or the Lemma of Sec. III-B.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I


# --------------------------------------------------------------------------
# Phi-step: one row of the box-QP (Alg. 2 Phi-comp)
# --------------------------------------------------------------------------

def _row_obj(phi, v, xh, q, rho):
    z = phi @ xh
    return q * z * z + 0.5 * rho * np.sum((phi - v) ** 2)


@pytest.mark.parametrize("seed", range(12))
def test_phi_row_matches_slsqp(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 7))
    v = rng.normal(size=n)
    xh = rng.normal(size=n)
    q = float(rng.uniform(0.2, 3.0))
    rho = float(rng.uniform(0.3, 3.0))
    lo, hi = sorted(rng.normal(size=2) * 0.5)
    got = O.phi_step_row(v, xh, q, rho, lo, hi)
    cons = [{"type": "ineq", "fun": lambda p: p @ xh - lo, "jac": lambda p: xh},
            {"type": "ineq", "fun": lambda p: hi - p @ xh, "jac": lambda p: -xh}]
    ref = scipy.optimize.minimize(
        _row_obj, v, args=(v, xh, q, rho),
        jac=lambda p, *a: 2 * q * (p @ xh) * xh + rho * (p - v),
        constraints=cons, method="SLSQP", options={"ftol": 1e-15, "maxiter": 500})
    assert ref.success
    assert np.allclose(got, ref.x, atol=1e-6)
    assert _row_obj(got, v, xh, q, rho) <= _row_obj(ref.x, v, xh, q, rho) + 1e-10
    # KKT: rho (phi - v) + (2 q z + mu) xh = 0, mu >= 0 at hi, <= 0 at lo, 0 inside
    z = got @ xh
    g = rho * (got - v) + 2 * q * z * xh
    mu = -(g @ xh) / (xh @ xh)
    assert np.allclose(g + mu * xh, 0, atol=1e-10)
    if lo + 1e-9 < z < hi - 1e-9:
        assert abs(mu) < 1e-9
    elif abs(z - hi) <= 1e-9:
        assert mu >= -1e-9
    else:
        assert abs(z - lo) <= 1e-9 and mu <= 1e-9


def test_phi_row_special_cases():
    rng = np.random.default_rng(7)
    v, xh = rng.normal(size=5), rng.normal(size=5)
    # no bounds: (rho I + 2 q xh xh^T) phi = rho v (Sherman-Morrison)
    q, rho = 1.3, 0.7
    got = O.phi_step_row(v, xh, q, rho, -np.inf, np.inf)
    ref = np.linalg.solve(rho * np.eye(5) + 2 * q * np.outer(xh, xh), rho * v)
    assert np.allclose(got, ref, atol=1e-12)
    # q = 0 and w inside the box: phi = v
    assert np.allclose(O.phi_step_row(v, xh, 0.0, rho, -1e9, 1e9), v)
    # xh = 0: phi = v
    assert np.allclose(O.phi_step_row(v, np.zeros(5), q, rho, -1.0, 1.0), v)
    # active bound: the row's output is exactly the bound
    big = v + 10 * xh / (xh @ xh)
    out = O.phi_step_row(big, xh, 0.01, rho, -0.5, 0.5)
    assert abs(out @ xh - 0.5) < 1e-12


def test_vectorised_phi_step_agrees_with_rows():
    p = I.make_instance(6, 4, 1, seed=3, boxes=True, x0_dist="uniform", x_bound=0.3, u_bound=0.2)
    lay = O.Layout(p)
    rng = np.random.default_rng(1)
    Psi, Lam = rng.normal(size=lay.nnz), rng.normal(size=lay.nnz)
    Phi, z = O.phi_step(lay, Psi, Lam, p.x0, p.rho)
    xf = p.x0.reshape(-1)
    for g in range(lay.n_rows):
        ent = np.nonzero(lay.rows == g)[0]
        ref = O.phi_step_row((Psi - Lam)[ent], xf[lay.cols[ent]], lay.qw[g], p.rho, lay.lo[g], lay.hi[g])
        assert np.allclose(Phi[ent], ref, atol=1e-12)
        assert abs(z[g] - ref @ xf[lay.cols[ent]]) < 1e-12


# --------------------------------------------------------------------------
# Psi-step: projection onto the achievability constraint (Alg. 2 Psi-comp)
# --------------------------------------------------------------------------

def _small_problems():
    return [I.chain10(), I.make_instance(9, 4, 1, graph="grid", seed=5),
            I.make_instance(7, 5, 2, graph="chain", seed=2)]


@pytest.mark.parametrize("k", range(3))
def test_projector_properties(k):
    p = _small_problems()[k]
    rng = np.random.default_rng(k)
    for j in range(p.n_sub):
        b = O.column_block(p, j)
        D = b.P.shape[0]
        assert b.feas < 1e-12
        assert np.allclose(b.P, b.P.T, atol=1e-10)
        assert np.allclose(b.P @ b.P, b.P, atol=1e-10)
        assert np.allclose(b.Z @ b.P, 0, atol=1e-10)
        Nul = scipy.linalg.null_space(b.Z)
        assert Nul.shape[1] == D - b.rank
        assert np.allclose(Nul @ Nul.T, b.P, atol=1e-10)
        for a in range(p.nx):
            ls = np.linalg.lstsq(b.Z, b.rhs[a], rcond=None)[0]
            assert np.allclose(ls, b.q[a], atol=1e-10)
            v = rng.normal(size=D)
            psi = b.P @ v + b.q[a]
            assert np.allclose(b.Z @ psi, b.rhs[a], atol=1e-11)
            assert np.allclose(Nul.T @ (psi - v), 0, atol=1e-10)


def test_constraint_block_counts():
    """Rows kept / rank / nullity of Z_j, derived by hand for the chain plant.

    Interior chain subsystem, d hops: the patch has 2d+1 members and the ring
    adds 2 more.  Rows kept = nx*T per patch member, plus per ring-only member
    the T-1 second-state rows (its first-state rows and its slot-0 rows have
    no patch variable).  Each ring-only member makes its slot-1 row redundant
    with the slot-0 rows of the patch, so rank = rows - 2.  Ends lose one ring
    member and one redundancy.
    """
    for (T, d) in [(5, 1), (10, 3), (15, 3)]:
        p = I.make_instance(4 * d + 6, T, d, seed=0)
        rs = 3 * T - 1
        mid = O.column_block(p, 2 * d + 3)
        npatch = 2 * d + 1
        rows = 2 * T * npatch + 2 * (T - 1)
        assert mid.Z.shape == (rows, rs * npatch)
        assert mid.rank == rows - 2
        end = O.column_block(p, 0)
        rows_e = 2 * T * (d + 1) + (T - 1)
        assert end.Z.shape == (rows_e, rs * (d + 1))
        assert end.rank == rows_e - 1


# --------------------------------------------------------------------------
# Lemma of Sec. III-B: D_row and D_col bounds
# --------------------------------------------------------------------------

@pytest.mark.parametrize("graph,n,T,d", [("chain", 20, 5, 1), ("chain", 30, 10, 3),
                                         ("grid", 49, 10, 2), ("grid", 36, 6, 3),
                                         ("grid", 27, 5, 1)])
def test_lemma_bounds(graph, n, T, d):
    p = I.make_instance(n, T, d, graph=graph, seed=1)
    l = max(int(p.adj_ptr[i + 1] - p.adj_ptr[i]) for i in range(n))
    s = max(p.nx, p.nu)
    brow, bcol = O.lemma_bounds(s, l, d, T)
    for j in range(n):
        m = len(O.patch_members(p, j))
        assert p.nx * m <= brow                 # D_row: entries of one Phi row
        assert p.r_sub * m <= bcol              # D_col: entries of one Psi column


# --------------------------------------------------------------------------
# Whole ADMM against the centralised problem
# --------------------------------------------------------------------------

def _support_mask(p):
    lay = O.Layout(p)
    M = np.zeros((lay.n_rows, p.n_sub * p.nx), bool)
    M[lay.rows, lay.cols] = True
    return lay, M


def _centralised_affine(p, x0):
    """y = y0 + G theta over every Phi in L_d with Z_AB Phi = I (all rows of Z_AB)."""
    Z = O.global_Z_AB(p)
    lay, M = _support_mask(p)
    ncol = p.n_sub * p.nx
    y0 = np.zeros(lay.n_rows)
    blocks = []
    for c in range(ncol):
        idx = np.nonzero(M[:, c])[0]
        Zc = Z[:, idx]
        e = np.zeros(Z.shape[0]); e[c] = 1.0
        part = np.linalg.lstsq(Zc, e, rcond=None)[0]
        assert np.allclose(Zc @ part, e, atol=1e-10)
        Nc = scipy.linalg.null_space(Zc)
        col = np.zeros(lay.n_rows); col[idx] = part
        y0 += x0.reshape(-1)[c] * col
        Gc = np.zeros((lay.n_rows, Nc.shape[1])); Gc[idx] = Nc
        blocks.append(x0.reshape(-1)[c] * Gc)
    return lay, y0, np.hstack(blocks)


@pytest.mark.parametrize("rho", [1.0, 0.7, 2.5])
def test_admm_matches_centralised_least_squares(rho):
    """The fixed point of ADMM does not depend on rho: every rho reaches the
    centralised optimum (a rho used inconsistently between the Phi-step and
    the dual update would move the fixed point)."""
    p = I.make_instance(5, 4, 1, seed=11, boxes=False, x0_dist="normal", rho=rho)
    lay, y0, G = _centralised_affine(p, p.x0)
    W = np.sqrt(lay.qw)
    theta = np.linalg.lstsq(W[:, None] * G, -W * y0, rcond=None)[0]
    y_ref = y0 + G @ theta
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=20000, eps_p=1e-11, eps_d=1e-11)
    assert res.status == O.STATUS_CONVERGED
    y = o.lay.trajectory(res.Phi, p.x0)
    assert np.allclose(y, y_ref, atol=1e-8)


@pytest.mark.parametrize("rho", [1.0, 0.7, 2.5])
def test_admm_matches_centralised_boxed_qp(rho):
    """Boxed case, for several rho.  The trajectory lives in y0 + range(G); with an orthonormal
    basis Bm of range(G) the centralised QP is strictly convex in phi.  Its
    dual (lambda >= 0) is solved by L-BFGS-B; the active set it exposes is then
    solved exactly as an equality-constrained KKT system, whose multipliers
    must carry the right signs.  The instance is feasible and its unconstrained
    optimum violates the box, so the box is exercised."""
    p = I.make_instance(4, 4, 1, seed=3, boxes=True, x0_dist="uniform", x_bound=1.0, u_bound=0.1, rho=rho)
    p.x0 = 0.9 * p.x0
    lay, y0, G = _centralised_affine(p, p.x0)
    U, S, _ = np.linalg.svd(G, full_matrices=False)
    Bm = U[:, S > 1e-10 * S[0]]
    bnd = np.isfinite(lay.lo)
    assert np.array_equal(bnd, np.isfinite(lay.hi))
    C = np.vstack([Bm[bnd], -Bm[bnd]])                       # C phi <= b
    b = np.concatenate([lay.hi[bnd] - y0[bnd], y0[bnd] - lay.lo[bnd]])
    W = lay.qw
    H = 2 * Bm.T @ (W[:, None] * Bm)
    f = 2 * Bm.T @ (W * y0)
    Hinv = np.linalg.inv(H)
    phi_unc = -Hinv @ f
    assert np.max(C @ phi_unc - b) > 1e-3, "unconstrained optimum must violate the box"
    M = C @ Hinv @ C.T
    g0 = C @ Hinv @ f + b
    dual = scipy.optimize.minimize(lambda l: 0.5 * l @ M @ l + g0 @ l, np.zeros(len(b)),
                                   jac=lambda l: M @ l + g0, method="L-BFGS-B",
                                   bounds=[(0, None)] * len(b),
                                   options={"ftol": 1e-16, "gtol": 1e-13, "maxiter": 20000})
    act = dual.x > 1e-7
    assert act.sum() >= 1
    Ca, ba = C[act], b[act]
    nC = Ca.shape[0]
    K = np.block([[H, Ca.T], [Ca, np.zeros((nC, nC))]])
    sol = np.linalg.solve(K, np.concatenate([-f, ba]))
    phi, lam = sol[:H.shape[0]], sol[H.shape[0]:]
    assert np.all(lam >= -1e-10)                              # dual feasibility
    assert np.all(C @ phi <= b + 1e-10)                       # primal feasibility
    y_ref = y0 + Bm @ phi
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=50000, eps_p=1e-10, eps_d=1e-10)
    assert res.status == O.STATUS_CONVERGED
    y = o.lay.trajectory(res.Phi, p.x0)
    assert np.allclose(y, y_ref, atol=1e-6)
    assert abs(np.sum(W * y * y) - np.sum(W * y_ref * y_ref)) < 1e-8


def _riccati_u0(A, B, Q, R, T, x0):
    P = Q.copy()                           # P_{T-1} = Q (last state slot)
    for _ in range(T - 2):                 # P_{T-2} .. P_1
        S = R + B.T @ P @ B
        P = Q + A.T @ P @ A - A.T @ P @ B @ np.linalg.solve(S, B.T @ P @ A)
    return -np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A @ x0)


@pytest.mark.parametrize("n,T", [(3, 4), (4, 5)])
def test_admm_matches_riccati_without_locality(n, T):
    """d >= N-1 removes locality; with no boxes u(0) is the finite-horizon LQR
    gain applied to x0.  Non-identity diagonal Q, R (with Q = R = I the
    min-norm projection alone already gives the LQR map)."""
    p = I.make_instance(n, T, n - 1, seed=21, boxes=False, x0_dist="normal")
    rng = np.random.default_rng(5)
    p.q = rng.uniform(0.3, 3.0, p.q.shape)
    p.r = rng.uniform(0.3, 3.0, p.r.shape)
    A, B = p.dense_A(), p.dense_B()
    u_ref = _riccati_u0(A, B, np.diag(p.q.reshape(-1)), np.diag(p.r.reshape(-1)), T, p.x0.reshape(-1))
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=50000, eps_p=1e-11, eps_d=1e-11)
    assert res.status == O.STATUS_CONVERGED
    assert np.allclose(o.control(res).reshape(-1), u_ref, atol=1e-8)


@pytest.mark.parametrize("k", range(3))
def test_invariants_after_admm(k):
    p = _small_problems()[k]
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=20000, eps_p=1e-9, eps_d=1e-9)
    assert res.status == O.STATUS_CONVERGED
    Z = O.global_Z_AB(p)
    Psi = o.lay.to_dense(res.Psi)
    rhs = np.zeros((Z.shape[0], p.n_sub * p.nx)); rhs[:p.n_sub * p.nx] = np.eye(p.n_sub * p.nx)
    assert np.max(np.abs(Z @ Psi - rhs)) < 1e-10          # Z_AB Psi = I
    assert np.max(np.abs(res.Phi - res.Psi)) < 1e-8      # Phi = Psi at convergence
    # support inside L_d: every stored entry links subsystems at most d hops apart
    near = {i: O.hop_distances(p, i, p.d) for i in range(p.n_sub)}
    assert all(int(c) in near[int(r)] for r, c in zip(o.lay.row_sub, o.lay.col_sub))
    y = o.lay.trajectory(res.Phi, p.x0)
    assert np.all(y <= o.lay.hi + 1e-8) and np.all(y >= o.lay.lo - 1e-8)


def test_dual_update_and_closed_loop_dynamics():
    p = I.chain10()
    o = O.Oracle(p)
    r1 = O.admm(o.lay, o.blocks, p.x0, fixed_iters=1)
    r2 = O.admm(o.lay, o.blocks, p.x0, fixed_iters=2)
    Phi2, _ = O.phi_step(o.lay, r1.Psi, r1.Lam, p.x0, p.rho)
    assert np.allclose(r2.Lam, r1.Lam + Phi2 - r2.Psi, atol=1e-13)  # Lambda-comp
    xs, us, its, _ = o.run_mpc(2, warm="cold")
    A, B = p.dense_A(), p.dense_B()
    assert np.allclose(xs[1].reshape(-1), A @ p.x0.reshape(-1) + B @ us[0].reshape(-1))


# --------------------------------------------------------------------------
# Planted mistakes: each one must be caught by a pin above
# --------------------------------------------------------------------------

def test_planted_dropped_cost_is_caught(monkeypatch):
    p = I.make_instance(3, 4, 2, seed=21, boxes=False, x0_dist="normal")
    orig = O.phi_step
    def bad(lay, Psi, Lam, x0, rho, w=None):
        saved = lay.qw.copy(); lay.qw[:] = 0.0
        try:
            return orig(lay, Psi, Lam, x0, rho, w=w)
        finally:
            lay.qw[:] = saved
    monkeypatch.setattr(O, "phi_step", bad)
    with pytest.raises(AssertionError):
        test_admm_matches_riccati_without_locality(3, 4)


def test_planted_missing_ring_rows_is_caught(monkeypatch):
    orig = O.ring_members
    monkeypatch.setattr(O, "ring_members", lambda prob, j: O.patch_members(prob, j))
    with pytest.raises(AssertionError):
        test_invariants_after_admm(0)
    monkeypatch.setattr(O, "ring_members", orig)


def test_planted_transposed_coupling_is_caught(monkeypatch):
    orig = O.z_row_coeffs
    def bad(prob, i, t, a):
        out = orig(prob, i, t, a)
        return [((k, r), (-val if (k != i and val != 0) else val)) for (k, r), val in out]
    monkeypatch.setattr(O, "z_row_coeffs", bad)
    with pytest.raises(AssertionError):
        test_dual_update_and_closed_loop_dynamics_consistency()


def test_dual_update_and_closed_loop_dynamics_consistency():
    """Z_AB rows must reproduce the plant: the slot-1 row of Psi x0 equals A x0 + B u_0."""
    p = I.make_instance(6, 4, 5, seed=8, boxes=False, x0_dist="normal")
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=20000, eps_p=1e-10, eps_d=1e-10)
    y = o.lay.trajectory(res.Psi, p.x0)
    Nx = p.n_sub * p.nx
    x1 = y[Nx:2 * Nx]
    u0 = y[p.T * Nx:p.T * Nx + p.n_sub]
    assert np.allclose(x1, p.dense_A() @ p.x0.reshape(-1) + p.dense_B() @ u0, atol=1e-8)


# --------------------------------------------------------------------------
# Full cost blocks Q_i, R_i (box-QP Phi-step)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_box_qp_matches_bounded_minimiser(seed):
    rng = np.random.default_rng(seed)
    n = 1 + seed % 4
    M = rng.normal(size=(n, n))
    H = M @ M.T + 0.2 * np.eye(n)
    c = rng.normal(size=n) * 3
    lo = np.where(rng.random(n) < 0.8, -rng.uniform(0.1, 1.0, n), -np.inf)
    hi = np.where(rng.random(n) < 0.8, rng.uniform(0.1, 1.0, n), np.inf)
    z = O.box_qp(H, c, lo, hi)
    ref = scipy.optimize.minimize(lambda v: 0.5 * v @ H @ v - c @ v, np.clip(np.zeros(n), lo, hi),
                                  jac=lambda v: H @ v - c, method="L-BFGS-B",
                                  bounds=[(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
                                          for a, b in zip(lo, hi)],
                                  options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    assert np.allclose(z, ref.x, atol=1e-6)
    f = lambda v: 0.5 * v @ H @ v - c @ v
    assert f(z) <= f(ref.x) + 1e-12


def test_box_qp_diagonal_is_the_clamp():
    rng = np.random.default_rng(1)
    d = rng.uniform(0.5, 3.0, 4)
    c = rng.normal(size=4) * 2
    lo, hi = np.array([-0.3, -np.inf, -1.0, -0.2]), np.array([0.3, 0.5, np.inf, 0.1])
    assert np.allclose(O.box_qp(np.diag(d), c, lo, hi), np.clip(c / d, lo, hi), atol=1e-14)


def test_block_phi_step_with_diagonal_blocks_equals_row_step():
    p = I.make_instance(6, 4, 1, seed=8, boxes=True, x0_dist="uniform", x_bound=0.6, u_bound=0.3)
    rng = np.random.default_rng(2)
    p.q = rng.uniform(0.5, 2.0, p.q.shape)
    p.r = rng.uniform(0.5, 2.0, p.r.shape)
    lay = O.Layout(p)
    Psi, Lam = rng.normal(size=lay.nnz), rng.normal(size=lay.nnz) * 0.3
    a, za = O.phi_step(lay, Psi, Lam, p.x0, p.rho)
    b, zb = O.phi_step_block(lay, Psi, Lam, p.x0, p.rho)
    assert np.allclose(a, b, atol=1e-12) and np.allclose(za, zb, atol=1e-12)


@pytest.mark.parametrize("n,T", [(3, 4), (4, 5)])
def test_block_cost_admm_matches_riccati(n, T):
    """d >= N-1, no boxes, full blocks Q_i, R_i: u(0) of the ADMM equals the
    finite-horizon LQR gain with block-diagonal Q = diag(Q_i), R = diag(R_i)."""
    p = I.with_block_costs(I.make_instance(n, T, n - 1, seed=21, boxes=False, x0_dist="normal"), seed=9)
    A, B = p.dense_A(), p.dense_B()
    Q = scipy.linalg.block_diag(*p.Q_blk)
    R = scipy.linalg.block_diag(*p.R_blk)
    u_ref = _riccati_u0(A, B, Q, R, T, p.x0.reshape(-1))
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=50000, eps_p=1e-11, eps_d=1e-11)
    assert res.status == O.STATUS_CONVERGED
    assert np.allclose(o.control(res).reshape(-1), u_ref, atol=1e-8)


def test_block_cost_admm_matches_centralised_boxed_qp():
    """Full blocks and boxes: the converged trajectory solves the centralised
    QP min y^T W y over the locality-constrained affine set with the box, W
    block-diagonal over (subsystem, slot); checked by the KKT conditions of
    that QP at the ADMM solution (stationarity on the free set, multiplier
    signs on the active box rows)."""
    base = I.make_instance(4, 4, 1, seed=3, boxes=True, x0_dist="uniform", x_bound=1.0, u_bound=0.1)
    base.x0 = 0.9 * base.x0
    p = I.with_block_costs(base, seed=4)
    lay, y0, G = _centralised_affine(p, p.x0)
    U, S, _ = np.linalg.svd(G, full_matrices=False)
    Bm = U[:, S > 1e-10 * S[0]]
    W = np.zeros((lay.n_rows, lay.n_rows))
    for i in range(p.n_sub):
        for t in range(p.T):
            rr = [O.global_row(p, i, t * p.nx + a) for a in range(p.nx)]
            W[np.ix_(rr, rr)] = p.Q_blk[i]
        for t in range(p.T - 1):
            rr = [O.global_row(p, i, p.nx * p.T + t * p.nu + b) for b in range(p.nu)]
            W[np.ix_(rr, rr)] = p.R_blk[i]
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=50000, eps_p=1e-10, eps_d=1e-10)
    assert res.status == O.STATUS_CONVERGED
    y = o.lay.trajectory(res.Phi, p.x0)
    # y = y0 + Bm phi, feasible
    phi = Bm.T @ (y - y0)
    assert np.allclose(y0 + Bm @ phi, y, atol=1e-8)
    assert np.all(y <= lay.hi + 1e-8) and np.all(y >= lay.lo - 1e-8)
    # KKT: 2 Bm^T W y + Bm^T (mu_hi - mu_lo) = 0 with mu >= 0 on the active rows only
    grad = 2 * Bm.T @ (W @ y)
    at_hi = np.isfinite(lay.hi) & (y >= lay.hi - 1e-7)
    at_lo = np.isfinite(lay.lo) & (y <= lay.lo + 1e-7)
    assert (at_hi | at_lo).sum() >= 1, "the box must be active"
    C = np.hstack([Bm[at_hi].T, -Bm[at_lo].T])
    mu = np.linalg.lstsq(C, -grad, rcond=None)[0]
    assert np.allclose(C @ mu, -grad, atol=1e-6)
    assert np.all(mu >= -1e-6)


@pytest.mark.parametrize("seed", range(4))
def test_block_phi_step_matches_slsqp_on_the_slot_problem(seed):
    """One time slot of one subsystem, solved directly in the Phi entries:
    min (Phi_s xh)^T C (Phi_s xh) + rho/2 ||Phi_s - V_s||_F^2 s.t. the box on
    Phi_s xh, with SLSQP over all nx (or nu) rows of the slot at once; the block
    Phi-step's rows must agree (this fixes the factor between the cost and the
    penalty, which a converged solution alone does not see)."""
    p = I.with_block_costs(I.make_instance(5, 4, 1, seed=seed, boxes=True, x0_dist="uniform",
                                           x_bound=0.4, u_bound=0.2), seed=seed + 10, coupling=0.8)
    rng = np.random.default_rng(seed)
    lay = O.Layout(p)
    Psi, Lam = rng.normal(size=lay.nnz) * 0.7, rng.normal(size=lay.nnz) * 0.3
    Phi, _ = O.phi_step_block(lay, Psi, Lam, p.x0, p.rho)
    V = Psi - Lam
    xf = p.x0.reshape(-1)
    i = 2
    for rows, C in [([O.global_row(p, i, 1 * p.nx + a) for a in range(p.nx)], p.Q_blk[i]),
                    ([O.global_row(p, i, p.nx * p.T + 0 * p.nu + b) for b in range(p.nu)], p.R_blk[i])]:
        sel = [np.nonzero(lay.rows == r)[0] for r in rows]
        cols = [lay.cols[e] for e in sel]
        xh = [xf[c] for c in cols]
        v = [V[e] for e in sel]
        sizes = [len(e) for e in sel]

        def unpack(theta):
            out, o = [], 0
            for k in sizes:
                out.append(theta[o:o + k]); o += k
            return out

        def f(theta):
            ph = unpack(theta)
            z = np.array([ph[a] @ xh[a] for a in range(len(rows))])
            return z @ C @ z + 0.5 * p.rho * sum(np.sum((ph[a] - v[a]) ** 2) for a in range(len(rows)))

        cons = []
        for a, r in enumerate(rows):
            if np.isfinite(lay.hi[r]):
                cons.append({"type": "ineq", "fun": (lambda th, a=a, r=r: lay.hi[r] - unpack(th)[a] @ xh[a])})
                cons.append({"type": "ineq", "fun": (lambda th, a=a, r=r: unpack(th)[a] @ xh[a] - lay.lo[r])})
        res = scipy.optimize.minimize(f, np.concatenate(v), method="SLSQP", constraints=cons,
                                      options={"ftol": 1e-14, "maxiter": 2000})
        assert res.success
        got = np.concatenate([Phi[e] for e in sel])
        assert np.allclose(got, res.x, atol=1e-6), (seed, rows)
        assert f(got) <= res.fun + 1e-9


# --------------------------------------------------------------------------
# Coupled per-slot constraints: the slot QP over a polytope (poly_qp)
# --------------------------------------------------------------------------

def _spd(rng, n):
    M = rng.normal(size=(n, n))
    return M @ M.T + 0.3 * np.eye(n)


@pytest.mark.parametrize("seed", range(10))
def test_poly_qp_matches_slsqp(seed):
    """Random strictly convex QPs with a few half-spaces (0 strictly feasible)
    against scipy's SLSQP; the linear term is scaled so that some rows bind."""
    rng = np.random.default_rng(100 + seed)
    n = 1 + seed % 4
    m = 2 + seed % 5
    H = _spd(rng, n)
    c = 4.0 * rng.normal(size=n)
    A = rng.normal(size=(m, n))
    b = rng.uniform(0.2, 1.0, m)
    z = O.poly_qp(H, c, A, b)
    f = lambda v: 0.5 * v @ H @ v - c @ v
    res = scipy.optimize.minimize(f, np.zeros(n), jac=lambda v: H @ v - c, method="SLSQP",
                                  constraints=[{"type": "ineq", "fun": lambda v: b - A @ v,
                                                "jac": lambda v: -A}],
                                  options={"ftol": 1e-13, "maxiter": 1000})
    # SLSQP may stop on its line search this close to the optimum: its point
    # must still be feasible, and the enumeration's point no worse
    assert np.all(A @ res.x <= b + 1e-8)
    assert np.all(A @ z <= b + 1e-10)
    assert np.allclose(z, res.x, atol=1e-5)
    assert f(z) <= f(res.x) + 1e-10
    z_unc = np.linalg.solve(H, c)
    if np.any(A @ z_unc > b):                     # the unconstrained optimum is cut off
        assert np.max(A @ z - b) > -1e-9         # so some row binds


@pytest.mark.parametrize("seed", range(6))
def test_poly_qp_with_box_rows_is_box_qp(seed):
    rng = np.random.default_rng(200 + seed)
    n = 1 + seed % 4
    H = _spd(rng, n)
    c = 3.0 * rng.normal(size=n)
    lo, hi = -rng.uniform(0.1, 0.8, n), rng.uniform(0.1, 0.8, n)
    A = np.vstack([-np.eye(n), np.eye(n)])
    b = np.concatenate([-lo, hi])
    assert np.allclose(O.poly_qp(H, c, A, b), O.box_qp(H, c, lo, hi), atol=1e-12)


def test_poly_qp_single_half_space_closed_form():
    """One row a^T z <= g: the optimum is the H-metric projection of the
    unconstrained minimiser z_u onto the half-space,
    z = z_u - H^{-1} a (a^T z_u - g) / (a^T H^{-1} a) when a^T z_u > g."""
    rng = np.random.default_rng(7)
    for n in (1, 2, 3, 4):
        H = _spd(rng, n)
        a = rng.normal(size=n)
        z_u = rng.normal(size=n)
        g = a @ z_u - 0.5                         # violated by 0.5
        Hia = np.linalg.solve(H, a)
        z_ref = z_u - Hia * (a @ z_u - g) / (a @ Hia)
        z = O.poly_qp(H, H @ z_u, a[None, :], np.array([g]))
        assert np.allclose(z, z_ref, atol=1e-12)
        # inactive: the unconstrained minimiser itself
        z2 = O.poly_qp(H, H @ z_u, a[None, :], np.array([a @ z_u + 0.5]))
        assert np.allclose(z2, z_u, atol=1e-12)


def test_poly_qp_degenerate_vertex():
    """Three rows through the origin of the plane (z1 <= 0, z2 <= 0,
    z1 + z2 <= 0) and a pull towards (5, 5): the optimum is the vertex 0,
    where the three active rows are linearly dependent."""
    A = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    z = O.poly_qp(np.eye(2), np.array([5.0, 5.0]), A, np.zeros(3))
    assert np.allclose(z, 0.0, atol=1e-12)
    # a pull along (1, -1) slides along z1 + z2 = 0 only if z2 <= 0 allows it
    z = O.poly_qp(np.eye(2), np.array([2.0, -1.0]), A, np.zeros(3))
    assert np.allclose(z, [0.0, -1.0], atol=1e-12)


def _slot_rows(p, i, kind, t):
    if kind == "x":
        return [O.global_row(p, i, t * p.nx + a) for a in range(p.nx)]
    return [O.global_row(p, i, p.nx * p.T + t * p.nu + b) for b in range(p.nu)]


def test_slot_constraints_rows():
    p = I.with_coupled_constraints(I.make_instance(4, 4, 1, seed=2, boxes=True, x0_dist="uniform"),
                                   seed=5, n_cx=2, n_cu=1)
    A, b = O.slot_constraints(p, 1, "x", 0)
    assert A.shape == (0, p.nx)                   # slot 0 is pinned, not constrained
    A, b = O.slot_constraints(p, 1, "x", 2)
    assert A.shape == (2 * p.nx + 2, p.nx)
    assert np.allclose(A[:p.nx], -np.eye(p.nx)) and np.allclose(b[:p.nx], -p.x_lo[1])
    assert np.allclose(A[p.nx:2 * p.nx], np.eye(p.nx)) and np.allclose(b[p.nx:2 * p.nx], p.x_hi[1])
    assert np.allclose(A[2 * p.nx:], p.Gx[1]) and np.allclose(b[2 * p.nx:], p.gx[1])
    A, b = O.slot_constraints(p, 3, "u", 0)
    assert A.shape == (2 * p.nu + 1, p.nu)
    assert np.allclose(A[-1], p.Gu[3]) and np.isclose(b[-1], p.gu[3, 0])


@pytest.mark.parametrize("seed", range(3))
def test_coupled_phi_step_matches_slsqp_on_the_slot_problem(seed):
    """One state slot and one input slot of one subsystem with coupled rows,
    solved directly in the Phi entries of the slot's rows by SLSQP:
    min (Phi_s xh)^T C (Phi_s xh) + rho/2 ||Phi_s - V_s||^2 s.t. the box and the
    coupled rows on Phi_s xh."""
    p = I.with_coupled_constraints(
        I.make_instance(5, 4, 1, seed=seed, boxes=True, x0_dist="uniform", x_bound=0.8, u_bound=0.5),
        seed=seed + 30, n_cx=2, n_cu=1, g_range=(0.05, 0.3))
    rng = np.random.default_rng(seed)
    lay = O.Layout(p)
    Psi, Lam = rng.normal(size=lay.nnz) * 0.7, rng.normal(size=lay.nnz) * 0.3
    Phi, z_all = O.phi_step_block(lay, Psi, Lam, p.x0, p.rho)
    V = Psi - Lam
    xf = p.x0.reshape(-1)
    i = 2
    binds = 0
    for kind, t, C in [("x", 1, p.Q_blk[i]), ("u", 0, p.R_blk[i])]:
        rows = _slot_rows(p, i, kind, t)
        Ac, bc = O.slot_constraints(p, i, kind, t)
        sel = [np.nonzero(lay.rows == r)[0] for r in rows]
        xh = [xf[lay.cols[e]] for e in sel]
        v = [V[e] for e in sel]
        sizes = [len(e) for e in sel]

        def unpack(theta):
            out, o = [], 0
            for k in sizes:
                out.append(theta[o:o + k]); o += k
            return out

        def zof(theta):
            ph = unpack(theta)
            return np.array([ph[a] @ xh[a] for a in range(len(rows))])

        def f(theta):
            ph, z = unpack(theta), zof(theta)
            return z @ C @ z + 0.5 * p.rho * sum(np.sum((ph[a] - v[a]) ** 2) for a in range(len(rows)))

        res = scipy.optimize.minimize(f, np.concatenate(v), method="SLSQP",
                                      constraints=[{"type": "ineq", "fun": lambda th: bc - Ac @ zof(th)}],
                                      options={"ftol": 1e-15, "maxiter": 3000})
        assert res.success
        got = np.concatenate([Phi[e] for e in sel])
        assert np.allclose(got, res.x, atol=1e-6), (seed, kind)
        assert f(got) <= res.fun + 1e-9
        binds += int(np.max(Ac @ z_all[rows] - bc) > -1e-9)
    assert binds >= 1, "some slot row must bind"


def test_coupled_admm_matches_centralised_qp():
    """Full blocks, boxes and coupled state rows: the converged trajectory
    solves the centralised QP min y^T W y over the locality-constrained affine
    set with every slot's rows A_s y_s <= b_s; checked by the KKT conditions of
    that QP at the ADMM solution (feasibility, stationarity with multipliers
    on the active rows only, their signs), with a coupled row active."""
    base = I.make_instance(4, 4, 1, seed=3, boxes=True, x0_dist="uniform", x_bound=1.0, u_bound=0.5)
    base.x0 = 0.3 * base.x0
    p = I.with_coupled_constraints(base, seed=8, n_cx=2, n_cu=0, g_range=(0.1, 0.3))
    lay, y0, G = _centralised_affine(p, p.x0)
    U, S, _ = np.linalg.svd(G, full_matrices=False)
    Bm = U[:, S > 1e-10 * S[0]]
    W = np.zeros((lay.n_rows, lay.n_rows))
    rows_all, rhs_all, coupled = [], [], []
    for i in range(p.n_sub):
        for kind, slots, C in [("x", range(p.T), p.Q_blk[i]), ("u", range(p.T - 1), p.R_blk[i])]:
            for t in slots:
                rr = _slot_rows(p, i, kind, t)
                W[np.ix_(rr, rr)] = C
                Ac, bc = O.slot_constraints(p, i, kind, t)
                nbox = Ac.shape[0] - (p.Gx.shape[1] if (kind == "x" and t >= 1) else 0)
                for k in range(Ac.shape[0]):
                    row = np.zeros(lay.n_rows); row[rr] = Ac[k]
                    rows_all.append(row); rhs_all.append(bc[k]); coupled.append(k >= nbox)
    Arow, brow, coupled = np.array(rows_all), np.array(rhs_all), np.array(coupled)
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=5000, eps_p=1e-10, eps_d=1e-10)
    assert res.status == O.STATUS_CONVERGED
    y = o.lay.trajectory(res.Phi, p.x0)
    assert np.allclose(y0 + Bm @ (Bm.T @ (y - y0)), y, atol=1e-8)
    slack = Arow @ y - brow
    assert np.all(slack <= 1e-8)
    act = slack >= -1e-7
    assert np.any(act & coupled), "a coupled row must be active"
    grad = 2 * Bm.T @ (W @ y)
    Cm = (Arow[act] @ Bm).T
    mu = np.linalg.lstsq(Cm, -grad, rcond=None)[0]
    assert np.allclose(Cm @ mu, -grad, atol=1e-6)
    assert np.all(mu >= -1e-6)


def test_planted_coupled_sign_flip_is_caught(monkeypatch):
    """A slot QP that reads the coupled rows with the wrong sign fails the
    centralised check above."""
    real = O.slot_constraints

    def flipped(prob, i, kind, t):
        A, b = real(prob, i, kind, t)
        n = prob.nx if kind == "x" else prob.nu
        if kind == "x" and t >= 1 and prob.Gx is not None:
            k = prob.Gx.shape[1]
            A = A.copy(); A[-k:] *= -1.0
        return A, b

    monkeypatch.setattr(O, "slot_constraints", flipped)
    with pytest.raises(AssertionError):
        test_coupled_admm_matches_centralised_qp()


# --------------------------------------------------------------------------
# Stale messages (the distributed setting simulated): admm(stale=(p, seed))
# --------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    """The first outputs of SplitMix64 seeded with 0, as its reference
    implementation prints them."""
    assert int(O.splitmix64_at(0, 0)) == 0xE220A8397B1DCDAF
    assert int(O.splitmix64_at(0, 1)) == 0x6E789E6AA1B965F4
    # vectorised draws equal the scalar ones
    v = O.splitmix64_at(12345, np.arange(5))
    assert [int(a) for a in v] == [int(O.splitmix64_at(12345, n)) for n in range(5)]


def test_loss_draws_are_uniform_and_independent():
    rng_n = 64
    k = np.repeat(np.arange(200), rng_n * rng_n)
    j = np.tile(np.repeat(np.arange(rng_n), rng_n), 200)
    m = np.tile(np.arange(rng_n), 200 * rng_n)
    for p in (0.1, 0.5):
        lost = O.message_lost(7, O.stale_threshold(p), 0, j[:rng_n * rng_n], m[:rng_n * rng_n], rng_n)
        n = lost.size
        assert abs(lost.mean() - p) < 4 * np.sqrt(p * (1 - p) / n)
    lost = np.concatenate([O.message_lost(7, O.stale_threshold(0.5), kk, j[:rng_n * rng_n], m[:rng_n * rng_n], rng_n)
                           for kk in range(20)]).reshape(20, -1).astype(float)
    c = np.corrcoef(lost[:-1].ravel(), lost[1:].ravel())[0, 1]          # iteration to iteration
    assert abs(c) < 0.02
    assert not O.message_lost(7, O.stale_threshold(0.0), 3, 1, 2, 8)
    assert O.message_lost(7, O.stale_threshold(1.0), 3, 1, 2, 8)


def test_stale_with_p0_is_plain_admm():
    p = I.make_instance(12, 5, 2, seed=4, boxes=True, x0_dist="uniform")
    o = O.Oracle(p)
    a = O.admm(o.lay, o.blocks, p.x0, fixed_iters=30)
    b = O.admm(o.lay, o.blocks, p.x0, fixed_iters=30, stale=(0.0, 9))
    assert np.allclose(a.Psi, b.Psi, atol=1e-12) and np.allclose(a.Phi, b.Phi, atol=1e-12)
    c = O.admm(o.lay, o.blocks, p.x0, fixed_iters=30, stale=(0.3, 9))
    assert np.max(np.abs(c.Psi - a.Psi)) > 1e-6                           # losses change the iterates


def _stale_admm_by_messages(p, K, prob_loss, seed):
    """Per-message restatement on a tiny instance: every (sender j, receiver
    m, local row r) value kept in a dict and updated by loops."""
    o = O.Oracle(p)
    lay = o.lay
    xf = p.x0.reshape(-1)
    thr = O.stale_threshold(prob_loss)

    def sums(V):
        out = {}
        for e in range(lay.nnz):
            key = (int(lay.col_sub[e]), int(lay.row_sub[e]), int(lay.row_local[e]))
            out[key] = out.get(key, 0.0) + V[e] * xf[lay.cols[e]]
        return out

    Psi = np.zeros(lay.nnz)
    Lam = np.zeros(lay.nnz)
    held = sums(Psi - Lam)
    for k in range(K):
        w = np.zeros(lay.n_rows)
        for (j, m, r), v in held.items():
            w[O.global_row(p, m, r)] += v
        Phi, _ = O.phi_step(lay, Psi, Lam, p.x0, p.rho, w=w)
        Psi_new = O.psi_step(lay, o.blocks, Phi + Lam)
        Lam = Lam + Phi - Psi_new
        Psi = Psi_new
        fresh = sums(Psi - Lam)
        for (j, m, r) in held:
            n = (k * p.n_sub + j) * p.n_sub + m                  # the message's draw number
            if not (int(O.splitmix64_at(seed, n)) >> 11) < thr:
                held[(j, m, r)] = fresh[(j, m, r)]
    return Psi, Lam


def test_stale_admm_matches_per_message_loops():
    p = I.make_instance(5, 3, 1, seed=2, boxes=True, x0_dist="uniform")
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=12, stale=(0.4, 77))
    Psi, Lam = _stale_admm_by_messages(p, 12, 0.4, 77)
    assert np.allclose(ref.Psi, Psi, atol=1e-12) and np.allclose(ref.Lam, Lam, atol=1e-12)


def test_stale_admm_keeps_the_affine_constraint():
    p = I.make_instance(8, 4, 2, seed=5, boxes=True, x0_dist="uniform")
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, fixed_iters=25, stale=(0.5, 3))
    Z = O.global_Z_AB(p)
    Psi = o.lay.to_dense(res.Psi)
    rhs = np.zeros((Z.shape[0], p.n_sub * p.nx)); rhs[:p.n_sub * p.nx] = np.eye(p.n_sub * p.nx)
    assert np.max(np.abs(Z @ Psi - rhs)) < 1e-10


def test_planted_wrong_receiver_is_caught(monkeypatch):
    """Loss draws keyed on the wrong receiver fail the per-message check."""
    real = O.message_lost
    monkeypatch.setattr(O, "message_lost", lambda seed, thr, k, j, m, n: real(seed, thr, k, m, j, n))
    with pytest.raises(AssertionError):
        test_stale_admm_matches_per_message_loops()


# --------------------------------------------------------------------------
# Other state and input sizes (1..4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nx,nu", [(1, 1), (3, 2), (4, 4), (4, 1)])
def test_general_shapes_admm_matches_riccati(nx, nu):
    """d >= N-1, no boxes: u(0) of the ADMM is the finite-horizon LQR gain for
    plants of other state and input sizes."""
    n, T = 4, 4
    p = I.make_general(n, T, n - 1, nx, nu, seed=13, boxes=False)
    rng = np.random.default_rng(6)
    p.q = rng.uniform(0.5, 2.0, p.q.shape)
    p.r = rng.uniform(0.5, 2.0, p.r.shape)
    A, B = p.dense_A(), p.dense_B()
    u_ref = _riccati_u0(A, B, np.diag(p.q.reshape(-1)), np.diag(p.r.reshape(-1)), T, p.x0.reshape(-1))
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=50000, eps_p=1e-11, eps_d=1e-11)
    assert res.status == O.STATUS_CONVERGED
    assert np.allclose(o.control(res).reshape(-1), u_ref, atol=1e-8)


@pytest.mark.parametrize("nx,nu,graph,seed", [(3, 2, "chain", 8), (1, 1, "grid", 9), (4, 2, "grid", 8)])
def test_general_shapes_invariants(nx, nu, graph, seed):
    p = I.make_general(9, 4, 1, nx, nu, graph=graph, seed=seed)
    o = O.Oracle(p)
    res = O.admm(o.lay, o.blocks, p.x0, max_iter=20000, eps_p=1e-9, eps_d=1e-9)
    assert res.status == O.STATUS_CONVERGED
    Z = O.global_Z_AB(p)
    Psi = o.lay.to_dense(res.Psi)
    rhs = np.zeros((Z.shape[0], p.n_sub * p.nx)); rhs[:p.n_sub * p.nx] = np.eye(p.n_sub * p.nx)
    assert np.max(np.abs(Z @ Psi - rhs)) < 1e-10
    assert np.max(np.abs(res.Phi - res.Psi)) < 1e-8
    y = o.lay.trajectory(res.Phi, p.x0)
    assert np.all(y <= o.lay.hi + 1e-8) and np.all(y >= o.lay.lo - 1e-8)


# --------------------------------------------------------------------------
# Conv (Alg. 2): residuals and the stopping rule, with rho != 1
# --------------------------------------------------------------------------

def _decoupled_pair(rho):
    """Two subsystems with no coupling edge, T = 2, d = 0, different plants,
    no boxes: every column problem is the one-subsystem one."""
    p = I.make_instance(2, 2, 0, seed=31, boxes=False, x0_dist="normal", rho=rho)
    p.adj_ptr = np.zeros(3, np.int32)
    p.adj_idx = np.zeros(0, np.int32)
    p.A_off = np.zeros((0, 2, 2))
    p.A_diag[1] = [[1.5, 0.8], [-0.6, 2.0]]          # a second, quite different plant
    p.B[1] = [[0.5], [0.2]]
    return p


def _first_iteration_residual_by_hand(p):
    """From a cold start the first Phi-step sees v = 0, so Phi^1 = 0 (z* = 0 is
    inside every box), Psi^1 = q (the projection of 0 is the min-norm point of
    Z_j psi = e_c) and r_j = ||Psi^1||_F, s_j = rho ||Psi^1 - 0||_F.  With T = 2
    the column problem of own state c is: x_0 = e_c, x_1 = A e_c + B u_0,
    min ||x_0||^2 + ||x_1||^2 + u_0^2, whose minimiser in u_0 is
    u_0 = -B^T A e_c / (1 + B^T B) (one-dimensional least squares)."""
    out = []
    for j in range(p.n_sub):
        A, B = p.A_diag[j], p.B[j][:, 0]
        sq = 0.0
        for c in range(p.nx):
            e = np.zeros(p.nx); e[c] = 1.0
            u = -(B @ A @ e) / (1.0 + B @ B)
            x1 = A @ e + B * u
            sq += 1.0 + x1 @ x1 + u * u
        out.append(np.sqrt(sq))
    return np.array(out)


def test_conv_first_iteration_closed_form():
    rho = 0.7
    p = _decoupled_pair(rho)
    o = O.Oracle(p)
    r_hand = _first_iteration_residual_by_hand(p)
    assert abs(r_hand[0] - r_hand[1]) > 0.05                 # the max picks one subsystem
    res = O.admm(o.lay, o.blocks, p.x0, fixed_iters=1)
    assert np.max(np.abs(res.Phi)) == 0.0
    assert np.isclose(res.r_max, r_hand.max(), rtol=1e-12)
    assert np.isclose(res.s_max, rho * r_hand.max(), rtol=1e-12)
    r_j, s_j = O.conv_residuals(o.lay, res.Phi, res.Psi, np.zeros(o.lay.nnz), rho)
    assert r_j.shape == s_j.shape == (p.n_sub,)
    assert np.allclose(r_j, r_hand, rtol=1e-12)
    assert np.allclose(s_j, rho * r_hand, rtol=1e-12)
    assert np.isclose(res.r_max, r_hand.max(), rtol=1e-12)
    assert np.isclose(res.s_max, rho * r_hand.max(), rtol=1e-12)
    # the stopping rule: eps between the two residuals stops after one iteration
    # exactly when both tests pass
    lo, hi = rho * r_hand.max(), r_hand.max()
    assert O.admm(o.lay, o.blocks, p.x0, eps_p=hi * 1.001, eps_d=lo * 1.001, max_iter=1).status == O.STATUS_CONVERGED
    assert O.admm(o.lay, o.blocks, p.x0, eps_p=hi * 1.001, eps_d=lo * 0.999, max_iter=1).status == O.STATUS_MAX_ITER
    assert O.admm(o.lay, o.blocks, p.x0, eps_p=hi * 0.999, eps_d=lo * 1.001, max_iter=1).status == O.STATUS_MAX_ITER


def _residuals_by_loops(p, Phi, Psi_new, Psi_old, rho):
    """r_j and s_j with explicit loops over the dense matrices: every entry of
    the nx columns of subsystem j (the whole column, not only the patch)."""
    lay = O.Layout(p)
    F, Pn, Po = lay.to_dense(Phi), lay.to_dense(Psi_new), lay.to_dense(Psi_old)
    r, s = np.zeros(p.n_sub), np.zeros(p.n_sub)
    for j in range(p.n_sub):
        for c in range(j * p.nx, (j + 1) * p.nx):
            for row in range(F.shape[0]):
                r[j] += (F[row, c] - Pn[row, c]) ** 2
                s[j] += (Pn[row, c] - Po[row, c]) ** 2
    return np.sqrt(r), rho * np.sqrt(s)


def test_conv_stops_at_the_first_iteration_meeting_both_tests():
    """Coupled chain with boxes and rho = 0.7, stepped one iteration at a time
    (the iteration is a map of (Psi, Lambda)); the residuals restated with
    loops decide the first iteration at which every subsystem meets both
    tests, and the stopped run must end exactly there with those residuals."""
    rho, eps = 0.7, 2e-3
    p = I.make_instance(4, 3, 1, seed=12, boxes=True, x0_dist="uniform", rho=rho, eps=eps, u_bound=0.3)
    o = O.Oracle(p)
    Psi, Lam = np.zeros(o.lay.nnz), np.zeros(o.lay.nnz)
    stop = None
    for k in range(1, 400):
        res = O.admm(o.lay, o.blocks, p.x0, Psi0=Psi, Lam0=Lam, fixed_iters=1)
        r, s = _residuals_by_loops(p, res.Phi, res.Psi, Psi, rho)
        rj, sj = O.conv_residuals(o.lay, res.Phi, res.Psi, Psi, rho)
        assert np.allclose(rj, r, rtol=1e-10, atol=1e-15) and np.allclose(sj, s, rtol=1e-10, atol=1e-15)
        Psi, Lam = res.Psi, res.Lam
        if np.max(r) <= eps and np.max(s) <= eps:
            stop = (k, np.max(r), np.max(s))
            break
    assert stop is not None and stop[0] > 5
    run = O.admm(o.lay, o.blocks, p.x0)
    assert run.status == O.STATUS_CONVERGED and run.iters == stop[0]
    assert np.isclose(run.r_max, stop[1], rtol=1e-9) and np.isclose(run.s_max, stop[2], rtol=1e-9)


def _plant_conv(monkeypatch, kind):
    def bad(lay, Phi, Psi_new, Psi_old, rho):
        if kind == "rho_dropped":
            return O.per_subsystem_norm(lay, Phi - Psi_new), O.per_subsystem_norm(lay, Psi_new - Psi_old)
        if kind == "global_norm":
            n = lay.prob.n_sub
            return (np.full(n, np.linalg.norm(Phi - Psi_new)),
                    rho * np.full(n, np.linalg.norm(Psi_new - Psi_old)))
        if kind == "per_column":
            def col_norm(v):
                return np.sqrt(np.bincount(lay.cols, weights=v * v, minlength=lay.prob.n_sub * lay.prob.nx))
            return col_norm(Phi - Psi_new), rho * col_norm(Psi_new - Psi_old)
        raise ValueError(kind)
    monkeypatch.setattr(O, "conv_residuals", bad)


@pytest.mark.parametrize("kind", ["rho_dropped", "global_norm", "per_column"])
def test_planted_conv_mistake_is_caught(monkeypatch, kind):
    _plant_conv(monkeypatch, kind)
    with pytest.raises(AssertionError):
        test_conv_first_iteration_closed_form()


def test_converged_warm_policy_reduces_to_its_two_limits():
    """The "converged" warm start is the previous-step start when every step
    meets Conv and the cold start when every step stops at max_iter."""
    p = I.make_instance(6, 4, 1, seed=4, boxes=False, x0_dist="normal", mpc_steps=4)
    o = O.Oracle(p)
    a = o.run_mpc(4, warm="converged")
    b = o.run_mpc(4, warm="previous")
    assert all(s.status == O.STATUS_CONVERGED for s in a[3])
    assert a[2] == b[2] and np.array_equal(a[1], b[1])
    c = o.run_mpc(4, warm="converged", max_iter=3)
    d = o.run_mpc(4, warm="cold", max_iter=3)
    e = o.run_mpc(4, warm="previous", max_iter=3)
    assert all(s.status == O.STATUS_MAX_ITER for s in c[3])
    assert np.array_equal(c[1], d[1]) and not np.array_equal(c[1], e[1])
