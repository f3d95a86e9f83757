"""FP64 oracle for the DLMPC ADMM (Sec. II-A, Alg. 1 and Alg. 2).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain CPU statement of what
the CUDA path computes.  Only the test-suite, the smoke check and the CPU
baseline / reference arm of the benchmark may import it; the product path never
does.  It shares no code with the CUDA path: it re-derives the locality pattern
with its own BFS, assembles its own constraint matrices and projects with a
pseudo-inverse taken from an SVD (the CUDA path uses a pivoted Householder QR
null-space basis instead).

Pinned parts (see tests/test_oracle_pins.py):
  * phi_step      - brute-force / KKT checks of the row box-QP and its special cases;
  * box_qp, phi_step_block (full Q_i, R_i blocks) - against scipy's bounded
                    minimiser, the diagonal closed form, the Riccati gain with
                    full blocks and the centralised boxed QP with full blocks;
  * poly_qp, slot_constraints (coupled per-slot rows) - against scipy's SLSQP,
                    box_qp when the rows are a box, the closed-form projection
                    onto one half-space, a degenerate vertex, and the
                    centralised QP with coupled rows (KKT at the ADMM solution);
  * psi projector - Z psi = e exactly, idempotent symmetric projector, min-norm offset
                    against lstsq, residual orthogonal to the null space;
  * admm(stale=) - p = 0 is the exchange-free admm; a per-message loop on
                    small cases gives the same iterates; the loss draws are
                    uniform and independent, at rate p; Z_AB Psi = I holds;
  * conv_residuals / conv_met - closed-form residuals of the first
                    iteration from a cold start (rho != 1, decoupled subsystems
                    of different norms), a restatement with explicit loops
                    over dense matrices, the stop at the first iteration that
                    meets both tests; planted mistakes (rho dropped, one
                    global norm, per-column norms) fail these pins;
  * admm / mpc    - converged trajectory against the centralised
                    locality-constrained QP (least squares / SLSQP) and, for
                    d >= N-1 with no boxes, against the textbook finite-horizon
                    Riccati recursion; the invariants Z_AB Psi = I, Phi = Psi at
                    convergence, support inside L_d; the Lemma bounds on
                    D_row and D_col (Sec. III-B).

Conventions (readings of the paper, each stated once):
  * Phi has T state slots t=0..T-1 and T-1 input slots t=0..T-2 (Sec. II-A:
    Phi in R^{(N_x T + N_u (T-1)) x N_x}); Q weights every state slot,
    including t=0; the last state slot carries the same Q.
  * Locality: Phi(r, c) may be nonzero iff dist(sub(r), sub(c)) <= d.
  * Global row order of Phi follows the paper: all states of slot 0, ..., all
    states of slot T-1, then all inputs of slot 0, ..., slot T-2.
  * ADMM in scaled form: Phi-step row-wise, Psi-step column-wise projection onto
    {Z_AB Psi = I} restricted to the column's d-hop patch, Lambda <- Lambda +
    Phi - Psi (Alg. 2).  Stop when, for every subsystem j, ||Phi - Psi||_F over
    j's columns <= eps_p and rho ||Psi^{k+1} - Psi^k||_F over j's columns <= eps_d.
  * Box bounds apply to states of slots 1..T-1 and to all inputs; the slot-0
    state is pinned by Z_AB Psi = I.
  * The Psi-step keeps every row of Z_AB with a nonzero coefficient on a patch
    variable (rows of subsystems up to d+1 hops away); all-zero rows are dropped.
"""
from __future__ import annotations

import collections
import dataclasses
import itertools
from typing import Dict, List, Optional

import numpy as np

STATUS_CONVERGED = 0
STATUS_MAX_ITER = 1


# ----------------------------------------------------------------------------
# Locality structure (Sec. II-A, d-locality on G_(A,B))
# ----------------------------------------------------------------------------

def hop_distances(prob, src: int, max_hops: int) -> Dict[int, int]:
    """Breadth-first search from `src`, returning {node: hops} for hops <= max_hops."""
    dist = {src: 0}
    queue = collections.deque([src])
    while queue:
        v = queue.popleft()
        if dist[v] == max_hops:
            continue
        for w in prob.adj_idx[prob.adj_ptr[v]:prob.adj_ptr[v + 1]]:
            w = int(w)
            if w not in dist:
                dist[w] = dist[v] + 1
                queue.append(w)
    return dist


def patch_members(prob, j: int) -> List[int]:
    """Subsystems within d hops of j, ascending."""
    return sorted(hop_distances(prob, j, prob.d).keys())


def ring_members(prob, j: int) -> List[int]:
    """Subsystems within d+1 hops of j, ascending."""
    return sorted(hop_distances(prob, j, prob.d + 1).keys())


def global_row(prob, i: int, r: int) -> int:
    """Global Phi row of local row r of subsystem i (paper's time-major order)."""
    Nx, Nu = prob.n_sub * prob.nx, prob.n_sub * prob.nu
    if r < prob.nx * prob.T:
        t, a = divmod(r, prob.nx)
        return t * Nx + i * prob.nx + a
    t, b = divmod(r - prob.nx * prob.T, prob.nu)
    return prob.T * Nx + t * Nu + i * prob.nu + b


def n_rows(prob) -> int:
    return prob.n_sub * prob.nx * prob.T + prob.n_sub * prob.nu * (prob.T - 1)


def lemma_bounds(s: int, l: int, d: int, T: int):
    """Lemma of Sec. III-B: D_row <= s (l^{d+1}-1)/(l-1), D_col <= (2T-1) times that."""
    nodes = d + 1 if l == 1 else (l ** (d + 1) - 1) // (l - 1)
    return s * nodes, (2 * T - 1) * s * nodes


# ----------------------------------------------------------------------------
# Z_AB and the column constraint blocks (Sec. II-A, SLS achievability Z_AB Phi = I)
# ----------------------------------------------------------------------------

def z_row_coeffs(prob, i: int, t: int, a: int):
    """Nonzero coefficients of the Z_AB row for state (t, i, a) as a list of
    ((subsystem, local row), value).  Slot 0 reads x_0 = I; slot t >= 1 reads
    x_t - A x_{t-1} - B u_{t-1} = 0."""
    nx, nu = prob.nx, prob.nu
    out = [((i, t * nx + a), 1.0)]
    if t == 0:
        return out
    for b in range(nx):
        out.append(((i, (t - 1) * nx + b), -prob.A_diag[i][a, b]))
    for e in range(prob.adj_ptr[i], prob.adj_ptr[i + 1]):
        k = int(prob.adj_idx[e])
        for b in range(nx):
            out.append(((k, (t - 1) * nx + b), -prob.A_off[e][a, b]))
    for b in range(nu):
        out.append(((i, nx * prob.T + (t - 1) * nu + b), -prob.B[i][a, b]))
    return out


def global_Z_AB(prob) -> np.ndarray:
    """Dense Z_AB (N_x T rows x Phi rows); for small instances only."""
    nrow = prob.n_sub * prob.nx * prob.T
    Z = np.zeros((nrow, n_rows(prob)))
    for t in range(prob.T):
        for i in range(prob.n_sub):
            for a in range(prob.nx):
                zr = t * prob.n_sub * prob.nx + i * prob.nx + a
                for (k, r), val in z_row_coeffs(prob, i, t, a):
                    Z[zr, global_row(prob, k, r)] += val
    return Z


@dataclasses.dataclass
class ColumnBlock:
    """Restricted achievability constraint of column-subsystem j."""
    members: List[int]        # Patch(j), ascending
    Z: np.ndarray             # rows kept x D_col
    rhs: np.ndarray           # [nx, rows kept]: e_c restricted to kept rows, for each own column
    rank: int
    P: np.ndarray             # D_col x D_col projector onto null(Z) = I - Z^+ Z
    q: np.ndarray             # [nx, D_col] min-norm solutions Z^+ e_c
    feas: float               # max_c ||Z q_c - e_c||


def column_block(prob, j: int, rtol: float = 1e-12) -> ColumnBlock:
    """Assemble Z_j and its projector by pseudo-inverse from an SVD (Sec. II-A Psi-comp)."""
    members = patch_members(prob, j)
    ring = ring_members(prob, j)
    rs = prob.r_sub
    var_index = {}
    for m_pos, m in enumerate(members):
        for r in range(rs):
            var_index[(m, r)] = m_pos * rs + r
    D = len(members) * rs
    rows, rhs_rows = [], []
    for t in range(prob.T):
        for i in ring:
            for a in range(prob.nx):
                row = np.zeros(D)
                for key, val in z_row_coeffs(prob, i, t, a):
                    if key in var_index:
                        row[var_index[key]] += val
                if np.any(row != 0.0):
                    rows.append(row)
                    rhs_rows.append((t, i, a))
    Z = np.array(rows)
    rhs = np.zeros((prob.nx, len(rows)))
    for c in range(prob.nx):
        for k, (t, i, a) in enumerate(rhs_rows):
            if t == 0 and i == j and a == c:
                rhs[c, k] = 1.0
    try:
        U, S, Vt = np.linalg.svd(Z, full_matrices=False)
    except np.linalg.LinAlgError:
        # LAPACK's divide-and-conquer driver (gesdd) gives up on a few
        # matrices; the QR-iteration driver computes the same decomposition
        import scipy.linalg
        U, S, Vt = scipy.linalg.svd(Z, full_matrices=False, lapack_driver="gesvd")
    rank = int(np.sum(S > rtol * S[0]))
    Zp = (Vt[:rank].T / S[:rank]) @ U[:, :rank].T          # Z^+
    P = np.eye(D) - Zp @ Z
    q = (Zp @ rhs.T).T
    feas = float(np.max(np.abs(q @ Z.T - rhs)))
    return ColumnBlock(members, Z, rhs, rank, P, q, feas)


# ----------------------------------------------------------------------------
# Sparse (support-only) storage of Phi / Psi / Lambda
# ----------------------------------------------------------------------------

class Layout:
    """Support entries of L_d stored column-patch-major: for column-subsystem j,
    own column a, patch member m (ascending), local row r.  Column c = j*nx + a
    owns the contiguous entries [col_off[c], col_off[c] + D_col(j))."""

    def __init__(self, prob):
        self.prob = prob
        nx = prob.nx
        rs = prob.r_sub
        self.members = [patch_members(prob, j) for j in range(prob.n_sub)]
        rows, cols, sub_of_row, lrow = [], [], [], []
        self.col_off = np.zeros(prob.n_sub * nx + 1, np.int64)
        pos = 0
        for j in range(prob.n_sub):
            for a in range(nx):
                c = j * nx + a
                self.col_off[c] = pos
                for m in self.members[j]:
                    for r in range(rs):
                        rows.append(global_row(prob, m, r))
                        cols.append(c)
                        sub_of_row.append(m)
                        lrow.append(r)
                        pos += 1
        self.col_off[-1] = pos
        self.rows = np.asarray(rows, np.int64)
        self.cols = np.asarray(cols, np.int64)
        self.row_sub = np.asarray(sub_of_row, np.int64)
        self.row_local = np.asarray(lrow, np.int64)
        self.nnz = pos
        self.n_rows = n_rows(prob)
        self.col_sub = self.cols // nx
        # per-row cost weight and bounds (indexed by global row)
        self.qw = np.zeros(self.n_rows)
        self.lo = np.full(self.n_rows, -np.inf)
        self.hi = np.full(self.n_rows, np.inf)
        for i in range(prob.n_sub):
            for r in range(rs):
                g = global_row(prob, i, r)
                if r < nx * prob.T:
                    t, a = divmod(r, nx)
                    self.qw[g] = prob.q[i, a]
                    if t >= 1 and prob.x_lo is not None:
                        self.lo[g], self.hi[g] = prob.x_lo[i, a], prob.x_hi[i, a]
                else:
                    t, b = divmod(r - nx * prob.T, prob.nu)
                    self.qw[g] = prob.r[i, b]
                    if prob.u_lo is not None:
                        self.lo[g], self.hi[g] = prob.u_lo[i, b], prob.u_hi[i, b]

    def to_dense(self, vals: np.ndarray) -> np.ndarray:
        """Dense Phi (n_rows x N_x) from support values (small instances only)."""
        M = np.zeros((self.n_rows, self.prob.n_sub * self.prob.nx))
        M[self.rows, self.cols] = vals
        return M

    def trajectory(self, vals: np.ndarray, x0: np.ndarray) -> np.ndarray:
        """y = Phi x0 over all global rows."""
        xf = x0.reshape(-1)
        return np.bincount(self.rows, weights=vals * xf[self.cols], minlength=self.n_rows)


# ----------------------------------------------------------------------------
# The three ADMM steps and Conv (Alg. 2)
# ----------------------------------------------------------------------------

def phi_step_row(v: np.ndarray, xh: np.ndarray, qw: float, rho: float,
                 lo: float, hi: float) -> np.ndarray:
    """argmin_phi qw (phi.xh)^2 + rho/2 ||phi - v||^2  s.t. lo <= phi.xh <= hi.

    phi = v + alpha xh; in z = phi.xh the objective is qw z^2 + rho (z-w)^2/(2s)
    with w = v.xh, s = ||xh||^2, minimised at z* = rho w / (rho + 2 qw s) and then
    clipped to [lo, hi] (one-dimensional convex problem).  s = 0 gives phi = v."""
    s = float(xh @ xh)
    if s == 0.0:
        return v.copy()
    w = float(v @ xh)
    z = min(max(rho * w / (rho + 2.0 * qw * s), lo), hi)
    return v + ((z - w) / s) * xh


def phi_step(lay: Layout, Psi: np.ndarray, Lam: np.ndarray, x0: np.ndarray, rho: float,
             w: Optional[np.ndarray] = None):
    """Row-wise Phi-comp for every row at once: returns (Phi, z) with z = Phi x0 per row.
    `w` replaces the row sums (Psi - Lambda) x_hat when the rows see other
    values than the current ones (stale messages, `admm(stale=...)`)."""
    xf = x0.reshape(-1)
    xe = xf[lay.cols]
    V = Psi - Lam
    if w is None:
        w = np.bincount(lay.rows, weights=V * xe, minlength=lay.n_rows)
    s = np.bincount(lay.rows, weights=xe * xe, minlength=lay.n_rows)
    zstar = rho * w / (rho + 2.0 * lay.qw * s)
    z = np.minimum(np.maximum(zstar, lay.lo), lay.hi)
    alpha = np.zeros(lay.n_rows)
    nz = s > 0.0
    alpha[nz] = (z[nz] - w[nz]) / s[nz]
    z = np.where(nz, z, w)
    Phi = V + alpha[lay.rows] * xe
    return Phi, z


def box_qp(H: np.ndarray, c: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """argmin 1/2 z^T H z - c^T z  s.t. lo <= z <= hi, H symmetric positive
    definite, n <= 4.  Active-set enumeration: every component is free, at lo
    or at hi (only finite bounds); the free part solves H_FF z_F = c_F - H_FA z_A,
    and the pattern is accepted when z is feasible and the gradient
    g = H z - c satisfies the KKT signs (g >= 0 at lo, g <= 0 at hi).  The
    optimum of a strictly convex QP is unique, so exactly one pattern fits
    (up to degenerate ties, which give the same z)."""
    n = len(c)
    choices = [[0] + ([1] if np.isfinite(lo[a]) else []) + ([2] if np.isfinite(hi[a]) else []) for a in range(n)]
    tol = 1e-12 * (1.0 + np.max(np.abs(c)) + np.max(np.abs(H)))
    for pattern in itertools.product(*choices):
        z = np.zeros(n)
        free = [a for a in range(n) if pattern[a] == 0]
        fixed = [a for a in range(n) if pattern[a] != 0]
        for a in fixed:
            z[a] = lo[a] if pattern[a] == 1 else hi[a]
        if free:
            rhs = c[free] - H[np.ix_(free, fixed)] @ z[fixed] if fixed else c[free]
            z[free] = np.linalg.solve(H[np.ix_(free, free)], rhs)
        if np.any(z < lo - tol) or np.any(z > hi + tol):
            continue
        g = H @ z - c
        if all((pattern[a] == 1 and g[a] >= -tol) or (pattern[a] == 2 and g[a] <= tol) for a in fixed):
            return z
    raise RuntimeError("box_qp: no KKT point (H not positive definite?)")


def poly_qp(H: np.ndarray, c: np.ndarray, A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """argmin 1/2 z^T H z - c^T z  s.t.  A z <= b, H symmetric positive
    definite, n <= 4 unknowns and a few rows.  Active-set enumeration of the
    KKT conditions: for every set S of at most n rows whose A_S has full row
    rank, the stationarity and the active rows give
        [H  A_S^T] [z ]   [c  ]
        [A_S  0  ] [mu] = [b_S],
    and S is accepted when z satisfies every row and mu >= 0.  A strictly
    convex QP has one optimum; its active rows contain a linearly independent
    subset carrying non-negative multipliers (Caratheodory on the normal cone),
    so the enumeration meets it."""
    n, m = len(c), len(b)
    tol = 1e-12 * (1.0 + np.max(np.abs(c)) + np.max(np.abs(H)) + (np.max(np.abs(b)) if m else 0.0))
    for k in range(0, min(n, m) + 1):
        for S in itertools.combinations(range(m), k):
            S = list(S)
            As = A[S]
            if k and np.linalg.matrix_rank(As, tol=1e-10) < k:
                continue
            K = np.block([[H, As.T], [As, np.zeros((k, k))]]) if k else H
            sol = np.linalg.solve(K, np.concatenate([c, b[S]]) if k else c)
            z, mu = sol[:n], sol[n:]
            if m and np.any(A @ z > b + tol):
                continue
            if np.any(mu < -tol):
                continue
            return z
    raise RuntimeError("poly_qp: no KKT point (infeasible rows or H not positive definite?)")


def slot_constraints(prob, i: int, kind: str, t: int):
    """Rows (A, b) of A z <= b on the slot vector z of subsystem i: kind "x"
    for the state slot t, "u" for the input slot t.  The boxes (finite bounds
    only) come first as -z_a <= -lo_a and z_a <= hi_a, then the coupled rows
    Gx[i] (states, t >= 1) or Gu[i] (inputs).  The slot-0 state has none: it is
    pinned by Z_AB Psi = I."""
    n = prob.nx if kind == "x" else prob.nu
    if kind == "x":
        if t == 0:
            return np.zeros((0, n)), np.zeros(0)
        lo, hi = (prob.x_lo[i], prob.x_hi[i]) if prob.x_lo is not None else (None, None)
        G, g = (prob.Gx[i], prob.gx[i]) if prob.Gx is not None else (None, None)
    else:
        lo, hi = (prob.u_lo[i], prob.u_hi[i]) if prob.u_lo is not None else (None, None)
        G, g = (prob.Gu[i], prob.gu[i]) if prob.Gu is not None else (None, None)
    rows, rhs = [], []
    if lo is not None:
        for a in range(n):
            if np.isfinite(lo[a]):
                e = np.zeros(n); e[a] = -1.0
                rows.append(e); rhs.append(-lo[a])
        for a in range(n):
            if np.isfinite(hi[a]):
                e = np.zeros(n); e[a] = 1.0
                rows.append(e); rhs.append(hi[a])
    if G is not None:
        for k in range(G.shape[0]):
            rows.append(np.asarray(G[k], float)); rhs.append(float(g[k]))
    return (np.array(rows).reshape(-1, n), np.array(rhs))


def phi_step_block(lay: Layout, Psi: np.ndarray, Lam: np.ndarray, x0: np.ndarray, rho: float,
                   w: Optional[np.ndarray] = None):
    """Phi-comp with full cost blocks Q_i, R_i (Sec. II-A with non-diagonal
    Q_t, R_t): the rows of subsystem i at one time slot (its nx state rows, or
    its nu input rows) share x_hat_i, so with w = (Psi - Lambda) x_hat per row,
    s = ||x_hat_i||^2 and z = Phi x_hat, the slot's rows solve
        min z^T Q_i z + rho/(2 s) ||z - w||^2  s.t.  lo <= z <= hi,
    a box-QP with H = 2 Q_i + (rho/s) I and c = (rho/s) w (box_qp); each row is
    then v + ((z - w)/s) x_hat.  s = 0 gives phi = v.  With coupled
    constraints (Gx / Gu) the slot QP takes them beside the box
    (slot_constraints, poly_qp).  Returns (Phi, z)."""
    prob = lay.prob
    nx, nu, T = prob.nx, prob.nu, prob.T
    xf = x0.reshape(-1)
    xe = xf[lay.cols]
    V = Psi - Lam
    if w is None:
        w = np.bincount(lay.rows, weights=V * xe, minlength=lay.n_rows)
    s = np.bincount(lay.rows, weights=xe * xe, minlength=lay.n_rows)
    Qb = prob.Q_blk if prob.Q_blk is not None else np.array([np.diag(q) for q in prob.q])
    Rb = prob.R_blk if prob.R_blk is not None else np.array([np.diag(r) for r in prob.r])
    coupled = prob.Gx is not None or prob.Gu is not None
    z = w.copy()
    alpha = np.zeros(lay.n_rows)
    for i in range(prob.n_sub):
        groups = [([global_row(prob, i, t * nx + a) for a in range(nx)], Qb[i], "x", t) for t in range(T)]
        groups += [([global_row(prob, i, nx * T + t * nu + b) for b in range(nu)], Rb[i], "u", t)
                   for t in range(T - 1)]
        for rows, C, kind, t in groups:
            rows = np.asarray(rows)
            si = s[rows[0]]
            if si == 0.0:
                continue
            H = 2.0 * C + (rho / si) * np.eye(len(rows))
            if coupled:
                Ac, bc = slot_constraints(prob, i, kind, t)
                zz = poly_qp(H, (rho / si) * w[rows], Ac, bc)
            else:
                zz = box_qp(H, (rho / si) * w[rows], lay.lo[rows], lay.hi[rows])
            z[rows] = zz
            alpha[rows] = (zz - w[rows]) / si
    Phi = V + alpha[lay.rows] * xe
    return Phi, z


def psi_step(lay: Layout, blocks: List[ColumnBlock], V: np.ndarray) -> np.ndarray:
    """Column-wise Psi-comp: psi_c = argmin ||psi - v_c|| s.t. Z_j psi = e_c,
    i.e. psi = P_j v + Z_j^+ e_c, for every column c of every subsystem j."""
    out = np.empty_like(V)
    nx = lay.prob.nx
    for j, blk in enumerate(blocks):
        for a in range(nx):
            c = j * nx + a
            sl = slice(lay.col_off[c], lay.col_off[c + 1])
            out[sl] = blk.P @ V[sl] + blk.q[a]
    return out


def per_subsystem_norm(lay: Layout, vals: np.ndarray) -> np.ndarray:
    """Frobenius norm of vals over the columns owned by each subsystem."""
    sq = np.bincount(lay.col_sub, weights=vals * vals, minlength=lay.prob.n_sub)
    return np.sqrt(sq)


def conv_residuals(lay: Layout, Phi: np.ndarray, Psi_new: np.ndarray, Psi_old: np.ndarray,
                   rho: float):
    """Conv of Alg. 2 (the paper leaves the criterion open; reading: absolute
    residuals per subsystem, no relative scaling).  For every subsystem j,
    over the columns j owns (its nx columns, on their whole patch support):
        r_j = ||Phi - Psi^{k+1}||_F          (primal: consensus Phi = Psi)
        s_j = rho ||Psi^{k+1} - Psi^k||_F    (dual: change of the Psi iterate)
    Returns the two per-subsystem arrays."""
    return per_subsystem_norm(lay, Phi - Psi_new), rho * per_subsystem_norm(lay, Psi_new - Psi_old)


def conv_met(r: np.ndarray, s: np.ndarray, eps_p: float, eps_d: float) -> bool:
    """The d-local checks combined over the network: every subsystem has
    r_j <= eps_p and s_j <= eps_d."""
    return bool(np.max(r) <= eps_p and np.max(s) <= eps_d)


@dataclasses.dataclass
class AdmmResult:
    Phi: np.ndarray
    Psi: np.ndarray
    Lam: np.ndarray
    z: np.ndarray             # Phi x0 per global row from the last Phi-step
    iters: int
    status: int
    r_max: float
    s_max: float


# ----------------------------------------------------------------------------
# Stale messages: the fully distributed setting (Sec. V), simulated
# ----------------------------------------------------------------------------
#
# In the distributed setting every subsystem j tells each member m of its patch
# the sums over j's columns of (Psi - Lambda)[row of m, c] x_c, one per row of
# m (the column-patch exchange of Sec. III-D).  A message (j -> m) sent at the
# end of iteration k is lost with probability p; the receiver then keeps the
# last value it received from j (dropouts, and delays of one or more
# iterations, look the same to it).  The draws come from the counter-based
# SplitMix64 generator (Steele, Lea and Flood, 2014): draw n of seed S is the
# generator's output after n + 1 steps, mix(S + (n + 1) gamma); message
# (k, j, m) uses n = (k N + j) N + m and is lost when the top 53 bits of the
# draw are below floor(p 2^53).

_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_MUL1 = 0xBF58476D1CE4E5B9
_SM_MUL2 = 0x94D049BB133111EB


def splitmix64_at(seed: int, n):
    """Output n (0-based) of SplitMix64 seeded with `seed`; n an int or an
    array of non-negative integers (uint64 arithmetic, wrapping mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(n, dtype=np.uint64) + np.uint64(1)) * np.uint64(_SM_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_MUL2)
        return z ^ (z >> np.uint64(31))


def stale_threshold(p: float) -> int:
    """floor(p 2^53): a message is lost when (draw >> 11) < this."""
    return int(p * 9007199254740992.0)


def message_lost(seed: int, thr: int, k: int, j, m, n_sub: int):
    n = (np.uint64(k) * np.uint64(n_sub) + np.asarray(j, np.uint64)) * np.uint64(n_sub) + np.asarray(m, np.uint64)
    return (splitmix64_at(seed, n) >> np.uint64(11)) < np.uint64(thr)


class Messages:
    """The (row, sending subsystem) pairs of one layout: pair of every stored
    entry, and the row, sender j and receiver m of every pair."""

    def __init__(self, lay: Layout):
        n = lay.prob.n_sub
        key = lay.rows * n + lay.col_sub
        uniq, first, self.pair_of_entry = np.unique(key, return_index=True, return_inverse=True)
        self.row = uniq // n
        self.j = uniq % n
        self.m = lay.row_sub[first]          # row_sub is per stored entry
        self.n_pairs = len(uniq)

    def sums(self, lay: Layout, V: np.ndarray, x0: np.ndarray) -> np.ndarray:
        """The message values: per pair, sum over the sender's columns of V x."""
        xe = x0.reshape(-1)[lay.cols]
        return np.bincount(self.pair_of_entry, weights=V * xe, minlength=self.n_pairs)

    def row_sums(self, lay: Layout, D: np.ndarray) -> np.ndarray:
        """w per row: the sum of the values the row's owner holds."""
        return np.bincount(self.row, weights=D, minlength=lay.n_rows)


def admm(lay: Layout, blocks: List[ColumnBlock], x0: np.ndarray, *,
         Psi0: Optional[np.ndarray] = None, Lam0: Optional[np.ndarray] = None,
         learned: Optional[tuple] = None, max_iter: Optional[int] = None,
         fixed_iters: Optional[int] = None, eps_p: Optional[float] = None,
         eps_d: Optional[float] = None, stale: Optional[tuple] = None) -> AdmmResult:
    """Alg. 2: repeat Phi-comp, Psi-comp, Lambda-comp, Conv.

    Start: cold (Psi = Lambda = 0) unless Psi0/Lam0 are given.  `learned`
    = (Phi_init, Lam_init) replaces the first Phi-step: Psi0 = proj(Phi_init +
    Lam_init), Lam0 = Lam_init + Phi_init - Psi0.  `fixed_iters` runs exactly
    that many iterations with Conv ignored.  `stale` = (p, seed) simulates lost
    messages (see Messages): the Phi-step's row sums are the values last
    received, the start state's being received before the first iteration."""
    prob = lay.prob
    rho = prob.rho
    eps_p = prob.eps_p if eps_p is None else eps_p
    eps_d = prob.eps_d if eps_d is None else eps_d
    max_iter = prob.max_iter if max_iter is None else max_iter
    Psi = np.zeros(lay.nnz) if Psi0 is None else Psi0.astype(np.float64).copy()
    Lam = np.zeros(lay.nnz) if Lam0 is None else Lam0.astype(np.float64).copy()
    if learned is not None:
        Phi_i, Lam_i = learned
        Psi = psi_step(lay, blocks, Phi_i + Lam_i)
        Lam = Lam_i + Phi_i - Psi
    n_it = fixed_iters if fixed_iters is not None else max_iter
    status = STATUS_MAX_ITER
    it = 0
    r_max = s_max = np.inf
    Phi = z = None
    block = (prob.Q_blk is not None or prob.R_blk is not None
             or prob.Gx is not None or prob.Gu is not None)
    msg = held = None
    if stale is not None:
        msg = Messages(lay)
        thr = stale_threshold(stale[0])
        held = msg.sums(lay, Psi - Lam, x0)
    for it in range(1, n_it + 1):
        w = msg.row_sums(lay, held) if msg is not None else None
        Phi, z = (phi_step_block if block else phi_step)(lay, Psi, Lam, x0, rho, w=w)
        Psi_new = psi_step(lay, blocks, Phi + Lam)
        Lam = Lam + Phi - Psi_new
        if msg is not None:
            fresh = msg.sums(lay, Psi_new - Lam, x0)
            lost = message_lost(int(stale[1]), thr, it - 1, msg.j, msg.m, prob.n_sub)
            held = np.where(lost, held, fresh)
        r_j, s_j = conv_residuals(lay, Phi, Psi_new, Psi, rho)
        r_max, s_max = float(np.max(r_j)), float(np.max(s_j))
        Psi = Psi_new
        if fixed_iters is None and conv_met(r_j, s_j, eps_p, eps_d):
            status = STATUS_CONVERGED
            break
    if fixed_iters is not None:
        status = STATUS_CONVERGED if (r_max <= eps_p and s_max <= eps_d) else STATUS_MAX_ITER
    return AdmmResult(Phi, Psi, Lam, z, it, status, r_max, s_max)


# ----------------------------------------------------------------------------
# Alg. 1: the MPC loop
# ----------------------------------------------------------------------------

class Oracle:
    """Holds the one-time precomputation (Alg. 1, first line) of one instance."""

    def __init__(self, prob):
        self.prob = prob
        self.lay = Layout(prob)
        self.blocks = [column_block(prob, j) for j in range(prob.n_sub)]
        self.A = prob.dense_A()
        self.Bm = prob.dense_B()

    def input_rows(self) -> np.ndarray:
        """Global rows of the slot-0 inputs, subsystem-major."""
        p = self.prob
        return np.array([global_row(p, i, p.nx * p.T + b)
                         for i in range(p.n_sub) for b in range(p.nu)], np.int64)

    def control(self, res: AdmmResult) -> np.ndarray:
        """u(tau) = Phi_{u,0} x(tau): the slot-0 input rows of the last Phi iterate."""
        return res.z[self.input_rows()].reshape(self.prob.n_sub, self.prob.nu)

    def dynamics(self, x: np.ndarray, u: np.ndarray) -> np.ndarray:
        """x(tau+1) = A x(tau) + B u(tau)."""
        return (self.A @ x.reshape(-1) + self.Bm @ u.reshape(-1)).reshape(x.shape)

    def run_mpc(self, steps: int, *, x0: Optional[np.ndarray] = None, warm: str = "cold",
                fixed_iters: Optional[int] = None, max_iter: Optional[int] = None,
                x_feed: Optional[np.ndarray] = None):
        """Closed loop of Alg. 1.  warm = "cold" restarts every ADMM from zeros,
        "previous" starts from the previous MPC step's Psi and Lambda,
        "converged" does so only when that step met Conv (zeros after a step
        stopped at max_iter).
        If x_feed [steps, n_sub, nx] is given, the MPC step tau solves from
        x_feed[tau] instead of the closed-loop state (per-step parity)."""
        x = (self.prob.x0 if x0 is None else x0).copy()
        xs, us, its, stats = [x.copy()], [], [], []
        Psi = Lam = None
        for tau in range(steps):
            xt = x if x_feed is None else x_feed[tau]
            if warm == "cold" or (warm == "converged" and stats and stats[-1].status != STATUS_CONVERGED):
                Psi = Lam = None
            res = admm(self.lay, self.blocks, xt, Psi0=Psi, Lam0=Lam,
                       fixed_iters=fixed_iters, max_iter=max_iter)
            u = self.control(res)
            x = self.dynamics(xt, u)
            Psi, Lam = res.Psi, res.Lam
            xs.append(x.copy())
            us.append(u.copy())
            its.append(res.iters)
            stats.append(res)
        return np.array(xs), np.array(us), its, stats


def column_major_state(lay: Layout, vals: np.ndarray) -> List[np.ndarray]:
    """Split support values into per-subsystem [nx, D_col] arrays (the column-owned
    export order: own column, patch member ascending, local row)."""
    out = []
    nx = lay.prob.nx
    for j in range(lay.prob.n_sub):
        a0, a1 = lay.col_off[j * nx], lay.col_off[(j + 1) * nx]
        out.append(vals[a0:a1].reshape(nx, -1))
    return out
