"""Seeded synthetic DLMPC instances.

This module only draws random numbers and lays out the plant of Sec. II-A
(LTI dynamics x(t+1) = A x(t) + B u(t) over an undirected coupling graph
G_(A,B), per-subsystem costs and box bounds).  It holds none of the ADMM
arithmetic: both the CUDA path and the FP64 oracle consume the same
`Problem` objects built here.

Plant (a randomised variant of the chain of Sec. IV-A): every subsystem i has
two states and one input,

    A_ii = [[1, 0.1], [-0.1 k_i, 1 - 0.1 d_i]],   k_i ~ U[0.5, 1.5], d_i ~ U[0.1, 0.5]
    A_ij = a_ij [[0, 0], [1, 1]]  for every neighbour j of i,   a_ij ~ U[-0.1, 0.1]
    B_i  = [0, 0.1]^T

The coupling block mirrors the paper's [A]_ij = [[0, 0], [0.1, 0.1]] (Sec. IV-A):
only the second state of i is driven by the neighbour's states; a_ij is drawn
independently for each ordered pair (i, j).

Draw order for one instance (numpy PCG64, `default_rng(seed)`):
  1. (batch instances only) chain/grid coin, N, T, d;
  2. for i = 0..N-1: k_i then d_i;
  3. for every CSR entry (i, j) in row-major CSR order: a_ij;
  4. x(0): N(0,1) or U[-0.9, 0.9] per state, subsystem-major.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One DLMPC instance (Eq. MPC of Sec. II-A with Q_t = Q, R_t = R for all t)."""

    n_sub: int
    nx: int
    nu: int
    T: int                      # horizon: T state slots (t=0..T-1), T-1 input slots
    d: int                      # locality radius in hops of G_(A,B)
    adj_ptr: np.ndarray         # int32 [n_sub+1] CSR of the undirected graph, no self loops
    adj_idx: np.ndarray         # int32 [nnz], ascending within each row
    A_diag: np.ndarray          # f64 [n_sub, nx, nx]   A_ii
    A_off: np.ndarray           # f64 [nnz, nx, nx]     A_{i, adj_idx[e]} for CSR entry e of row i
    B: np.ndarray               # f64 [n_sub, nx, nu]   B_ii (B is block diagonal)
    q: np.ndarray               # f64 [n_sub, nx]       diagonal of Q_i
    r: np.ndarray               # f64 [n_sub, nu]       diagonal of R_i
    x_lo: Optional[np.ndarray]  # f64 [n_sub, nx] or None (unbounded)
    x_hi: Optional[np.ndarray]
    u_lo: Optional[np.ndarray]  # f64 [n_sub, nu] or None
    u_hi: Optional[np.ndarray]
    rho: float
    eps_p: float
    eps_d: float
    max_iter: int
    x0: np.ndarray              # f64 [n_sub, nx] initial measured state x(0)
    mpc_steps: int              # closed-loop MPC steps T_sim
    name: str = ""
    graph: str = "chain"        # "chain" or "grid"
    grid_shape: Optional[tuple] = None
    Q_blk: Optional[np.ndarray] = None  # f64 [n_sub, nx, nx] full SPD Q_i (replaces q), or None
    R_blk: Optional[np.ndarray] = None  # f64 [n_sub, nu, nu] full SPD R_i (replaces r), or None
    # Coupled constraints of one subsystem at one time slot, beside the boxes:
    # Gx[i] x_t <= gx[i] for the state slots t = 1..T-1, Gu[i] u_t <= gu[i] for
    # every input slot.  Gx f64 [n_sub, n_cx, nx], gx f64 [n_sub, n_cx]; None = none.
    Gx: Optional[np.ndarray] = None
    gx: Optional[np.ndarray] = None
    Gu: Optional[np.ndarray] = None
    gu: Optional[np.ndarray] = None

    @property
    def r_sub(self) -> int:
        """Rows of Phi owned by one subsystem: nx*T state rows + nu*(T-1) input rows."""
        return self.nx * self.T + self.nu * (self.T - 1)

    def neighbours(self, i: int) -> np.ndarray:
        return self.adj_idx[self.adj_ptr[i]:self.adj_ptr[i + 1]]

    def dense_A(self) -> np.ndarray:
        """Global A (N*nx square); only for small instances and host-side dynamics."""
        n, nx = self.n_sub, self.nx
        A = np.zeros((n * nx, n * nx))
        for i in range(n):
            A[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx] = self.A_diag[i]
            for e in range(self.adj_ptr[i], self.adj_ptr[i + 1]):
                j = int(self.adj_idx[e])
                A[i * nx:(i + 1) * nx, j * nx:(j + 1) * nx] = self.A_off[e]
        return A

    def dense_B(self) -> np.ndarray:
        n, nx, nu = self.n_sub, self.nx, self.nu
        B = np.zeros((n * nx, n * nu))
        for i in range(n):
            B[i * nx:(i + 1) * nx, i * nu:(i + 1) * nu] = self.B[i]
        return B


def chain_graph(n: int):
    """CSR of a path graph 0-1-...-(n-1)."""
    ptr = [0]
    idx: List[int] = []
    for i in range(n):
        if i > 0:
            idx.append(i - 1)
        if i < n - 1:
            idx.append(i + 1)
        ptr.append(len(idx))
    return np.asarray(ptr, np.int32), np.asarray(idx, np.int32)


def grid_graph(n: int, rows: Optional[int] = None):
    """CSR of a 4-neighbour grid with n nodes filled row-major.

    rows = floor(sqrt(n)) by default, cols = ceil(n / rows); the last row may be
    partial.  Returns (ptr, idx, (rows, cols)).
    """
    if rows is None:
        rows = max(1, int(math.isqrt(n)))
    cols = -(-n // rows)
    ptr = [0]
    idx: List[int] = []
    for v in range(n):
        rr, cc = divmod(v, cols)
        cand = []
        if rr > 0:
            cand.append(v - cols)
        if cc > 0:
            cand.append(v - 1)
        if cc < cols - 1 and v + 1 < n:
            cand.append(v + 1)
        if v + cols < n:
            cand.append(v + cols)
        idx.extend(sorted(cand))
        ptr.append(len(idx))
    return np.asarray(ptr, np.int32), np.asarray(idx, np.int32), (rows, cols)


def _plant(rng, n, adj_ptr, adj_idx):
    """Draw k_i, d_i then a_ij in CSR order; return (A_diag, A_off, B)."""
    A_diag = np.zeros((n, 2, 2))
    for i in range(n):
        k = rng.uniform(0.5, 1.5)
        dd = rng.uniform(0.1, 0.5)
        A_diag[i] = [[1.0, 0.1], [-0.1 * k, 1.0 - 0.1 * dd]]
    nnz = int(adj_ptr[-1])
    A_off = np.zeros((nnz, 2, 2))
    for e in range(nnz):
        a = rng.uniform(-0.1, 0.1)
        A_off[e] = [[0.0, 0.0], [a, a]]
    B = np.zeros((n, 2, 1))
    B[:, 1, 0] = 0.1
    return A_diag, A_off, B


def make_instance(n: int, T: int, d: int, *, graph: str = "chain", seed: int = 0,
                  boxes: bool = True, x0_dist: str = "uniform", rng=None,
                  rho: float = 1.0, eps: float = 1e-4, max_iter: int = 5000,
                  mpc_steps: int = 50, grid_rows: Optional[int] = None,
                  x_bound: float = 1.0, u_bound: float = 2.0, name: str = "") -> Problem:
    """Build one instance of the randomised chain/grid plant.

    boxes=True gives |x| <= x_bound and |u| <= u_bound for every subsystem.
    x0_dist: "normal" (N(0,1)) or "uniform" (U[-0.9, 0.9]).
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    if graph == "chain":
        ptr, idx = chain_graph(n)
        shape = None
    elif graph == "grid":
        ptr, idx, shape = grid_graph(n, grid_rows)
    else:
        raise ValueError(graph)
    A_diag, A_off, B = _plant(rng, n, ptr, idx)
    if x0_dist == "normal":
        x0 = rng.standard_normal((n, 2))
    elif x0_dist == "uniform":
        x0 = rng.uniform(-0.9, 0.9, (n, 2))
    else:
        raise ValueError(x0_dist)
    if boxes:
        x_lo, x_hi = np.full((n, 2), -x_bound), np.full((n, 2), x_bound)
        u_lo, u_hi = np.full((n, 1), -u_bound), np.full((n, 1), u_bound)
    else:
        x_lo = x_hi = u_lo = u_hi = None
    return Problem(n_sub=n, nx=2, nu=1, T=T, d=d, adj_ptr=ptr, adj_idx=idx,
                   A_diag=A_diag, A_off=A_off, B=B,
                   q=np.ones((n, 2)), r=np.ones((n, 1)),
                   x_lo=x_lo, x_hi=x_hi, u_lo=u_lo, u_hi=u_hi,
                   rho=rho, eps_p=eps, eps_d=eps, max_iter=max_iter, x0=x0,
                   mpc_steps=mpc_steps, name=name, graph=graph, grid_shape=shape)


def make_general(n: int, T: int, d: int, nx: int, nu: int, *, graph: str = "chain", seed: int = 0,
                 boxes: bool = True, x_bound: float = 1.0, u_bound: float = 2.0, max_iter: int = 5000,
                 name: str = "") -> Problem:
    """A plant of any state and input size (1..4 each): A_ii = 0.8 I + E with
    E ~ U[-0.1, 0.1], B_ii ~ U[0, 0.3], and couplings that enter through the
    neighbour's input directions, A_ij = B_ii C_ij with C_ij ~ U[-0.3, 0.3]
    (as in the chain plant, where the coupling enters the input-driven state;
    this keeps the d-local problem feasible).  Q = I, R = I; x0 ~ U[-0.9,
    0.9].  Draw order (numpy PCG64 `default_rng(seed)`): per subsystem E then
    B_ii, then per CSR entry C_ij, then x0."""
    rng = np.random.default_rng(seed)
    if graph == "chain":
        ptr, idx = chain_graph(n)
        shape = None
    else:
        ptr, idx, shape = grid_graph(n)
    A_diag = np.zeros((n, nx, nx))
    B = np.zeros((n, nx, nu))
    for i in range(n):
        A_diag[i] = 0.8 * np.eye(nx) + rng.uniform(-0.1, 0.1, (nx, nx))
        B[i] = rng.uniform(0.0, 0.3, (nx, nu))
    nnz = int(ptr[-1])
    A_off = np.zeros((nnz, nx, nx))
    for i in range(n):
        for e in range(ptr[i], ptr[i + 1]):
            A_off[e] = B[i] @ rng.uniform(-0.3, 0.3, (nu, nx))
    x0 = rng.uniform(-0.9, 0.9, (n, nx))
    if boxes:
        x_lo, x_hi = np.full((n, nx), -x_bound), np.full((n, nx), x_bound)
        u_lo, u_hi = np.full((n, nu), -u_bound), np.full((n, nu), u_bound)
    else:
        x_lo = x_hi = u_lo = u_hi = None
    return Problem(n_sub=n, nx=nx, nu=nu, T=T, d=d, adj_ptr=ptr, adj_idx=idx,
                   A_diag=A_diag, A_off=A_off, B=B, q=np.ones((n, nx)), r=np.ones((n, nu)),
                   x_lo=x_lo, x_hi=x_hi, u_lo=u_lo, u_hi=u_hi, rho=1.0, eps_p=1e-4, eps_d=1e-4,
                   max_iter=max_iter, x0=x0, mpc_steps=10, name=name, graph=graph, grid_shape=shape)


def with_block_costs(p: Problem, seed: int, coupling: float = 0.5) -> Problem:
    """A copy of p whose cost blocks Q_i, R_i are full symmetric positive
    definite matrices: M M^T / n + 0.5 I with M ~ U[-coupling, coupling] plus
    the identity (numpy PCG64 `default_rng(seed)`, Q_i then R_i per subsystem,
    subsystem-major).  The diagonal q, r are set to the blocks' diagonals."""
    rng = np.random.default_rng(seed)
    nx, nu = p.nx, p.nu
    Q = np.empty((p.n_sub, nx, nx))
    R = np.empty((p.n_sub, nu, nu))
    for i in range(p.n_sub):
        M = np.eye(nx) + rng.uniform(-coupling, coupling, (nx, nx))
        Q[i] = M @ M.T / nx + 0.5 * np.eye(nx)
        M = np.eye(nu) + rng.uniform(-coupling, coupling, (nu, nu))
        R[i] = M @ M.T / nu + 0.5 * np.eye(nu)
    out = dataclasses.replace(p, Q_blk=Q, R_blk=R, q=np.array([np.diag(b) for b in Q]),
                              r=np.array([np.diag(b) for b in R]),
                              name=(p.name + "_blockQR") if p.name else "")
    return out


def with_coupled_constraints(p: Problem, seed: int, n_cx: int = 2, n_cu: int = 0,
                             g_range: tuple = (0.4, 0.8)) -> Problem:
    """A copy of p with coupled per-slot constraints: n_cx half-spaces
    a^T x_t <= g on each subsystem's state and n_cu on its input, a a unit
    vector of random direction, g ~ U[g_range] (so 0 is strictly feasible).
    Draw order (numpy PCG64 `default_rng(seed)`): per subsystem, the n_cx state
    rows (a then g), then the n_cu input rows.  Full cost blocks are added when
    p has none (the coupled Phi-step runs on the slot QP)."""
    rng = np.random.default_rng(seed)
    nx, nu = p.nx, p.nu
    Gx = np.zeros((p.n_sub, n_cx, nx)); gx = np.zeros((p.n_sub, n_cx))
    Gu = np.zeros((p.n_sub, n_cu, nu)); gu = np.zeros((p.n_sub, n_cu))
    for i in range(p.n_sub):
        for k in range(n_cx):
            a = rng.normal(size=nx)
            Gx[i, k] = a / np.linalg.norm(a)
            gx[i, k] = rng.uniform(*g_range)
        for k in range(n_cu):
            a = rng.normal(size=nu)
            Gu[i, k] = a / np.linalg.norm(a)
            gu[i, k] = rng.uniform(*g_range)
    base = p if p.Q_blk is not None else with_block_costs(p, seed + 1)
    return dataclasses.replace(base, Gx=Gx if n_cx else None, gx=gx if n_cx else None,
                               Gu=Gu if n_cu else None, gu=gu if n_cu else None,
                               name=(base.name + "_coupled") if base.name else "")


# --- the five workloads -------------------------------------------------------

def chain10(seed: int = 0) -> Problem:
    """Chain N=10, T=5, d=1, Q=R=I, no boxes, rho=1, eps=1e-4, x0~N(0,1), 20 MPC steps."""
    return make_instance(10, 5, 1, graph="chain", seed=seed, boxes=False,
                         x0_dist="normal", mpc_steps=20, name="chain_N10_T5_d1")


def chain1024(seed: int = 0) -> Problem:
    """Chain N=1024, T=10, d=3, |x|<=1, |u|<=2, x0~U[-0.9,0.9], 50 MPC steps.

    max_iter = 1000: some draws of x0 put a subsystem where the boxes cannot be
    met (state 1 keeps integrating state 2 while |u| <= 2 moves state 2 by at
    most 0.2 per step); those MPC steps never reach eps and stop at the cap."""
    return make_instance(1024, 10, 3, graph="chain", seed=seed, boxes=True,
                         x0_dist="uniform", mpc_steps=50, max_iter=1000,
                         name="chain_N1024_T10_d3_box")


def grid64(seed: int = 0) -> Problem:
    """64x64 4-neighbour grid (4096 subsystems), T=10, d=2, boxes, 50 MPC steps."""
    return make_instance(4096, 10, 2, graph="grid", seed=seed, boxes=True,
                         x0_dist="uniform", mpc_steps=50, grid_rows=64, max_iter=1000,
                         name="grid_64x64_T10_d2_box")


def batch_instance(index: int) -> Problem:
    """Instance `index` of the mixed batch: seed = index; coin, N~U{16..512},
    T~U{5..15}, d~U{1..3} drawn first from that seed, then the plant."""
    rng = np.random.default_rng(index)
    graph = "grid" if rng.integers(0, 2) == 1 else "chain"
    n = int(rng.integers(16, 513))
    T = int(rng.integers(5, 16))
    d = int(rng.integers(1, 4))
    return make_instance(n, T, d, graph=graph, rng=rng, boxes=True, x0_dist="uniform",
                         mpc_steps=50, max_iter=1000, name=f"batch{index}_{graph}_N{n}_T{T}_d{d}")


def batch256(count: int = 256) -> List[Problem]:
    """The mixed batch of `count` independent instances (seed = index)."""
    return [batch_instance(i) for i in range(count)]


def random_x0(n_sub: int, count: int, seed: int, lo: float = -0.9, hi: float = 0.9) -> np.ndarray:
    """`count` random initial states U[lo,hi]^(n_sub x 2) (learned warm-start data)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (count, n_sub, 2))
