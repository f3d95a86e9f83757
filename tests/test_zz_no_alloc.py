"""The allocation-free single-patch re-factorisation against the precomputation.

dlmpc_factor_patch_noalloc is for callers that cannot allocate device memory
while their control loop runs (a real-time thread refreshing patch operators
after a model update, or code tied to a fixed memory budget).  Its outputs
must equal what dlmpc_precompute stores for the same patch: the projector
N N^T onto the null space and the min-norm offsets q, within the tolerance of
the operator parity tests.  Several calls in a row share the library's static
workspace, so each call is checked, including a repeat of the first one.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _call(lib, torch, Z, rhs, k_cap):
    m, D = Z.shape
    Zd = torch.tensor(Z, dtype=torch.float64, device="cuda")
    Rd = torch.tensor(rhs, dtype=torch.float64, device="cuda")
    Nd = torch.full((D, k_cap), 7.0, dtype=torch.float64, device="cuda")
    qd = torch.empty((rhs.shape[0], D), dtype=torch.float64, device="cuda")
    rn = torch.empty(2, dtype=torch.int32, device="cuda")
    fe = torch.empty(1, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    rc = lib.dlmpc_factor_patch_noalloc(vp(Zd.data_ptr()), m, D, vp(Rd.data_ptr()), rhs.shape[0],
                                        vp(Nd.data_ptr()), k_cap, vp(qd.data_ptr()), vp(rn.data_ptr()),
                                        vp(fe.data_ptr()), vp(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, Nd.cpu().numpy(), qd.cpu().numpy(), rn.cpu().numpy(), float(fe.item())


def test_noalloc_factorisation_matches_precompute():
    import torch
    import paper_2103_14990_gb300 as pkg
    lib = pkg.load_library()
    p = I.make_instance(16, 10, 3, seed=1, boxes=True)
    s = pkg.Solver([p])
    for j in [7, 0, 15, 7]:                       # interior, end, end, interior again
        N_ref, q_ref = s.operator(j)
        blk = O.column_block(p, j)
        D = blk.Z.shape[1]
        rc, N, q, rn, feas = _call(lib, torch, blk.Z, blk.rhs, D)
        assert rc == 0
        k = int(rn[1])
        assert k == N_ref.shape[1] and int(rn[0]) == D - k
        assert feas < 1e-9
        assert np.all(N[:, k:] == 0.0)
        assert np.max(np.abs(N[:, :k] @ N[:, :k].T - N_ref @ N_ref.T)) < TOL
        assert np.max(np.abs(q - q_ref)) < TOL
    s.close()


def test_noalloc_rejects_blocks_above_the_static_workspace():
    import torch
    import paper_2103_14990_gb300 as pkg
    lib = pkg.load_library()
    m, D = 1100, 1000                               # D*m alone exceeds 2^20 doubles
    vp = ctypes.c_void_p
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    a = vp(dummy.data_ptr())
    rc = lib.dlmpc_factor_patch_noalloc(a, m, D, a, 2, a, 8, a, a, a, None)
    assert rc == pkg.DLMPC_ERR_ARG


def _dup_row_block():
    """An interior chain patch block with its first row appended again (same
    right-hand side): the rank drops by one against the row count."""
    p = I.make_instance(16, 10, 3, seed=1, boxes=True)
    blk = O.column_block(p, 7)
    Z = np.vstack([blk.Z, blk.Z[:1]])
    rhs = np.hstack([blk.rhs, blk.rhs[:, :1]])
    return Z, rhs


def test_noalloc_duplicated_row_rank_and_projector():
    """rank = the rank of Z (one less than its rows), feas ~ 0, and the
    projector N N^T equal to the one of scipy's SVD null space."""
    import scipy.linalg
    import torch
    import paper_2103_14990_gb300 as pkg
    lib = pkg.load_library()
    Z, rhs = _dup_row_block()
    m, D = Z.shape
    r_ref = np.linalg.matrix_rank(Z)
    assert r_ref < m
    Nn = scipy.linalg.null_space(Z)
    for _ in range(2):                              # two calls in a row on the shared workspace
        rc, N, q, rn, feas = _call(lib, torch, Z, rhs, D)
        assert rc == 0
        assert int(rn[0]) == r_ref and int(rn[1]) == D - r_ref == Nn.shape[1]
        k = int(rn[1])
        assert feas < 1e-9
        assert np.max(np.abs(N[:, :k] @ N[:, :k].T - Nn @ Nn.T)) < TOL
        assert np.all(N[:, k:] == 0.0)
        q_ref = np.linalg.lstsq(Z, rhs.T, rcond=None)[0].T          # min-norm solutions
        assert np.max(np.abs(q - q_ref)) < TOL


def test_noalloc_inconsistent_rhs_reports_infeasibility():
    """The duplicated row with a different right-hand side has no solution:
    feas (max |Z q - rhs|) is reported well above zero."""
    import torch
    import paper_2103_14990_gb300 as pkg
    lib = pkg.load_library()
    Z, rhs = _dup_row_block()
    rhs = rhs.copy()
    rhs[:, -1] = rhs[:, 0] + 1.0                    # row m-1 repeats row 0 with another value
    rc, N, q, rn, feas = _call(lib, torch, Z, rhs, Z.shape[1])
    assert rc == 0
    assert feas > 0.1


def test_noalloc_null_space_wider_than_the_buffer():
    """k_cap below the nullity: DLMPC_ERR_CAPACITY, the true sizes in
    rank_nullity, and only the first k_cap columns written, each a unit vector
    of the null space."""
    import torch
    import paper_2103_14990_gb300 as pkg
    lib = pkg.load_library()
    p = I.make_instance(16, 10, 3, seed=1, boxes=True)
    blk = O.column_block(p, 7)
    D = blk.Z.shape[1]
    k_true = D - blk.rank
    k_cap = k_true - 5
    rc, N, q, rn, feas = _call(lib, torch, blk.Z, blk.rhs, k_cap)
    assert rc == pkg.DLMPC_ERR_CAPACITY
    assert int(rn[1]) == k_true and int(rn[0]) == blk.rank
    assert N.shape == (D, k_cap)
    assert np.allclose(N.T @ N, np.eye(k_cap), atol=1e-10)
    assert np.max(np.abs(blk.Z @ N)) < 1e-10
    assert feas < 1e-9
