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
