"""Failure handling on the GPU without faulting it: a bounded wait that runs
out (one CTA never arrives at the iteration barrier) and non-finite inputs
come back as error codes, and the context keeps working afterwards."""
import numpy as np
import pytest

from paper_2103_14990_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _solver(p):
    import paper_2103_14990_gb300 as pkg
    return pkg.Solver([p])


def test_barrier_timeout_is_reported_and_recoverable():
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.make_instance(40, 6, 2, seed=3, boxes=True)
    s = _solver(p)
    assert s.info()["grid_ctas"] >= 2
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    u = torch.zeros(p.n_sub, 1, device="cuda")
    s.set_option(pkg.OPT_TIMEOUT_MS, 100)
    s.set_option(pkg.OPT_TEST_SKIP_ARRIVAL, 1)
    with pytest.raises(pkg.DlmpcError) as e:
        s.step(x, u, None, warm=pkg.WARM_COLD)
    assert e.value.code == pkg.DLMPC_ERR_TIMEOUT
    # the same context steps normally once the test switch is off
    s.set_option(pkg.OPT_TEST_SKIP_ARRIVAL, -1)
    rc, st = s.step(x, u, None, warm=pkg.WARM_COLD)
    assert rc in (pkg.DLMPC_OK, pkg.DLMPC_MAX_ITER) and st[0]["iters"] > 0
    s.close()


def test_nonfinite_state_is_reported():
    import torch
    import paper_2103_14990_gb300 as pkg
    p = I.make_instance(12, 5, 1, seed=4, boxes=False, x0_dist="normal")
    s = _solver(p)
    x0 = p.x0.astype(np.float32).copy()
    x0[3, 1] = np.nan
    x = torch.tensor(x0, device="cuda")
    u = torch.zeros(p.n_sub, 1, device="cuda")
    with pytest.raises(pkg.DlmpcError) as e:
        s.step(x, u, None, warm=pkg.WARM_COLD)
    assert e.value.code == pkg.DLMPC_ERR_NONFINITE
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    rc, st = s.step(x, u, None, warm=pkg.WARM_COLD)
    assert rc == pkg.DLMPC_OK
    s.close()
