"""Learned warm start on the GPU: the network kernels against the FP64 network
oracle, training, and the gain of the learned start over a cold start with
the polished solution at the same accuracy."""
import numpy as np
import pytest

from oracle import dlmpc_oracle as O
from oracle import mlp_oracle as M
from paper_2103_14990_gb300 import instances as I

pytestmark = pytest.mark.gpu


def relerr(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.fixture(scope="module")
def small_net():
    import torch
    import paper_2103_14990_gb300 as pkg
    rng = np.random.default_rng(3)
    I_, H, O_ = 14, 72, 40                  # ragged against the 64-wide tiles
    mlp = pkg.MLP(I_, H, O_, seed=5)
    p = M.round_bf16(mlp.get_params()).astype(np.float32)   # weights exactly representable in BF16
    mlp.set_params(p)
    n = 70
    x = M.round_bf16(rng.uniform(-1, 1, (n, I_))).astype(np.float32)
    t = rng.normal(size=(n, O_)).astype(np.float32)
    return mlp, p, x, t, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")


def test_forward_matches_oracle(small_net):
    mlp, p, x, t, xd, td = small_net
    P = {k: v.astype(np.float64) for k, v in mlp.unpack(p).items()}
    y = mlp.forward(xd).cpu().numpy()
    y_bf, _ = M.forward(P, x, bf16=True)
    y_64, _ = M.forward(P, x)
    assert relerr(y, y_bf) < 2e-3
    assert relerr(y, y_64) < 1e-2


def test_gradients_match_oracle(small_net):
    mlp, p, x, t, xd, td = small_net
    P = {k: v.astype(np.float64) for k, v in mlp.unpack(p).items()}
    g, loss = mlp.gradients(xd, td)
    G = mlp.unpack(g)
    l_bf, G_bf = M.loss_and_grads(P, x, t, bf16=True)
    l_64, G_64 = M.loss_and_grads(P, x, t)
    assert abs(loss - l_bf) / l_bf < 1e-4
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        assert relerr(G[name], G_bf[name]) < 5e-3, name       # same rounding points
        assert relerr(G[name], G_64[name]) < 3e-2, name       # BF16 against exact


def test_network_kernels_at_the_benchmark_sizes():
    """The learned start's network on the N = 1024 chain: 1024 rows (one per
    subsystem), 70 inputs (patch state and each member's plant blocks), two
    hidden layers of 256 and 812 outputs (Phi rows and Lambda of a
    subsystem): forward and gradients against the FP64 network oracle with
    the same BF16 rounding points, and against exact arithmetic."""
    import torch
    import paper_2103_14990_gb300 as pkg
    s = pkg.Solver([I.chain1024()])
    s.set_option(pkg.OPT_LEARN_PLANT, 1)
    d_in, d_out = s.learned_dims()
    s.close()
    assert (d_in, d_out) == (70, 812)
    rng = np.random.default_rng(11)
    mlp = pkg.MLP(d_in, 256, d_out, seed=12)
    p = M.round_bf16(mlp.get_params()).astype(np.float32)
    mlp.set_params(p)
    x = M.round_bf16(rng.uniform(-1, 1, (1024, d_in))).astype(np.float32)
    t = rng.normal(size=(1024, d_out)).astype(np.float32)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    P = {k: v.astype(np.float64) for k, v in mlp.unpack(p).items()}
    y = mlp.forward(xd).cpu().numpy()
    y_bf, _ = M.forward(P, x, bf16=True)
    y_64, _ = M.forward(P, x)
    assert relerr(y, y_bf) < 2e-3
    assert relerr(y, y_64) < 1e-2
    g, loss = mlp.gradients(xd, td)
    G = mlp.unpack(g)
    l_bf, G_bf = M.loss_and_grads(P, x, t, bf16=True)
    _, G_64 = M.loss_and_grads(P, x, t)
    assert abs(loss - l_bf) / l_bf < 1e-4
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        assert relerr(G[name], G_bf[name]) < 5e-3, name
        assert relerr(G[name], G_64[name]) < 3e-2, name
    mlp.close()


def test_adamw_steps_match_oracle():
    """Three training steps: each GPU update against the oracle's AdamW applied
    to the GPU's own gradient of that step (isolates the optimiser kernel)."""
    import torch
    import paper_2103_14990_gb300 as pkg
    rng = np.random.default_rng(4)
    mlp = pkg.MLP(10, 64, 12, seed=7)
    x = torch.tensor(rng.uniform(-1, 1, (96, 10)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.normal(size=(96, 12)), dtype=torch.float32, device="cuda")
    w = mlp.get_params().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    lr, wd = 2e-3, 0.05
    for step in range(1, 4):
        g, _ = mlp.gradients(x, t)
        mlp.train_step(x, t, lr, wd)
        w_ref, m, v = M.adamw_step(w, g.astype(np.float64), m, v, step, lr, wd)
        w_gpu = mlp.get_params().astype(np.float64)
        assert relerr(w_gpu - w, w_ref - w) < 1e-4, step
        w = w_gpu


def test_training_reduces_loss():
    import torch
    import paper_2103_14990_gb300 as pkg
    rng = np.random.default_rng(0)
    W = rng.normal(size=(14, 30))
    X = rng.uniform(-1, 1, (4096, 14))
    Y = np.tanh(X @ W) @ rng.normal(size=(30, 50)) * 0.3
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(Y, dtype=torch.float32, device="cuda")
    mlp = pkg.MLP(14, 128, 50, seed=1)
    first = mlp.train_step(xd[:1024], yd[:1024], 2e-3, 0.0, want_loss=True)
    for it in range(300):
        i = (it % 4) * 1024
        last = mlp.train_step(xd[i:i + 1024], yd[i:i + 1024], 2e-3, 0.0, want_loss=True)
    assert last < 0.1 * first


def test_learned_start_beats_cold_start_at_same_accuracy():
    """Chain N=64, T=10, d=3 with the benchmark's plant and boxes: train on
    converged closed-loop steps, evaluate on held-out visited states."""
    import paper_2103_14990_gb300 as pkg
    from paper_2103_14990_gb300 import warmstart as W
    p = I.make_instance(64, 10, 3, seed=0, boxes=True, x0_dist="uniform", max_iter=2000)
    x0s = I.random_x0(p.n_sub, 24, seed=100)
    pairs = W.closed_loop_pairs(p, x0s, steps=30)
    assert pairs.steps_used >= 200
    mlp = W.train(pairs, hidden=256, epochs=150, batch=1024, lr=1e-3, seed=0)
    assert W.prediction_error(mlp, pairs) < 0.25
    states, status = W.heldout_states(p, seed=999, trajectories=16, steps=30)
    keep = np.nonzero(status == 0)[0][::3]
    assert len(keep) >= 60
    ic, il, sc, sl, uc, ul = W.compare_starts(p, mlp, states[keep])
    assert np.all(sc == 0) and np.all(sl == 0)
    # the measured gain on this shape is about 5% fewer iterations
    assert il.mean() < 0.985 * ic.mean(), (il.mean(), ic.mean())
    assert np.mean(il < ic) > 0.5
    # polished solutions at a tight tolerance agree with the oracle's optimum
    sub = keep[:3]
    ic2, il2, sc2, sl2, uc2, ul2 = W.compare_starts(p, mlp, states[sub], eps=1e-6, max_iter=20000)
    o = O.Oracle(p)
    for b, k in enumerate(sub):
        ref = O.admm(o.lay, o.blocks, states[k], max_iter=20000, eps_p=1e-9, eps_d=1e-9)
        u_ref = o.control(ref).ravel()
        ul_b = ul2.reshape(len(sub), -1)[b]
        assert relerr(ul_b, u_ref) < 1e-4
