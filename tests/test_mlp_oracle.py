"""Pins of the FP64 warm-start network oracle: finite differences of every
parameter gradient on a small network, the GELU derivative, bf16 rounding,
closed-form AdamW steps."""
import numpy as np

from oracle import mlp_oracle as M


def _params(rng, I, H, O):
    return {"W1": rng.normal(size=(I, H)) * 0.5, "b1": rng.normal(size=H) * 0.1,
            "W2": rng.normal(size=(H, H)) * 0.3, "b2": rng.normal(size=H) * 0.1,
            "W3": rng.normal(size=(H, O)) * 0.3, "b3": rng.normal(size=O) * 0.1}


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    P = _params(rng, 4, 6, 5)
    x, t = rng.normal(size=(7, 4)), rng.normal(size=(7, 5))
    loss, G = M.loss_and_grads(P, x, t)
    h = 1e-6
    for name, W in P.items():
        flat = W.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = M.loss_and_grads(P, x, t)
            flat[idx] = old - h
            lm, _ = M.loss_and_grads(P, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[name].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (name, idx)


def test_gelu_and_derivative():
    x = np.linspace(-5, 5, 101)
    assert np.allclose(M.gelu(np.array([0.0, 1.0])), [0.0, 0.8413447460685429], atol=1e-12)
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.allclose(fd, M.gelu_grad(x), atol=1e-8)


def test_bf16_rounding():
    assert M.round_bf16(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is exactly half-way between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert M.round_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert M.round_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    v = np.random.default_rng(1).normal(size=1000)
    assert np.max(np.abs(M.round_bf16(v) - v) / np.abs(v)) <= 2 ** -8


def test_adamw_first_step_is_a_sign_step():
    # from m = v = 0 the bias-corrected moments are g and g^2 exactly:
    # w1 = w0 (1 - lr wd) - lr g / (|g| + eps)
    rng = np.random.default_rng(2)
    w0, g = rng.normal(size=50), rng.normal(size=50)
    lr, wd, eps = 1e-2, 0.1, 1e-8
    w1, m, v = M.adamw_step(w0, g, np.zeros(50), np.zeros(50), 1, lr, wd, eps=eps)
    assert np.allclose(w1, w0 * (1 - lr * wd) - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adamw_constant_gradient_moves_by_lr_each_step():
    # with a constant gradient the bias corrections make m_hat = g and
    # v_hat = g^2 at every step, so each step (no decay) moves by lr g / (|g| + eps)
    rng = np.random.default_rng(3)
    w, g = rng.normal(size=20), rng.normal(size=20)
    m, v = np.zeros(20), np.zeros(20)
    lr = 3e-3
    for step in range(1, 30):
        w_new, m, v = M.adamw_step(w, g, m, v, step, lr, 0.0)
        assert np.allclose(w - w_new, lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
        w = w_new
