"""FP64 oracle of the warm-start network (test infrastructure only).

Three layers, x -> GELU(x W1 + b1) -> GELU(. W2 + b2) -> . W3 + b3, exact GELU
0.5 x (1 + erf(x / sqrt 2)), loss = mean squared error.  Gradients by the
chain rule, written out layer by layer.  `bf16=True` rounds the operands of
every product to bfloat16 (round to nearest even) at the points where the GPU
kernels hold them in BF16, with the products themselves in FP64.  The
optimiser is AdamW (Adam with bias-corrected moments and decoupled weight
decay, Loshchilov & Hutter): w <- w (1 - lr wd) - lr m_hat / (sqrt(v_hat) + eps).
Pinned by finite differences and closed-form Adam steps in
tests/test_mlp_oracle.py.
"""
import math

import numpy as np

_erf = np.vectorize(math.erf)


def round_bf16(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(P, x, bf16=False):
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    h1p = r(x) @ r(P["W1"]) + P["b1"]
    a1 = gelu(h1p)
    h2p = r(a1) @ r(P["W2"]) + P["b2"]
    a2 = gelu(h2p)
    y = r(a2) @ r(P["W3"]) + P["b3"]
    return y, (h1p, a1, h2p, a2)


def loss_and_grads(P, x, t, bf16=False):
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    y, (h1p, a1, h2p, a2) = forward(P, x, bf16)
    n = y.size
    res = y - t
    loss = float(np.mean(res * res))
    dy = 2.0 * res / n
    G = {}
    G["W3"] = r(a2).T @ r(dy)
    G["b3"] = dy.sum(0)
    da2 = r(dy) @ r(P["W3"]).T
    dh2 = da2 * gelu_grad(h2p)
    G["W2"] = r(a1).T @ r(dh2)
    G["b2"] = dh2.sum(0)
    da1 = r(dh2) @ r(P["W2"]).T
    dh1 = da1 * gelu_grad(h1p)
    G["W1"] = r(x).T @ r(dh1)
    G["b1"] = dh1.sum(0)
    return loss, G


def adamw_step(w, g, m, v, step, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW update of the flat parameter vector w (FP64) with gradient g
    and moment estimates m, v after `step - 1` updates; returns (w, m, v)."""
    w, g, m, v = (np.asarray(a, np.float64) for a in (w, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** step)
    v_hat = v / (1.0 - b2 ** step)
    w = w * (1.0 - lr * wd) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return w, m, v
