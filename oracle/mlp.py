"""Float64 reference of the learned selector's network (test infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing on the product
path).  It shares no code with the CUDA library.

The selector (the paper's adaptive solver selection, Sec. IV, with a small
network in place of its decision tree) maps 12 mode features to one score per
class with a multilayer perceptron:

    a1 = relu(W1 x + b1),  a2 = relu(W2 a1 + b2),  out = W3 a2 + b3.

Parameters are one flat vector: W1 [H x IN] row-major, b1 [H], W2 [H x H],
b2 [H], W3 [K x H], b3 [K].  The training loss is the masked mean squared
error sum(M (out - Y)^2) / sum(M) over a batch.  ``grad`` is backpropagation
written out layer by layer; ``adam_step`` is Adam (Kingma & Ba, ICLR 2015)
with bias correction.

Parity status: pinned in ``tests/test_oracle_pins.py`` by central finite
differences of the loss on random parameters (the gradient is not checked
against itself), by the closed-form gradient of a network whose last hidden
layer is dead, and by Adam's first step, which moves every parameter with a
non-zero gradient by exactly lr against the gradient's sign.
"""
from __future__ import annotations

import numpy as np


def param_count(n_in: int, h: int, k: int) -> int:
    return h * n_in + h + h * h + h + k * h + k


def unpack(params, n_in: int, h: int, k: int):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == param_count(n_in, h, k)
    o = 0
    W1 = p[o:o + h * n_in].reshape(h, n_in); o += h * n_in
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    W3 = p[o:o + k * h].reshape(k, h); o += k * h
    b3 = p[o:o + k]
    return W1, b1, W2, b2, W3, b3


def forward(params, X, n_in: int, h: int, k: int):
    """Outputs (B x k) and the cache of pre-activations and activations."""
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in, h, k)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    out = a2 @ W3.T + b3
    return out, (X, z1, a1, z2, a2)


def loss(params, X, Y, M, n_in: int, h: int, k: int) -> float:
    out, _ = forward(params, X, n_in, h, k)
    M = np.asarray(M, dtype=np.float64)
    cnt = M.sum() if M.sum() > 0 else 1.0
    return float((M * (out - Y) ** 2).sum() / cnt)


def grad(params, X, Y, M, n_in: int, h: int, k: int):
    """(loss, gradient) by backpropagation through the three layers."""
    W1, b1, W2, b2, W3, b3 = unpack(params, n_in, h, k)
    out, (X, z1, a1, z2, a2) = forward(params, X, n_in, h, k)
    M = np.asarray(M, dtype=np.float64)
    cnt = M.sum() if M.sum() > 0 else 1.0
    L = float((M * (out - Y) ** 2).sum() / cnt)
    g3 = 2.0 * (out - Y) * M / cnt          # dL/d out
    dW3 = g3.T @ a2
    db3 = g3.sum(axis=0)
    g2 = (g3 @ W3) * (z2 > 0)               # dL/d z2
    dW2 = g2.T @ a1
    db2 = g2.sum(axis=0)
    g1 = (g2 @ W2) * (z1 > 0)               # dL/d z1
    dW1 = g1.T @ X
    db1 = g1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, g


def adam_step(params, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step at step number t (1-based); returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
