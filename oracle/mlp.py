"""FP64 CPU definition of the design surrogate MLP.  TEST INFRASTRUCTURE ONLY.

Model (the surrogate of the benchmark's learned-screening workload):
    Z1 = X W1^T + b1,  H1 = GELU(Z1),  Z2 = H1 W2^T + b2,  H2 = GELU(Z2),
    y  = H2 w3 + b3,   loss = 0.5 mean_b (y_b - t_b)^2,
GELU(z) = z Phi(z) with Phi the standard normal CDF, trained with Adam
(bias-corrected first and second moments).  Parameters are one flat vector
in the order W1 [h][n_in], b1 [h], W2 [h][h], b2 [h], w3 [h], b3.
Plain numpy; matrix products are library calls, everything else is written
out.  Gradients are derived by hand (chain rule, below) and pinned by finite
differences in the tests.
"""
from __future__ import annotations

import math

import numpy as np

_SQRT1_2 = 1.0 / math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z * _SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z * _SQRT1_2)) + z * _INV_SQRT_2PI * np.exp(-0.5 * z * z)


def unpack(p, n_in, h):
    p = np.asarray(p, np.float64)
    o = 0
    W1 = p[o:o + h * n_in].reshape(h, n_in); o += h * n_in
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    w3 = p[o:o + h]; o += h
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def n_params(n_in, h):
    return h * n_in + h + h * h + h + h + 1


def forward(p, X, n_in, h):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, h)
    X = np.asarray(X, np.float64)
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    y = H2 @ w3 + b3
    return y, (X, Z1, H1, Z2, H2)


def loss_and_grad(p, X, t, n_in, h):
    """Loss and its gradient w.r.t. the flat parameter vector."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, h)
    y, (X, Z1, H1, Z2, H2) = forward(p, X, n_in, h)
    B = X.shape[0]
    r = y - np.asarray(t, np.float64)
    loss = 0.5 * np.mean(r * r)
    dy = r / B                                  # dL/dy
    dw3 = H2.T @ dy
    db3 = dy.sum()
    dZ2 = np.outer(dy, w3) * gelu_grad(Z2)      # dL/dZ2
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)            # dL/dZ1
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return loss, g


def adam(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def one_hot(materials, n_mat=4):
    """[B, n_vox] material ids -> [B, n_vox * n_mat] one-hot (voxel-major)."""
    m = np.asarray(materials).reshape(len(materials), -1)
    out = np.zeros((m.shape[0], m.shape[1] * n_mat))
    for q in range(n_mat):
        out[:, q::n_mat] = (m == q)
    return out
