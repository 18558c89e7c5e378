"""Oracle: the Newton initial-guess network in plain FP64.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.

A 5 -> 64 -> 64 -> 1 perceptron with GELU activations (x Phi(x), exact erf
form) maps normalized features (ln V_prev, ln theta, tau/sigma, a, b) of an
element to the normalized residual ln V* - ln V_prev of its Newton solve
(Eq. momentum).  Loss: mean squared error over a batch.

Parameter vector layout (4609 values): W1[64][5], b1[64], W2[64][64], b2[64],
W3[64], b3; followed in the deployed vector by 12 normalization values
in_mean[5], in_std[5], out_mean, out_std.
"""
from __future__ import annotations

import numpy as np
from scipy import special

N_IN, N_H = 5, 64
N_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1   # 4609
N_NORM = 12


def unpack(theta: np.ndarray):
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = t[o:o + N_H * N_IN].reshape(N_H, N_IN); o += N_H * N_IN
    b1 = t[o:o + N_H]; o += N_H
    W2 = t[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = t[o:o + N_H]; o += N_H
    W3 = t[o:o + N_H]; o += N_H
    b3 = t[o]
    return W1, b1, W2, b2, W3, b3


def gelu(z):
    return 0.5 * z * (1.0 + special.erf(z / np.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + special.erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(theta, X):
    """X: [B, 5] normalized features -> (y [B], cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    y = H2 @ W3 + b3
    return y, (X, Z1, H1, Z2, H2)


def loss_and_grad(theta, X, t):
    """Mean squared error over the batch and its gradient (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    y, (X, Z1, H1, Z2, H2) = forward(theta, X)
    B = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    dW3 = H2.T @ dy
    db3 = dy.sum()
    dZ2 = np.outer(dy, W3) * gelu_prime(Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_prime(Z1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3, [db3]])
    return loss, g
