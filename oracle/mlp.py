"""FP64 reference of the learned root-find start (test infrastructure only).

The network 6 -> 32 -> 32 -> 1 with ReLU (parameters W1[32][6], b1[32], W2[32][32], b2[32],
W3[32], b3) and its mean-squared-error gradient, written as plain matrix products; the
features of a cell from E = T^tt - pi^tt, M^2 and Pi; and the exact target
y = 10 ln(e / e_conf) with e the root of Eq. (eInferred), e_conf = sqrt(4E^2 - 3M^2) - E.
It shares no code with the CUDA kernels.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 6, 32
NPARAM = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + N_H * N_IN].reshape(N_H, N_IN); o += N_H * N_IN
    b1 = p[o:o + N_H]; o += N_H
    W2 = p[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = p[o:o + N_H]; o += N_H
    W3 = p[o:o + N_H]; o += N_H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def forward(params, X, bf16=False):
    """y for rows of X; bf16 rounds weights (not biases) and each layer's input to bfloat16."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    r = bf16_round if bf16 else (lambda a: a)
    a0 = r(X)
    z1 = a0 @ r(W1).T + b1
    h1 = np.maximum(z1, 0.0)
    a1 = r(h1)
    z2 = a1 @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    a2 = r(h2)
    y = a2 @ r(W3) + b3
    return y, (a0, z1, a1, z2, a2)


def loss_and_grad(params, X, Y):
    """Mean squared error and its gradient by back-propagation (FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    y, (a0, z1, a1, z2, a2) = forward(params, X)
    n = len(Y)
    r = y - np.asarray(Y, dtype=np.float64)
    loss = np.mean(r * r)
    dy = 2.0 * r / n
    gW3 = a2.T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ a0
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def features(E, M2, Pi):
    """[(ln E - 1)/6, M^2/E^2, 5 Pi/E, ln(1 - M^2/E^2)/2, e_conf/E, |M|/E] and e_conf/E."""
    E, M2, Pi = (np.asarray(a, dtype=np.float64) for a in (E, M2, Pi))
    r2 = np.clip(M2 / (E * E), 0.0, 0.999999)
    r = np.sqrt(r2)
    ec = np.sqrt(4.0 - 3.0 * r2) - 1.0  # (sqrt(4E^2 - 3M^2) - E) / E
    X = np.stack([(np.log(E) - 1.0) / 6.0, r2, 5.0 * Pi / E, 0.5 * np.log(1.0 - r2), ec, r], axis=-1)
    return X, ec
