"""FP64 numpy reference of the learned kappa_P model (forward pass, loss gradient).

TEST INFRASTRUCTURE (see the package docstring).  The learned model stands in
for the solve of Eq. 10: it maps (y = beta hbar w, P) to the ratio
kappa_P / theta = F_P(y) / f(y).  Network: inputs
    x1 = asinh(y) / asinh(1000),   x2 = (ln P - ln 2) / (ln 32 - ln 2),
two hidden layers of 64 SiLU units, one linear output; loss = mean squared
error over the batch.  The flat parameter layout (4417 values) is
    W1[64][2], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
from __future__ import annotations

import numpy as np

H = 64
NPARAM = H * 2 + H + H * H + H + H + 1  # 4417
YSCALE = float(np.arcsinh(1000.0))
LNP0, LNP1 = float(np.log(2.0)), float(np.log(32.0))


def features(y, P):
    y = np.asarray(y, np.float64)
    P = np.broadcast_to(np.asarray(P, np.float64), y.shape)
    return np.stack([np.arcsinh(y) / YSCALE, (np.log(P) - LNP0) / (LNP1 - LNP0)], axis=-1)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    o = 0
    W1 = theta[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, W3, b3


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    out = h2 @ W3 + b3
    return out, (z1, h1, z2, h2)


def loss_and_grad(theta, x, t):
    """Mean squared error and its gradient with respect to the flat parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    out, (z1, h1, z2, h2) = forward(theta, x)
    n = len(t)
    r = out - t
    loss = float((r * r).mean())
    d3 = 2.0 * r / n                       # dL/dout
    gW3 = h2.T @ d3
    gb3 = d3.sum()
    d2 = np.outer(d3, W3) * dsilu(z2)      # dL/dz2
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * dsilu(z1)             # dL/dz1
    gW1 = d1.T @ x
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g
