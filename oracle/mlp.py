"""CPU oracle for the planner's network (fp64 numpy).  TEST INFRASTRUCTURE ONLY.

The perceptron of the cost model, written out plainly:
    h1 = relu(x W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 . w3 + b3,   L = mean((y - t)^2)
with its gradient by the chain rule.  The flat parameter layout matches the library's:
[W1 (in x 64), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1)].
Pinned by central finite differences of L (tests/test_mlp_oracle.py).
"""
from __future__ import annotations

import numpy as np

H = 64


def param_count(in_dim: int) -> int:
    return in_dim * H + H + H * H + H + H + 1


def split(p: np.ndarray, in_dim: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + in_dim * H].reshape(in_dim, H); o += in_dim * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, x):
    x = np.asarray(x, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = split(p, x.shape[1])
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ w3 + b3, h1, h2


def loss(p, x, t):
    y, _, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(p, x, t):
    """dL/dp for L = mean((y - t)^2), by the chain rule through both ReLU layers."""
    x = np.asarray(x, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = split(p, x.shape[1])
    y, h1, h2 = forward(p, x)
    dy = 2.0 * (y - np.asarray(t, np.float64)) / len(y)
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, w3) * (h2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (h1 > 0)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def init(in_dim: int, seed: int = 0) -> np.ndarray:
    """He-style initialisation (a seeded input, not part of the arithmetic under test)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / in_dim), (in_dim, H))
    W2 = rng.normal(0, np.sqrt(2.0 / H), (H, H))
    w3 = rng.normal(0, np.sqrt(1.0 / H), H)
    return np.concatenate([W1.ravel(), np.full(H, 0.01), W2.ravel(), np.full(H, 0.01), w3, [0.0]])
