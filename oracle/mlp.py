"""Reference MLP for the per-edge multipole-rank selector, FP64 NumPy.

Network: x [nin] -> h1 = relu(x W1 + b1) [H] -> h2 = relu(h1 W2 + b2) [H]
-> y = h2 W3 + b3 [nout]; loss = mean over samples and outputs of (y - t)^2.
Weights are stored row-major: W1 [nin, H], W2 [H, H], W3 [H, nout].  The
flat parameter vector is W1, b1, W2, b2, W3, b3 in that order.  Adam uses
beta1 = 0.9, beta2 = 0.999, eps = 1e-8 with bias correction.

This is the CPU reference for the GPU training and inference kernels (the
selector is this build's addition to the paper's method).  Test
infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def sizes(nin, H, nout):
    return [(nin, H), (H,), (H, H), (H,), (H, nout), (nout,)]


def nparams(nin, H, nout):
    return sum(int(np.prod(s)) for s in sizes(nin, H, nout))


def unpack(theta, nin, H, nout):
    out, o = [], 0
    for s in sizes(nin, H, nout):
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def forward(theta, X, nin, H, nout):
    W1, b1, W2, b2, W3, b3 = unpack(theta, nin, H, nout)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (z1, h1, z2, h2)


def loss_and_grad(theta, X, T, nin, H, nout):
    W1, b1, W2, b2, W3, b3 = unpack(theta, nin, H, nout)
    y, (z1, h1, z2, h2) = forward(theta, X, nin, H, nout)
    n = X.shape[0]
    d = y - T
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (n * nout)
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    dz2 = dh2 * (z2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2.T
    dz1 = dh1 * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init(nin, H, nout, seed):
    """He-uniform weights, zero biases (the GPU library draws its own; tests
    pass weights explicitly)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in sizes(nin, H, nout):
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[0])
            parts.append(rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)
