"""FP64 oracle of the surrogate network's forward and backward pass.

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the product).  The
network: x [m][512] -> four layers h = GELU(W h + b) with W [512][512] -> output
y = W_out h + b_out (18) ; loss = mean over rows and outputs of (y - t)^2.
GELU is the exact one, z Phi(z) with the Gaussian CDF written with erf.  The
flat parameter layout: for each hidden layer W [out][in] then b, then W_out
[18][512] and b_out [18].  Pinned by central finite differences in the tests.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN, LAYERS, OUT, IN = 512, 4, 18, 512
_erf = np.vectorize(math.erf, otypes=[np.float64])


def n_params() -> int:
    return LAYERS * (HIDDEN * IN + HIDDEN) + OUT * HIDDEN + OUT


def unflatten(p):
    p = np.asarray(p, dtype=np.float64)
    layers, o = [], 0
    for _ in range(LAYERS):
        W = p[o:o + HIDDEN * IN].reshape(HIDDEN, IN)
        o += HIDDEN * IN
        b = p[o:o + HIDDEN]
        o += HIDDEN
        layers.append((W, b))
    Wo = p[o:o + OUT * HIDDEN].reshape(OUT, HIDDEN)
    o += OUT * HIDDEN
    bo = p[o:o + OUT]
    return layers, (Wo, bo)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(p, x):
    layers, (Wo, bo) = unflatten(p)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for W, b in layers:
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z)
    y = h @ Wo.T + bo
    return y, (cache, h)


def loss_and_grad(p, x, t):
    """Mean squared error over rows and outputs and its gradient (flat)."""
    layers, (Wo, bo) = unflatten(p)
    t = np.asarray(t, dtype=np.float64)
    y, (cache, hlast) = forward(p, x)
    m = y.shape[0]
    d = y - t
    loss = float(np.sum(d * d) / (m * OUT))
    dy = 2.0 * d / (m * OUT)
    grads = []
    dWo = dy.T @ hlast
    dbo = dy.sum(axis=0)
    dh = dy @ Wo
    for (W, b), (h, z) in zip(reversed(layers), reversed(cache)):
        dz = dh * gelu_grad(z)
        grads.append((dz.T @ h, dz.sum(axis=0)))
        dh = dz @ W
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.ravel())
        flat.append(db)
    flat.append(dWo.ravel())
    flat.append(dbo)
    return loss, np.concatenate(flat)


def loss_only(p, x, t):
    y, _ = forward(p, x)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.sum(d * d) / d.size)
