"""FP64 oracle of the surrogate network: forward and backward pass, the
AdamW update, and a BF16 reading of the network's arithmetic.

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the product).  The
network: x [m][512] -> four layers h = GELU(W h + b) with W [512][512] -> output
y = W_out h + b_out (18) ; loss = mean over rows and outputs of (y - t)^2.
GELU is the exact one, z Phi(z) with the Gaussian CDF written with erf.  The
flat parameter layout: for each hidden layer W [out][in] then b, then W_out
[18][512] and b_out [18].

BF16 reading (``rounded=True``).  The network keeps FP32 master parameters
but multiplies BF16 values: the weight matrices, the input features, every
hidden activation h and every back-propagated pre-activation error dz are
rounded to the nearest BF16 value (8 significant bits, ties to even) where
they enter a product; biases, pre-activations z, outputs y and the errors
dy and dh stay unrounded.  Everything else is FP64.  This is a statement of
where the network's arithmetic loses precision, not of how any device tiles
it.

AdamW (Loshchilov and Hutter's decoupled weight decay, with Adam's bias
corrections): per step t, m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
w <- w - lr wd w on weight matrices only (biases are not decayed), then
w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pinned in the tests: the backward pass by central finite differences, BF16
rounding by the library's conversion and hand-worked ties, AdamW by the
closed form of its first step and of a constant gradient, and by torch's
AdamW in FP64.
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


def bf16_round(a):
    """Nearest value with 8 significant bits (BF16's 7 stored fraction bits
    and the implicit one), ties to even; BF16 shares FP32's exponent range,
    which the network's values stay well inside.  Zeros, infinities and NaN
    pass through."""
    a = np.asarray(a, dtype=np.float64)
    out = a.copy()
    fin = np.isfinite(a) & (a != 0.0)
    mant, expo = np.frexp(a[fin])              # a = mant * 2^expo, 0.5 <= |mant| < 1
    out[fin] = np.ldexp(np.round(np.ldexp(mant, 8)), expo - 8)   # np.round: half to even
    return out


def _identity(a):
    return np.asarray(a, dtype=np.float64)


def weight_mask() -> np.ndarray:
    """True at the entries of the flat vector that are weight matrices (the
    ones AdamW decays), False at the biases."""
    mask = np.zeros(n_params(), dtype=bool)
    o = 0
    for _ in range(LAYERS):
        mask[o:o + HIDDEN * IN] = True
        o += HIDDEN * IN + HIDDEN
    mask[o:o + OUT * HIDDEN] = True
    return mask


def forward(p, x, rounded=False, rnd=None):
    """Outputs y [m][18] and the cache of (h_in, z) per hidden layer plus the
    last activation.  With rounded=True the BF16 reading of the module
    docstring: rnd (default bf16_round) is applied to the weight matrices, the
    input and every hidden activation."""
    r = (rnd or bf16_round) if rounded else _identity
    layers, (Wo, bo) = unflatten(p)
    h = r(x)
    cache = []
    for W, b in layers:
        z = h @ r(W).T + b
        cache.append((h, z))
        h = r(gelu(z))
    y = h @ r(Wo).T + bo
    return y, (cache, h)


def loss_and_grad(p, x, t, rounded=False, rnd=None, magnitudes=False):
    """Mean squared error over rows and outputs and its gradient (flat).
    rounded=True: the BF16 reading (the back-propagated pre-activation errors
    dz are rounded too, and every weight gradient and bias gradient is formed
    from the rounded dz).  magnitudes=True also returns, in the same layout,
    each gradient entry's sum of absolute values of its terms (for weights
    sum_m |dz_mn| |h_mk|, for biases sum_m |dz_mn|), the scale that rounding
    and summation errors are relative to."""
    r = (rnd or bf16_round) if rounded else _identity
    layers, (Wo, bo) = unflatten(p)
    t = np.asarray(t, dtype=np.float64)
    y, (cache, hlast) = forward(p, x, rounded, rnd)
    m = y.shape[0]
    d = y - t
    loss = float(np.sum(d * d) / (m * OUT))
    dy = 2.0 * d / (m * OUT)
    grads, mags = [], []
    dWo = dy.T @ hlast
    dbo = dy.sum(axis=0)
    if magnitudes:
        mags.append((np.abs(dy).T @ np.abs(hlast), np.abs(dy).sum(axis=0)))
    dh = dy @ r(Wo)
    for (W, b), (h, z) in zip(reversed(layers), reversed(cache)):
        dz = r(dh * gelu_grad(z))
        grads.append((dz.T @ h, dz.sum(axis=0)))
        if magnitudes:
            mags.append((np.abs(dz).T @ np.abs(h), np.abs(dz).sum(axis=0)))
        dh = dz @ r(W)

    def flatten(head, per_layer):
        flat = []
        for dW, db in reversed(per_layer):
            flat.append(dW.ravel())
            flat.append(db)
        flat.append(head[0].ravel())
        flat.append(head[1])
        return np.concatenate(flat)

    g = flatten((dWo, dbo), grads)
    if magnitudes:
        return loss, g, flatten(mags[0], mags[1:])
    return loss, g


def adamw_step(w, g, m1, m2, t, lr, wd, b1=0.9, b2=0.999, eps=1e-8, mask=None):
    """One AdamW step t >= 1 on flat vectors (returns new w, m1, m2): moments
    first, then the decoupled decay of the weight matrices (mask, default
    weight_mask()), then the bias-corrected Adam step."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    mask = weight_mask() if mask is None else mask
    m1 = b1 * np.asarray(m1, dtype=np.float64) + (1.0 - b1) * g
    m2 = b2 * np.asarray(m2, dtype=np.float64) + (1.0 - b2) * g * g
    w = np.where(mask, w - lr * wd * w, w)
    mhat = m1 / (1.0 - b1 ** t)
    vhat = m2 / (1.0 - b2 ** t)
    w = w - lr * mhat / (np.sqrt(vhat) + eps)
    return w, m1, m2


def loss_only(p, x, t, rounded=False):
    y, _ = forward(p, x, rounded)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.sum(d * d) / d.size)
