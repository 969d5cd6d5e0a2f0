"""Pins of the FP64 surrogate-network oracle (no GPU): GELU special values and
identities, and the analytic gradient against central finite differences."""
import math

import numpy as np

from oracle import mlp as M


def test_gelu_identities():
    z = np.array([-6.0, -1.0, -0.3, 0.0, 0.3, 1.0, 6.0])
    g = M.gelu(z)
    assert g[3] == 0.0
    np.testing.assert_allclose(g - M.gelu(-z), z, atol=1e-15)          # z Phi(z) - (-z) Phi(-z) = z
    assert abs(g[-1] - 6.0) < 1e-8 and abs(g[0]) < 1e-8
    assert M.gelu(np.array([1.0]))[0] == 0.5 * (1.0 + math.erf(1.0 / math.sqrt(2.0)))
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, M.n_params()) / math.sqrt(512.0)
    x = rng.normal(size=(3, 512))
    t = rng.normal(size=(3, 18)) * 0.3
    loss, g = M.loss_and_grad(p, x, t)
    assert loss == M.loss_only(p, x, t)
    idx = np.concatenate([rng.integers(0, M.n_params(), 30),
                          [0, 512 * 512, 512 * 512 + 511, M.n_params() - 1, M.n_params() - 19]])
    h = 1e-5
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (M.loss_only(p + e, x, t) - M.loss_only(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])
