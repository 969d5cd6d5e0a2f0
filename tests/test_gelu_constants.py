"""The surrogate's GELU takes erf from Abramowitz and Stegun, Handbook of
Mathematical Functions, formula 7.1.26 (absolute error at most 1.5e-7 for
x >= 0).  The constants are read from the kernel source, so a mistyped one
fails here: the published bound must hold on a dense grid, and the formula
must reduce to erf(0) = 0 and erf(inf) = 1."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2007_09884_gb300", "csrc", "mlp.cu")


def constants():
    line = [l for l in open(SRC) if "A&S 7.1.26:" in l]
    assert len(line) == 1, "one marked line of constants"
    vals = dict(re.findall(r"\b(p|a[1-5]) (-?[0-9.]+)", line[0]))
    assert set(vals) == {"p", "a1", "a2", "a3", "a4", "a5"}
    return {k: float(v) for k, v in vals.items()}


def erf_as(x, c):
    t = 1.0 / (1.0 + c["p"] * x)
    poly = t * (c["a1"] + t * (c["a2"] + t * (c["a3"] + t * (c["a4"] + t * c["a5"]))))
    return 1.0 - poly * np.exp(-x * x)


def test_published_error_bound_holds():
    c = constants()
    x = np.linspace(0.0, 6.0, 600001)
    ref = np.array([math.erf(v) for v in x[::10]])
    err = np.abs(erf_as(x[::10], c) - ref)
    assert err.max() <= 1.5e-7, err.max()


def test_limits():
    c = constants()
    # erf(0) = 0: the coefficients sum to 1
    assert abs(c["a1"] + c["a2"] + c["a3"] + c["a4"] + c["a5"] - 1.0) <= 1e-8
    assert abs(erf_as(np.array([40.0]), c)[0] - 1.0) == 0.0


def test_cdf_form_matches_normal_cdf():
    # Phi(z) = 1 - q (z >= 0), q (z < 0), q = poly(t) e^(-z^2/2) / 2, t = 1 / (1 + p |z| / sqrt 2)
    c = constants()
    z = np.linspace(-8.0, 8.0, 16001)
    x = np.abs(z) / math.sqrt(2.0)
    t = 1.0 / (1.0 + c["p"] * x)
    poly = t * (c["a1"] + t * (c["a2"] + t * (c["a3"] + t * (c["a4"] + t * c["a5"]))))
    q = 0.5 * poly * np.exp(-0.5 * z * z)
    phi = np.where(z >= 0.0, 1.0 - q, q)
    ref = np.array([0.5 * math.erfc(-v / math.sqrt(2.0)) for v in z])
    assert np.max(np.abs(phi - ref)) <= 0.75e-7 + 1e-15
