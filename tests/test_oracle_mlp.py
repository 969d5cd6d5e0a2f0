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


# ------------------------------------------------------------ BF16 reading
def test_bf16_rounding_hand_worked_ties_and_specials():
    # BF16 keeps 8 significant bits: the spacing just above 1 is 2^-7
    cases = {1.0 + 2.0 ** -8: 1.0,                 # tie: to the even neighbour 1
             1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,  # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
             1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,   # just above the tie
             -(1.0 + 3 * 2.0 ** -8): -(1.0 + 2.0 ** -6),
             255.0: 255.0, 257.0: 256.0, 259.0: 260.0,        # 9-bit integers: ties to even
             0.0: 0.0}
    for x, want in cases.items():
        assert M.bf16_round(np.array([x]))[0] == want, (x, want)
    sp = M.bf16_round(np.array([np.inf, -np.inf, np.nan]))
    assert sp[0] == np.inf and sp[1] == -np.inf and np.isnan(sp[2])


def test_bf16_rounding_matches_the_library_conversion():
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-3, 5000), rng.normal(0, 300, 5000)])
    x = x.astype(np.float32)     # the library converts FP32 values
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16_round(x.astype(np.float64)), ref)


def _small_problem(seed=0, m=4):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-1, 1, M.n_params()) / math.sqrt(512.0)
    x = rng.normal(size=(m, 512))
    t = rng.normal(size=(m, 18)) * 0.3
    return p, x, t


def test_rounded_reading_differs_from_the_exact_pass_only_by_its_rounding():
    p, x, t = _small_problem(1)
    loss, g = M.loss_and_grad(p, x, t)
    loss_i, g_i = M.loss_and_grad(p, x, t, rounded=True, rnd=lambda a: np.asarray(a, np.float64))
    assert loss_i == loss
    np.testing.assert_array_equal(g_i, g)
    # with BF16 rounding every value that enters a product is representable
    _, (cache, hlast) = M.forward(p, x, rounded=True)
    for h, _z in cache:
        np.testing.assert_array_equal(M.bf16_round(h), h)
    np.testing.assert_array_equal(M.bf16_round(hlast), hlast)
    # and the result moves by what rounding at a handful of layer boundaries
    # allows: a few BF16 half-ulps (2^-8) of each parameter block's scale (the
    # relative errors of the five boundaries on a path add up, with random signs)
    loss_r, g_r = M.loss_and_grad(p, x, t, rounded=True)
    assert abs(loss_r - loss) <= 4 * 2.0 ** -8 * loss
    for a, b in _blocks():
        scale = np.abs(g[a:b]).max()
        assert np.abs(g_r[a:b] - g[a:b]).max() <= 4 * 2.0 ** -8 * scale, (a, b)
    assert np.any(g_r != g)


def _blocks():
    out, o = [], 0
    for _ in range(4):
        out += [(o, o + 512 * 512), (o + 512 * 512, o + 512 * 512 + 512)]
        o += 512 * 512 + 512
    return out + [(o, o + 18 * 512), (o + 18 * 512, o + 18 * 512 + 18)]


def test_gradient_magnitudes_bound_the_gradient():
    p, x, t = _small_problem(2)
    _, g, mag = M.loss_and_grad(p, x, t, magnitudes=True)
    assert np.all(mag >= np.abs(g) * (1 - 1e-12))
    # an entry with a single term (one row) has |g| equal to its magnitude
    _, g1, mag1 = M.loss_and_grad(p, x[:1], t[:1], magnitudes=True)
    np.testing.assert_allclose(np.abs(g1), mag1, rtol=1e-12, atol=0)


# ------------------------------------------------------------ AdamW
def test_adamw_first_step_from_zero_moments():
    # from zero moments the bias corrections cancel: m_hat = g, v_hat = g^2, so
    # each entry moves by -lr g / (|g| + eps), after the weights decay by lr wd
    rng = np.random.default_rng(4)
    n = M.n_params()
    w0 = rng.normal(0, 0.05, n)
    g = rng.normal(0, 1e-2, n)
    lr, wd = 1e-3, 0.1
    w1, m1, m2 = M.adamw_step(w0, g, np.zeros(n), np.zeros(n), 1, lr, wd)
    mask = M.weight_mask()
    want = np.where(mask, w0 * (1 - lr * wd), w0) - lr * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(w1, want, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(m2, 0.001 * g * g, rtol=1e-12)


def test_adamw_weight_mask_follows_the_flat_layout():
    mask = M.weight_mask()
    assert mask.sum() == 4 * 512 * 512 + 18 * 512
    o = 0
    for _ in range(4):
        assert mask[o] and mask[o + 512 * 512 - 1] and not mask[o + 512 * 512] and not mask[o + 512 * 512 + 511]
        o += 512 * 512 + 512
    assert mask[o] and mask[o + 18 * 512 - 1] and not mask[o + 18 * 512] and not mask[-1]


def test_adamw_constant_gradient_and_pure_decay_closed_forms():
    rng = np.random.default_rng(5)
    n = 64
    mask = np.arange(n) % 3 != 0
    w0 = rng.normal(0, 1, n)
    g = rng.normal(0, 1e-3, n)
    lr, wd, T = 2e-3, 0.05, 7
    # constant gradient, no decay: the corrected moments are g and g^2 exactly,
    # so every step moves by lr g / (|g| + eps)
    w, m1, m2 = w0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, T + 1):
        w, m1, m2 = M.adamw_step(w, g, m1, m2, t, lr, 0.0, mask=mask)
    np.testing.assert_allclose(w, w0 - T * lr * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=1e-15)
    # zero gradient: weights shrink by (1 - lr wd)^T, biases do not move
    w, m1, m2 = w0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, T + 1):
        w, m1, m2 = M.adamw_step(w, np.zeros(n), m1, m2, t, lr, wd, mask=mask)
    np.testing.assert_allclose(w, np.where(mask, w0 * (1 - lr * wd) ** T, w0), rtol=1e-14)


def test_adamw_matches_torch_adamw_in_fp64():
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(6)
    n = 200
    mask = rng.random(n) < 0.7
    w0 = rng.normal(0, 0.3, n)
    lr, wd = 3e-3, 0.02
    pw = torch.tensor(w0[mask], dtype=torch.float64, requires_grad=True)
    pb = torch.tensor(w0[~mask], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([{"params": [pw], "weight_decay": wd}, {"params": [pb], "weight_decay": 0.0}],
                            lr=lr, betas=(0.9, 0.999), eps=1e-8)
    w, m1, m2 = w0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.normal(0, 10.0 ** rng.uniform(-4, 0), n)
        pw.grad = torch.tensor(g[mask], dtype=torch.float64)
        pb.grad = torch.tensor(g[~mask], dtype=torch.float64)
        opt.step()
        w, m1, m2 = M.adamw_step(w, g, m1, m2, t, lr, wd, mask=mask)
    np.testing.assert_allclose(w[mask], pw.detach().numpy(), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(w[~mask], pb.detach().numpy(), rtol=1e-13, atol=1e-16)
