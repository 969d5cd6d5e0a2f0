"""The learned surrogate on the GPU: the tcgen05 GEMM against torch, and the
featurizer, the forward and backward passes and AdamW element by element
against the oracle (oracle/features.py, oracle/mlp.py); training and seeding.

Tolerances: the GEMM accumulates BF16 products in FP32 exactly like the
reference matmul up to summation order (1e-3 relative).  The network is
compared with the oracle's BF16 reading (weights, inputs, hidden activations
and back-propagated pre-activation errors rounded to BF16 where they enter a
product), so both sides round at the same places; what remains is FP32
accumulation (K 2^-24 of a sum's magnitude, K <= 512) and the rare value
whose FP32 and FP64 forms fall on either side of a BF16 rounding boundary and
round one BF16 ulp (2^-7 relative) apart.  A term of a sum has two such
factors, so each entry is allowed 2^-6 of its magnitude (the sum of the
absolute values of its terms, which the oracle returns).  AdamW runs in FP32
on FP32 parameters: a few FP32 ulps per step."""
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2007_09884_gb300 as G
import workloads as W
from _support import centres, oracle_inputs, to_batch
from oracle import features as F
from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = G.opmm_create(0)
    yield h
    G.opmm_destroy(h)


def bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("M_,N_,K_", [(128, 128, 64), (256, 512, 512), (512, 512, 4096), (384, 256, 192)])
def test_tcgen05_gemm_matches_torch(ctx, M_, N_, K_):
    torch = pytest.importorskip("torch")
    g = torch.Generator(device="cuda").manual_seed(M_ + N_ + K_)
    A = torch.randn(M_, K_, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N_, K_, device="cuda", generator=g).to(torch.bfloat16)
    D = G.opmm_gemm_bf16(ctx, A, B)
    ref = A.double() @ B.double().T
    err = (D.double() - ref).abs().max().item()
    assert err <= 1e-3 * ref.abs().max().item() + 1e-3, err


def test_featurizer_matches_oracle(ctx):
    """Every feature of 24 uneven saccades (three rates, both directions).
    The device computes in FP32 and stores BF16, so a feature is allowed half
    a BF16 ulp of its value (2^-8 relative) plus its FP32 error before that
    rounding: the sample position onset + i fs 1e-3 is off by at most ~1e-4
    samples (FP32 rounding of the product and of 1e-3), which moves an
    interpolated position by 1e-4 times the largest step of the trace, plus a
    few FP32 ulps of the trace's scale; a velocity is 10 times the difference
    of two positions, so 20 times that."""
    items = oracle_inputs(W.uneven10k(B=24))
    got = G.opmm_featurize(ctx, to_batch(items))
    for j, it in enumerate(items):
        y = np.float32(it["y"]).astype(np.float64)
        ref = F.featurize(y, it["fs"], it["onset"], it["th0"], it["thf"])
        amp = max(abs(it["thf"] - it["th0"]), 0.5)
        d_pos = (1e-4 * np.abs(np.diff(y)).max() + 8 * 2.0 ** -24 * (np.abs(y).max() + abs(it["th0"]))) / amp
        delta = np.concatenate([np.full(256, d_pos), np.full(256, 20 * d_pos)])
        tol = 2.0 ** -8 * np.abs(ref) + 1.01 * delta
        err = np.abs(got[j] - ref)
        assert np.all(err <= tol), (j, int(np.argmax(err - tol)), float((err / tol).max()))


def _blocks():
    out, o = [], 0
    for l in range(4):
        out += [(f"W{l}", o, o + 512 * 512), (f"b{l}", o + 512 * 512, o + 512 * 512 + 512)]
        o += 512 * 512 + 512
    return out + [("W_out", o, o + 18 * 512), ("b_out", o + 18 * 512, o + 18 * 512 + 18)]


def _check_network_against_oracle(ctx, p32, seed):
    """Forward outputs, loss and every gradient entry of 256 rows against the
    oracle's BF16 reading on the same FP32 parameters and inputs."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (256, 512)).astype(np.float32)
    t = rng.normal(0, 0.5, (256, 18)).astype(np.float32)
    loss_g, grad_g, y_g = G.opmm_surrogate_grad(ctx, x, t)
    p = np.asarray(p32, dtype=np.float64)
    xo, to = x.astype(np.float64), t.astype(np.float64)
    loss_o, grad_o, mag = M.loss_and_grad(p, xo, to, rounded=True, magnitudes=True)
    y_o, (_, h_last) = M.forward(p, xo, rounded=True)
    # outputs: 512-term sums of BF16 products plus the bias
    Wo = M.bf16_round(M.unflatten(p)[1][0])
    y_mag = np.abs(h_last) @ np.abs(Wo).T + np.abs(M.unflatten(p)[1][1])
    assert np.all(np.abs(y_g - y_o) <= 2.0 ** -6 * y_mag), float((np.abs(y_g - y_o) / y_mag).max())
    assert abs(loss_g - loss_o) <= 2.0 ** -6 * loss_o
    worst = {}
    for name, a, b in _blocks():
        err = np.abs(grad_g[a:b].astype(np.float64) - grad_o[a:b])
        tol = 2.0 ** -6 * mag[a:b] + 1e-30
        worst[name] = float((err / tol).max())
        assert np.all(err <= tol), (name, worst[name], int(np.argmax(err / tol)))
    return worst


def test_forward_backward_match_fp64_oracle_element_by_element(ctx):
    G.opmm_surrogate_init(ctx, 7)
    worst = _check_network_against_oracle(ctx, G.opmm_surrogate_get_params(ctx), 1)
    print("largest error / tolerance per block:", worst)


def test_adamw_matches_oracle_element_by_element(ctx):
    """Three AdamW steps on fixed gradients (entries spread over five decades,
    some exactly zero) through the library, against the oracle's FP64 AdamW
    from the same FP32 start; then the updated network's forward and backward
    passes, which run on the BF16 copies that AdamW refreshes.  Per step the
    device rounds the moments, the decay, the update and the parameter to
    FP32 (about ten roundings of 2^-24 relative on the update, which the
    moments carry into later steps, and a few on the parameter), and its
    betas are the FP32 values nearest 0.9 and 0.999, which the bias
    corrections cancel to the same order: over three steps an entry may
    differ by 3 x 4 FP32 ulps of its value plus 2e-6 of how far it moved,
    with a floor of 3 x 8 ulps of lr."""
    G.opmm_surrogate_init(ctx, 21)
    p0 = G.opmm_surrogate_get_params(ctx).astype(np.float64)
    n = p0.size
    rng = np.random.default_rng(22)
    lr, wd = 2e-3, 0.1
    w, m1, m2 = p0.copy(), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = (rng.normal(0, 1, n) * 10.0 ** rng.uniform(-6, -1, n)).astype(np.float32)
        g[rng.random(n) < 0.01] = 0.0
        G.opmm_surrogate_apply_grad(ctx, g, lr, wd)
        w, m1, m2 = M.adamw_step(w, g.astype(np.float64), m1, m2, step, lr, wd)
    got = G.opmm_surrogate_get_params(ctx).astype(np.float64)
    moved = np.abs(w - p0)
    tol = 3 * (4 * 2.0 ** -24 * np.abs(w) + 8 * 2.0 ** -24 * lr * 1.01)
    err = np.abs(got - w)
    assert np.all(err <= tol + 2e-6 * moved), float((err / (tol + 2e-6 * moved)).max())
    # the update is visible: every entry with a gradient moved by about lr
    assert np.median(moved[M.weight_mask()]) > 0.5 * lr
    _check_network_against_oracle(ctx, got.astype(np.float32), 23)


def test_training_reduces_loss_and_weights_round_trip(ctx, tmp_path):
    # targets ln(U(0.8, 1.2)) / 0.2 have variance ~0.333 per output: an untrained
    # network starts there; 600 steps of 2,048 generated saccades must cut it.
    # Over 12 (initialisation, data) seed pairs the last-50 / first-5 loss
    # ratio measured 0.910-0.938 (mean 0.922, standard deviation 0.007); the
    # bound is the mean plus four standard deviations.
    G.opmm_surrogate_init(ctx, 3)
    losses = G.opmm_surrogate_train(ctx, 600, batch=2048, lr=2e-3, data_seed=11)
    assert np.all(np.isfinite(losses))
    assert 0.30 < losses[:5].mean() < 0.37
    assert losses[-50:].mean() < 0.95 * losses[:5].mean(), (losses[:5], losses[-50:])
    path = str(tmp_path / "w.bin")
    G.opmm_surrogate_save(ctx, path)
    p1 = G.opmm_surrogate_get_params(ctx)
    G.opmm_surrogate_init(ctx, 99)
    G.opmm_surrogate_load(ctx, path)
    np.testing.assert_array_equal(G.opmm_surrogate_get_params(ctx), p1)


def test_training_is_deterministic_and_split_calls_continue_it(ctx):
    # Steps run in graph-replayed pairs plus a direct odd step, with the
    # sample bases, the step index and the AdamW corrections in device
    # memory: five steps in one call must equal three then two (sample_base
    # continued), bit for bit, in the parameters and in every step's loss.
    B = 512
    G.opmm_surrogate_init(ctx, 7)
    la = G.opmm_surrogate_train(ctx, 5, batch=B, lr=1e-3, data_seed=3)
    pa = G.opmm_surrogate_get_params(ctx)
    G.opmm_surrogate_init(ctx, 7)
    l1 = G.opmm_surrogate_train(ctx, 3, batch=B, lr=1e-3, data_seed=3)
    l2 = G.opmm_surrogate_train(ctx, 2, batch=B, lr=1e-3, data_seed=3, sample_base=3 * B)
    pb = G.opmm_surrogate_get_params(ctx)
    np.testing.assert_array_equal(np.concatenate([l1, l2]), la)
    np.testing.assert_array_equal(pb, pa)
    assert np.all(np.isfinite(la)) and np.all(np.isfinite(pa))


def test_seeded_fit_stays_in_the_narrowed_box(ctx):
    G.opmm_surrogate_init(ctx, 5)
    G.opmm_surrogate_train(ctx, 50, batch=1024, lr=1e-3, data_seed=12)
    items = oracle_inputs(W.uneven10k(B=6))
    batch = to_batch(items)
    pred = G.opmm_surrogate_predict(ctx, batch)
    nominal = G.opmm_nominal_opc(ctx, batch, G.OPMM_PULSE_CALIBRATED)
    ratio = pred / nominal
    assert np.all(np.isfinite(pred)) and np.all(pred > 0)
    assert np.all(np.abs(np.log(ratio)) < 3.0)
    res = G.opmm_fit_batch(ctx, batch, candidates=22 * 16, iterations=8, box_lo=0.95, box_hi=1.05,
                           init_step=0.025, use_surrogate=True)
    assert np.all(res["status"] == 0)
    r = res["opc"] / pred
    assert np.all(r >= 0.95 * (1 - 1e-5)) and np.all(r <= 1.05 * (1 + 1e-5))


# 10 M generated saccades: steps x rows, with a stepped learning rate
TRAIN_SCHEDULE = [(800, 2e-3), (800, 1e-3), (500, 5e-4), (341, 2.5e-4)]


def test_trained_surrogate_gains_over_plain_search(ctx):
    """What the network adds to the estimator of Sec. 3.3, on held-out
    saccades of the uneven workload (drawn by the numpy generator, never seen
    in training, which draws on the device):
    * its estimate alone traces the recording more closely than the nominal
      centre it replaces;
    * a 1,024 x 20 search in a +-5% box around it fits more saccades to
      <= 0.1 deg RMS than the plain search with the same budget;
    * with the plain search as fallback for its misses it fits at least as
      many saccades as the plain full-budget search alone: with a full-budget
      fallback at under 0.15 of the candidate simulations, with a 4,096 x 30
      fallback at under a tenth."""
    G.opmm_surrogate_init(ctx, 1)
    base = 0
    for steps, lr in TRAIN_SCHEDULE:
        G.opmm_surrogate_train(ctx, steps, batch=4096, lr=lr, weight_decay=1e-4, data_seed=7, sample_base=base)
        base += steps * 4096
    items = oracle_inputs(W.uneven10k(B=400, config_index=3))
    batch = to_batch(items)
    pred = G.opmm_surrogate_predict(ctx, batch)
    nominal = centres(items)

    def rms_of(opc):
        traj, offs = G.opmm_simulate(ctx, opc.astype(np.float32), batch)
        return np.array([math.sqrt(np.mean((traj[offs[j]:offs[j] + it["L"]] - it["y"]) ** 2))
                         for j, it in enumerate(items)])

    # held-out medians over 100,000 saccades are 0.075 deg (network) against
    # 0.17 deg (nominal).  Over 10 held-out sets of 400 (config indices 3-12)
    # and two training seeds the ratio of the medians measured 0.402-0.495
    # (mean 0.44); this set (index 3) is the highest at 0.490, and the bound
    # leaves a tenth above the largest value seen.
    assert np.median(rms_of(pred)) < 0.55 * np.median(rms_of(nominal))

    small = dict(candidates=1024, iterations=20, seed=0)
    seeded = dict(small, box_lo=0.95, box_hi=1.05, init_step=0.025)
    full = dict(candidates=16384, iterations=30, seed=0)
    r_seed = G.opmm_fit_batch(ctx, batch, use_surrogate=True, **seeded)
    r_small = G.opmm_fit_batch(ctx, batch, **small)
    r_full = G.opmm_fit_batch(ctx, batch, **full)
    r_fb, n_fb = G.opmm_fit_batch_seeded(ctx, batch, seeded, full, fallback_rms_deg=0.1)

    def fitted(r):
        return float(np.mean((r["rms_deg"] <= 0.1) & (r["status"] == 0)))

    f_seed, f_small, f_full, f_fb = fitted(r_seed), fitted(r_small), fitted(r_full), fitted(r_fb)
    print(f"fitted<=0.1deg: seeded {f_seed:.3f} plain-same-budget {f_small:.3f} plain-full {f_full:.3f} "
          f"seeded+fallback {f_fb:.3f} (fallbacks {n_fb})")
    assert np.all(r_seed["source"] == G.OPMM_SOURCE_SEEDED) and np.all(r_small["source"] == G.OPMM_SOURCE_PLAIN)
    assert f_seed >= f_small + 0.10
    # the fallback re-fits exactly the misses and keeps the better result
    miss = (r_seed["rms_deg"] > 0.1) | (r_seed["status"] != 0)
    assert n_fb == int(miss.sum())
    np.testing.assert_array_equal(r_fb["opc"][~miss], r_seed["opc"][~miss])
    assert np.all(r_fb["rms_deg"][miss] <= r_seed["rms_deg"][miss])
    assert np.all(np.isin(r_fb["source"][miss], [G.OPMM_SOURCE_SEEDED, G.OPMM_SOURCE_FALLBACK]))
    assert f_fb >= f_full

    def evals(r):
        return float(np.sum(r["evaluations"].astype(np.float64)))

    assert evals(r_fb) < 0.15 * evals(r_full), (evals(r_fb), evals(r_full))
    light = dict(candidates=4096, iterations=30, seed=0)
    r_lt, n_lt = G.opmm_fit_batch_seeded(ctx, batch, seeded, light, fallback_rms_deg=0.1)
    print(f"seeded+4096x30 fallback {fitted(r_lt):.3f}")
    assert n_lt == n_fb
    assert fitted(r_lt) >= f_full
    assert evals(r_lt) < 0.1 * evals(r_full), (evals(r_lt), evals(r_full))


def test_seeded_fit_rejects_bad_option_pairs(ctx):
    G.opmm_surrogate_init(ctx, 5)
    batch = to_batch(oracle_inputs(W.uneven10k(B=2)))
    lib = G.load_library()
    so, _ = G.fit_opts(use_surrogate=False)
    po, _ = G.fit_opts(use_surrogate=False)
    descs, keep = batch.descriptors()
    res = (G.opmm_fit_result * 2)()
    import ctypes
    nfb = ctypes.c_int32(0)
    rc = lib.opmm_fit_batch_seeded(ctx, descs, 2, ctypes.byref(so), ctypes.byref(po), ctypes.c_float(0.1), res,
                                   ctypes.byref(nfb))
    assert rc == G.OPMM_EINVAL
    so.use_surrogate = 1
    rc = lib.opmm_fit_batch_seeded(ctx, descs, 2, ctypes.byref(so), ctypes.byref(po), ctypes.c_float(-1.0), res,
                                   ctypes.byref(nfb))
    assert rc == G.OPMM_EINVAL
