"""Pins of the oracle's parallel Nelder-Mead estimator (Algorithm 1, after
Lagarias et al. 1998) and of the multi-start OPC fit (no GPU).

Branch cases are small simplices whose outcome was worked out by hand from the
Nelder-Mead definitions; the textbook problems (quadratic, Rosenbrock) fix the
minimiser; brute-force grid search, planted recovery and the noise floor pin the
fit as a whole.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

REFLECT, EXPAND, CONTRACT_OUT, CONTRACT_IN, SHRINK = 1, 2, 3, 4, 5
QUAD, ROSEN, WELL = 0, 1, 2


def _check(case_fn, verts, branch, want_verts, want_f):
    b, v, f = O.nm_one_step(case_fn, np.array(verts, dtype=float))
    assert b == branch
    np.testing.assert_allclose(v, np.array(want_verts), atol=1e-12)
    np.testing.assert_allclose(f, np.array(want_f), atol=1e-12)


def test_branch_reflect_with_tie_goes_after():
    # f = (x-1)^2 + 2 (y-1)^2.  Sorted: (1,.5) f=.5, (0,1) f=1, (0,0) f=3.
    # centroid (.5,.75), xr = (1,1.5) f=.5 = f1 < fn -> reflect; the new point
    # ties with the best and is placed after it.
    _check(QUAD, [[0, 0], [1, 0.5], [0, 1]], REFLECT,
           [[1, 0.5], [1, 1.5], [0, 1]], [0.5, 0.5, 1.0])


def test_branch_expand():
    # Sorted: (.5,0) f=2.25, (0,0) f=3, (0,-.5) f=5.5; centroid (.25,0);
    # xr = (.5,.5) f=.75 < f1; xe = (.75,1) f=.0625 < fr -> expand.
    _check(QUAD, [[0, 0], [0.5, 0], [0, -0.5]], EXPAND,
           [[0.75, 1.0], [0.5, 0], [0, 0]], [0.0625, 2.25, 3.0])


def test_branch_contract_outside():
    # Sorted: (1,1.1) f=.02, (1.5,1.1) f=.27, (1.25,2) f=2.0625; centroid
    # (1.25,1.1); xr = (1.25,.2) f=1.3425 in [fn, fw); xco = (1.25,.65)
    # f=.3075 <= fr -> outside contraction.
    _check(QUAD, [[1.25, 2.0], [1.0, 1.1], [1.5, 1.1]], CONTRACT_OUT,
           [[1.0, 1.1], [1.5, 1.1], [1.25, 0.65]], [0.02, 0.27, 0.3075])


def test_branch_contract_inside():
    # Sorted: (1,1) f=0, (2,1) f=1, (1.5,3) f=8.25; centroid (1.5,1);
    # xr = (1.5,-1) f=8.25 >= fw; xci = (1.5,2) f=2.25 < fw -> inside.
    _check(QUAD, [[1.5, 3.0], [2.0, 1.0], [1.0, 1.0]], CONTRACT_IN,
           [[1.0, 1.0], [2.0, 1.0], [1.5, 2.0]], [0.0, 1.0, 2.25])


def test_branch_shrink():
    # 1-D double well f = (x^2-1)^2.  Sorted: .9 f=.0361, -.5 f=.5625;
    # xr = 2.3 f=18.4041 >= fw; xci = .2 f=.9216 >= fw -> shrink toward .9:
    # the other vertex becomes .9 + (-.5-.9)/2 = .2.
    _check(WELL, [[-0.5], [0.9]], SHRINK, [[0.9], [0.2]], [0.0361, 0.9216])


def test_quadratic_exact_minimiser():
    n = 4
    x0 = np.zeros(n)
    verts = np.vstack([x0] + [x0 + 0.5 * np.eye(n)[i] for i in range(n)])
    v, f, it, br = O.nm_testfn(QUAD, verts, 2000, 1e-10, 1e-20)
    np.testing.assert_allclose(v[0], np.ones(n), atol=1e-7)
    assert f[0] < 1e-13
    assert set(br.tolist()) >= {REFLECT, CONTRACT_IN}


def test_rosenbrock_from_standard_start():
    """Rosenbrock from (-1.2, 1) with the usual 5% initial simplex reaches (1, 1)."""
    x0 = np.array([-1.2, 1.0])
    verts = np.vstack([x0, x0 * [1.05, 1.0], x0 * [1.0, 1.05]])
    v, f, it, br = O.nm_testfn(ROSEN, verts, 1000, 1e-8, 1e-12)
    np.testing.assert_allclose(v[0], [1.0, 1.0], atol=1e-5)
    assert it < 400
    assert EXPAND in br.tolist()


def test_start_centres_are_philox_uniform_in_box():
    n, lo, hi = 18, 0.5, 2.0
    assert np.all(O.start_centre(n, 0, 7, 123, lo, hi) == 0.0)
    c = O.start_centre(n, 5, 7, 123, lo, hi)
    lnlo, lnhi = np.log(lo), np.log(hi)
    words = np.concatenate([O.philox4x32_10([7, 5, b, 0], [123, 0]) for b in range(5)])[:n]
    want = lnlo + (lnhi - lnlo) * (words >> 8).astype(np.float64) / 2.0**24
    np.testing.assert_array_equal(c, want)
    many = np.array([O.start_centre(n, s, 0, 0, lo, hi) for s in range(1, 400)])
    assert many.min() >= lnlo and many.max() < lnhi
    assert abs(many.mean() - 0.0) < 0.02


def _planted(noise=True, A=10.0):
    w = W.single10()
    pn = O.nominal_opc(A, 2.2 * A + 21, calibrated=False)
    ph = pn * w.mult[0]
    clean = O.simulate_rk4(ph, 150, 1000.0, 10, 0.0, A)
    return pn, ph, clean, (clean + w.noise[0]) if noise else clean


def test_grid_search_brute_force_agrees_with_nm():
    """T7: two free OPCs (passive viscosity, agonist pulse) on a noisy trace;
    the NM fit is at least as good as the best point of a 41 x 41 grid and lands
    next to it."""
    pn, ph, clean, y = _planted()
    free = (6, 15)
    mask = sum(1 << j for j in free)
    pc = ph.copy()
    pc[list(free)] = pn[list(free)]
    g = np.linspace(np.log(0.5), np.log(2.0), 41)
    U = np.array([(a, b) for a in g for b in g])
    f = O.score(pc, 150, 1000.0, 10, 0.0, 10.0, y, U, free_mask=mask)
    k = int(np.argmin(f))
    r = O.fit(pc, 150, 1000.0, 10, 0.0, 10.0, y, 6, 300, free_mask=mask, tolx=1e-10,
              tolf=1e-16)
    assert r["f"] <= f[k] + 1e-12
    assert np.max(np.abs(r["u"] - U[k])) <= (g[1] - g[0])


def test_planted_recovery_reduced():
    """T8: noiseless trace, four free OPCs, the rest at the hidden values: the
    fit recovers the trace and the hidden parameters."""
    pn, ph, clean, y = _planted(noise=False)
    free = (6, 9, 15, 17)
    mask = sum(1 << j for j in free)
    pc = ph.copy()
    pc[list(free)] = pn[list(free)]
    r = O.fit(pc, 150, 1000.0, 10, 0.0, 10.0, y, 8, 400, free_mask=mask, tolx=1e-10, tolf=1e-16)
    assert r["rms"] < 1e-9
    np.testing.assert_allclose(r["p"], ph, rtol=1e-6)


@pytest.mark.slow
def test_planted_recovery_full_18():
    """T8 in full: all 18 OPCs free from the Table 1 start; the noiseless trace is
    recovered to 1e-3 deg RMS (parameters need not be, identifiability is
    limited)."""
    pn, ph, clean, y = _planted(noise=False)
    r = O.fit(pn, 150, 1000.0, 10, 0.0, 10.0, y, 1, 2500, tolx=1e-12, tolf=1e-18, nthreads=1)
    assert r["rms"] < 1e-3


def test_noise_floor():
    """T9: with sigma = 0.05 deg noise the fit cannot do meaningfully better
    than the noise: a k-parameter least-squares fit leaves ~ sigma sqrt(1-k/L)."""
    pn, ph, clean, y = _planted()
    free = (6, 9, 15, 17)
    mask = sum(1 << j for j in free)
    pc = ph.copy()
    pc[list(free)] = pn[list(free)]
    r = O.fit(pc, 150, 1000.0, 10, 0.0, 10.0, y, 8, 400, free_mask=mask, tolx=1e-10, tolf=1e-16)
    noise_rms = np.sqrt(np.mean((y - clean) ** 2))
    expect = noise_rms * np.sqrt(1 - 4 / 150)
    assert abs(r["rms"] - expect) < 0.05 * expect
    assert r["rms"] <= noise_rms


def test_single10_fit_reaches_target_and_reports_consistently():
    """The single-saccade workload (4,096 candidates x 20 iterations, seed 0)
    reaches <= 0.1 deg RMS; the reported best value equals a re-computation of
    the winner's error (the OptErr / CPU_check pattern of Fig. 4)."""
    w = W.single10()
    pn = O.nominal_opc(10.0, float(w.dur_ms[0]), calibrated=False)
    y = O.simulate_rk4(pn * w.mult[0], 150, 1000.0, 10, 0.0, 10.0) + w.noise[0]
    r = O.fit(pn, 150, 1000.0, 10, 0.0, 10.0, y, w.simplices, w.iterations, seed=w.seed)
    assert w.simplices == 186
    assert r["rms"] < 0.1
    assert r["rms"] ** 2 == pytest.approx(r["f"], rel=1e-12)
    assert np.all(r["iters"] <= 20)
