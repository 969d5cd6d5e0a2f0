"""Pins of the FP64 oracle's plant model and integrator against what the paper
and the mathematics fix (no GPU).

Each test pins the oracle to something other than itself: values the paper
prints (Table 1, Fig. 4), published known-answer vectors (Philox), closed forms
derived by hand from the plant reading (fixation equilibrium, steady state,
first-order activation, the stiff-tendon limit that reduces to a textbook
mass-spring-damper), an independent exact solver and scipy's expm.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _box_opc(rng, base, lo=0.8, hi=1.2):
    return base * rng.uniform(lo, hi, base.shape[0])


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_table1_defaults_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_defaults.txt"))
            if l.strip() and not l.startswith("#")]
    p = O.nominal_table1(43.0)
    assert [r[0] for r in rows] == O.NAMES
    for j, r in enumerate(rows[:-1]):
        assert p[j] == float(r[2]), r
    assert p[17] == 43.0 - 6.0          # W = saccade duration - 6 ms


def test_fig4_bounds_are_table1_times_ten_or_tenth():
    """Fig. 4 row 1 prints several values that are exactly 10x or 0.1x of
    Table 1 (the reading of a multiplicative search box)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "fig4_example_rows.txt"))
            if l.strip() and not l.startswith("#")]
    r1 = [float(x) for x in rows[0][3:]]
    p = O.nominal_table1(43.0)
    assert r1[0] == pytest.approx(10 * p[0], abs=1e-6)    # SE_ag 25 = 10 x 2.5
    assert r1[3] == pytest.approx(0.1 * p[3], abs=1e-6)   # LT_ant 0.12 = 1.2 / 10
    assert r1[4] == pytest.approx(10 * p[4], abs=1e-6)    # PE_ag 8 = 10 x 0.8
    assert r1[9] == pytest.approx(p[9], abs=1e-7)         # Inert stays at default


def test_fixation_is_equilibrium():
    """T1: with the pulse at the step level and the same start and end
    fixation, the eye never moves; the derivative at the rest state is zero."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = _box_opc(rng, O.nominal_table1(40.0), 0.5, 2.0)
        th0 = rng.uniform(-20, 20)
        ag, ant = O.step_levels(p, th0)
        p[15], p[16] = ag, ant
        th = O.simulate_rk4(p, 200, 1000.0, 10, th0, th0)
        assert np.max(np.abs(th - th0)) < 1e-9
        s = O.rest_state(p, th0)
        ds = O.deriv(p, s, ag, ant, 2e-3, 2e-3)
        assert np.max(np.abs(ds)) < 1e-9


def _ss_closed_form(p, fa, fn):
    """Steady state of the plant under constant active-state tensions, derived
    by hand: at rest x = th + Ta/KSE, Fa = Ta + KLT x, hence
    Ta = a_g (Fa - KLT_AG th) with a_g = KSE/(KSE+KLT); likewise
    Tn = a_n (Fn + KLT_ANT th); the globe balance Ta - Tn = KP th gives th."""
    kse_ag, kse_ant, klt_ag, klt_ant = p[0], p[1], p[2], p[3]
    kp = p[4] + p[5]
    ag = kse_ag / (kse_ag + klt_ag)
    an = kse_ant / (kse_ant + klt_ant)
    return (ag * fa - an * fn) / (kp + ag * klt_ag + an * klt_ant)


def test_steady_state_closed_form():
    """eq. SS: long integration under arbitrary constant drives settles at the
    hand-derived closed form."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        p = _box_opc(rng, O.nominal_table1(40.0), 0.5, 2.0)
        s = O.rest_state(p, rng.uniform(-10, 10))
        na, nn = rng.uniform(0, 120), rng.uniform(-20, 40)
        s = O.integrate_const(p, s, na, nn, 3e-3, 3e-3, 1e-4, 40000)
        assert s[0] == pytest.approx(_ss_closed_form(p, na, nn), abs=1e-8)
        assert abs(s[1]) < 1e-7


def test_saccade_settles_at_target():
    """T2: after the pulse the plant comes to rest at the end fixation."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        A = rng.uniform(1, 40)
        p = _box_opc(rng, O.nominal_opc(A, 2.2 * A + 21))
        th = O.simulate_rk4(p, 3000, 1000.0, 10, 0.0, A)
        assert th[-1] == pytest.approx(A, abs=1e-8)


def test_activation_is_first_order_lag_with_phase_constants():
    """The active-state tension follows N + (F0 - N) exp(-t/tau) with the
    activation constant during the pulse and the deactivation constant after
    (reading of Sec. 2.1's activation/deactivation times), switching at
    onset + W."""
    p = O.nominal_opc(10.0, 43.0, calibrated=False)
    fs, onset = 1000.0, 10
    _, st = O.simulate_rk4(p, 150, fs, onset, 0.0, 10.0, return_state=True)
    f0 = O.step_levels(p, 0.0)[0]
    t_on, t_sw = onset / fs, onset / fs + p[17] * 1e-3
    tac, tde = p[10] * 1e-3, p[12] * 1e-3
    f_sw = p[15] + (f0 - p[15]) * math.exp(-(t_sw - t_on) / tac)
    fend = O.step_levels(p, 10.0)[0]
    for k in range(150):
        t = k / fs
        if t <= t_on:
            want = f0
        elif t <= t_sw:
            want = p[15] + (f0 - p[15]) * math.exp(-(t - t_on) / tac)
        else:
            want = fend + (f_sw - fend) * math.exp(-(t - t_sw) / tde)
        assert st[k, 4] == pytest.approx(want, rel=1e-8, abs=1e-8), k


def test_stiff_tendon_limit_is_textbook_second_order_system():
    """With very stiff series elasticity the tendon states follow the globe
    (x = th, y = -th) and the plant reduces to
    J th'' + (BP + B_AG + B_ANT) th' + (KP + KLT_AG + KLT_ANT) th = Fa - Fn,
    whose step response from rest is the textbook overdamped/underdamped form."""
    p = O.nominal_table1(40.0)
    p[0] = p[1] = 2.0e4
    fa, fn = 30.0, 10.0
    s = np.array([0.0, 0.0, 0.0, 0.0, fa, fn])
    J, B = p[9], p[6] + p[7] + p[8]
    K = p[4] + p[5] + p[2] + p[3]
    disc = B * B - 4 * J * K
    r1 = (-B + math.sqrt(disc)) / (2 * J)
    r2 = (-B - math.sqrt(disc)) / (2 * J)
    h = 2.0e-7
    t = 0.0
    for T in (0.005, 0.02, 0.05, 0.1):
        n = int(round((T - t) / h))
        s = O.integrate_const(p, s, fa, fn, 1.0, 1.0, h, n)
        t += n * h
        want = (fa - fn) / K * (1 + (r2 * math.exp(r1 * t) - r1 * math.exp(r2 * t)) / (r1 - r2))
        assert s[0] == pytest.approx(want, rel=2e-3), T


def test_expm_matches_scipy():
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(4)
    for scale in (1e-3, 0.3, 5.0, 80.0):
        m = rng.normal(size=(7, 7)) * scale
        ref = sl.expm(m)
        assert np.allclose(O.expm7(m), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("fs", [1000.0, 500.0, 250.0, 600.0])
def test_rk4_matches_exact_solution(fs):
    """T3: fixed-step RK4 (h ~ 0.1 ms) agrees with the exact piecewise solution
    of the linear plant."""
    rng = np.random.default_rng(5)
    for i in range(6):
        A = rng.uniform(1, 40)
        p = _box_opc(rng, O.nominal_opc(A, 2.2 * A + 21))
        L = int(0.25 * fs)
        on = int(math.ceil(0.01 * fs))
        rk = O.simulate_rk4(p, L, fs, on, 0.0, A)
        ex = O.simulate_exact(p, L, fs, on, 0.0, A)
        assert np.max(np.abs(rk - ex)) < 1e-6, (fs, i, np.max(np.abs(rk - ex)))


def test_rk4_is_fourth_order():
    """Halving the step divides the step-to-step difference by ~2^4 = 16: the
    integrator is a fourth-order method (a wrong stage weight or a dropped
    stage lowers the order)."""
    p = O.nominal_table1(43.0)
    s0 = O.rest_state(p, 0.0)
    T = 0.02
    out = []
    for h in (4e-4, 2e-4, 1e-4, 5e-5):
        out.append(O.integrate_const(p, s0, 80.0, 0.5, 11.7e-3, 1.9e-3, h, int(round(T / h))))
    d = [np.max(np.abs(out[i] - out[i + 1])) for i in range(3)]
    for a, b in zip(d, d[1:]):
        assert 13.0 < a / b < 19.0, d


def test_mirror_symmetry():
    """T4: a saccade toward negative angles is the mirror image of the positive
    one (Fig. 1 shows the plant for positive saccades)."""
    p = O.nominal_opc(12.0, 47.4)
    a = O.simulate_rk4(p, 180, 1000.0, 10, 0.0, 12.0)
    b = O.simulate_rk4(p, 180, 1000.0, 10, 0.0, -12.0)
    assert np.array_equal(a, -b)
    c = O.simulate_rk4(p, 180, 1000.0, 10, 3.0, -9.0)
    d = O.simulate_rk4(p, 180, 1000.0, 10, -3.0, 9.0)
    assert np.array_equal(c, -d)


def test_pulse_calibration_hits_amplitude_and_main_sequence():
    """The calibrated agonist pulse makes the nominal peak equal the amplitude,
    and the nominal saccades follow a main sequence: larger saccades are faster
    and last longer."""
    vmax, t90 = [], []
    for A in (5.0, 10.0, 20.0, 30.0, 40.0):
        D = 2.2 * A + 21
        n = O.calibrate_pulse(A, D)
        p = O.nominal_table1(D)
        p[15] = n
        th = O.simulate_rk4(p, 251, 1000.0, 0, 0.0, A)
        assert th.max() == pytest.approx(A, abs=1e-9)
        vmax.append(np.max(np.diff(th)) * 1000.0)
        t90.append(int(np.argmax(th >= 0.9 * A)))
    assert all(np.diff(vmax) > 0)
    assert all(np.diff(t90) > 0)
    assert 100.0 < vmax[1] < 1000.0      # deg/s for 10 deg
    # the agonist pulse grows with amplitude, Table 1's 55 g sits near 5-10 deg
    assert O.calibrate_pulse(5.0, 32.0) < 55.0 < O.calibrate_pulse(10.0, 43.0)


def test_table1_ten_degree_saccade_is_slow_but_arrives():
    """With Table 1's literal 55 g pulse a 10 deg saccade is under-driven: it
    approaches 10 deg within 150 ms without overshooting."""
    p = O.nominal_opc(10.0, 43.0, calibrated=False)
    th = O.simulate_rk4(p, 150, 1000.0, 10, 0.0, 10.0)
    assert np.all(np.diff(th) >= -1e-12)
    assert 9.0 < th[-1] < 10.0


def test_stiff_candidates_get_refined_substeps():
    """Candidates whose fastest mode is too fast for RK4 at ~0.1 ms get the
    step halved until h times the mode estimate is at most 2.5 (at most six
    times); the refined trajectory still matches the exact piecewise
    solution; beyond the finest step a candidate scores +inf."""
    p = O.nominal_table1(43.0)
    assert O.substeps(p, 1000.0) == 10 and not O.stiff(p, 1000.0)
    corner = p.copy()
    corner[6] *= 2.0
    corner[9] *= 0.5
    assert O.substeps(corner, 1000.0) == 10       # the [0.5x, 2x] box needs no refinement
    corner[6] = p[6] * 10.0
    corner[9] = p[9] * 0.1
    assert O.substeps(corner, 1000.0) == 80 and not O.stiff(corner, 1000.0)   # [0.1x, 10x]: 8x
    assert O.substeps(corner, 250.0) == 320
    for fs in (1000.0, 250.0):
        L, on = int(0.15 * fs), int(math.ceil(0.01 * fs))
        rk = O.simulate_rk4(corner, L, fs, on, 0.0, 10.0)
        ex = O.simulate_exact(corner, L, fs, on, 0.0, 10.0)
        assert np.max(np.abs(rk - ex)) < 1e-6
    extreme = p.copy()
    extreme[6] = p[6] * 1000.0
    extreme[9] = p[9] * 0.001
    assert O.stiff(extreme, 1000.0)
    assert O.errors(extreme, 150, 1000.0, 10, 0.0, 10.0, np.zeros(150))[0] == math.inf

