"""Oracle pins of the gradient-based refinement (Levenberg-Marquardt with a
central-difference Jacobian), the alternative estimator Sec. 5 proposes to
test after Nelder-Mead.

Pinned by textbook cases: on a linear least-squares problem one undamped
Gauss-Newton step lands on the normal-equation solution (numpy's lstsq as the
independent reference); Rosenbrock's residuals converge to (1, 1); on a
noiseless planted OPMM trace the refinement from a perturbed start recovers
the trace; and a refinement never ends worse than its start.
"""
import numpy as np

import oracle as O
import workloads as W


def test_linear_least_squares_is_solved_by_one_step():
    A = np.array([[1, 2, 0], [0, 1, 1], [1, 0, 3], [2, 1, 1], [0, 0, 1], [1, 1, 1]], float)
    b = np.arange(1, 7, dtype=float)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    u, f, acc = O.lm_testfn(0, [0.0, 0.0, 0.0], 1, lambda0=1e-12)
    assert acc == 1
    np.testing.assert_allclose(u, x, rtol=1e-8, atol=1e-9)
    assert abs(f - np.sum((A @ x - b) ** 2) / 6) < 1e-10


def test_box_projection_and_monotone_descent():
    # the unconstrained optimum has u2 ~ 1.49; a box of [-1, 1] keeps every
    # iterate inside and the value never rises above the start's
    u, f, acc = O.lm_testfn(0, [0.0, 0.0, 0.0], 30, lo=-1.0, hi=1.0)
    assert np.all(u >= -1.0) and np.all(u <= 1.0)
    assert f <= np.sum(np.arange(1, 7) ** 2) / 6


def test_rosenbrock_converges():
    u, f, acc = O.lm_testfn(1, [-1.2, 1.0], 200)
    np.testing.assert_allclose(u, [1.0, 1.0], atol=1e-6)
    assert f < 1e-12


def test_planted_trace_recovered_from_a_perturbed_start():
    """Noiseless trace of a hidden OPC vector; the 18-coordinate refinement
    starts 8% (in ln units) off on four coordinates and recovers the trace."""
    w = W.single10()
    A = 10.0
    pn = O.nominal_opc(A, 2.2 * A + 21, calibrated=False)
    ph = pn * w.mult[0]
    y = O.simulate_rk4(ph, 150, 1000.0, 10, 0.0, A)
    uh = np.log(ph / pn)
    u0 = uh.copy()
    u0[[6, 9, 15, 17]] += 0.08
    start = O.errors(O.u_to_p(pn, u0), 150, 1000.0, 10, 0.0, A, y)[0]
    r = O.refine(pn, 150, 1000.0, 10, 0.0, A, y, u0, 30)
    assert r["rms"] < 1e-4 < np.sqrt(start)
    assert r["accepted"] >= 3


def test_refinement_after_the_search_never_ends_worse():
    w = W.uneven10k(B=3)
    for i in range(3):
        A, D = float(w.amplitude[i]), float(w.dur_ms[i])
        pn = O.nominal_opc(A, D)
        L, fs, on = int(w.L[i]), float(w.fs[i]), int(w.onset[i])
        th0, thf = float(w.theta0[i]), float(w.thetaf[i])
        y = O.simulate_rk4(pn * w.mult[i], L, fs, on, th0, thf) + w.noise[i]
        s = O.fit(pn, L, fs, on, th0, thf, y, 8, 10, sac_index=i)
        r = O.refine(pn, L, fs, on, th0, thf, y, s["u"], 8)
        assert r["f"] <= s["f"]
        assert r["rms"] <= s["rms"] + 1e-12
        # the model reaches the noise: sigma = 0.05 deg
        assert r["rms"] < 0.06
