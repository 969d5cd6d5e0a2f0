"""Pins of the surrogate's feature definition (oracle/features.py, no GPU):
traces whose resampled features are known in closed form."""
import numpy as np

from oracle import features as F


def _ramp_features(c, fs, onset, L, amp, n=256):
    """Closed form for y_k = c k from a start fixation 0: linear interpolation
    of a linear trace is exact, so position i = c s_i / amp with
    s_i = min(onset + i fs / 1000, L - 1), and velocity i is 10 times the
    difference of consecutive positions (0 for the last)."""
    s = np.minimum(onset + np.arange(n + 1) * fs / 1000.0, L - 1)
    pos = c * s / amp
    vel = 10.0 * np.diff(pos)
    vel[-1] = 0.0
    return np.concatenate([pos[:n], vel])


def test_ramp_at_each_rate():
    for fs, onset in ((1000.0, 10), (500.0, 5), (250.0, 3)):
        L = 400
        c, A = 0.05, 12.0
        got = F.featurize(c * np.arange(L), fs, onset, 0.0, A)
        want = _ramp_features(c, fs, onset, L, A)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
        # unclamped velocity is 10 c fs / 1000 / A per point
        assert abs(got[256] - 10 * c * fs / 1000.0 / A) < 1e-12


def test_window_end_holds_the_last_sample():
    L, c, A = 120, 0.1, 10.0
    got = F.featurize(c * np.arange(L), 1000.0, 10, 0.0, A)
    pos, vel = got[:256], got[256:]
    k = L - 1 - 10          # first point at or past the last sample
    np.testing.assert_allclose(pos[k:], c * (L - 1) / A, rtol=1e-14)
    assert np.all(vel[k:] == 0.0)
    np.testing.assert_allclose(vel[:k], 10 * c / A, rtol=1e-12)


def test_mirrored_saccade_has_the_features_of_its_mirror_image():
    L = 300
    y = 2.0 + 0.07 * np.arange(L) + 0.01 * np.sin(np.arange(L))
    up = F.featurize(y, 1000.0, 10, 2.0, 14.0)
    down = F.featurize(-y, 1000.0, 10, -2.0, -14.0)
    np.testing.assert_array_equal(up, down)


def test_constant_trace_and_amplitude_floor():
    got = F.featurize(np.full(200, 3.0), 500.0, 5, 3.0, 3.0)
    assert np.all(got == 0.0)
    # amplitude 0.2 deg is floored at 0.5: the end fixation maps to 0.4
    y = np.concatenate([np.full(50, 1.0), np.full(150, 1.2)])
    got = F.featurize(y, 1000.0, 10, 1.0, 1.2)
    np.testing.assert_allclose(got[100:256], 0.4, rtol=1e-12)
