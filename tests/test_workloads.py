"""The seeded input recipe: the synthetic workloads have the sizes, value
ranges and structure stated for them (window lengths, rates, amplitude law,
room in the window for onset + duration + 20 ms of fixation, hidden-OPC
spread, noise level, candidate budgets and simplex counts), and every
saccade is regenerated identically on its own."""
import math

import numpy as np

import workloads as W


def _fits_window(w):
    on_ms = 1000.0 * w.onset / w.fs
    need = on_ms + W.duration_ms(w.amplitude.astype(np.float64)) + W.TAIL_MS
    return np.all(need <= 1000.0 * w.L / w.fs + 1e-6)


def test_single_saccade_workload():
    w = W.single10()
    assert (w.B, float(w.fs[0]), int(w.L[0]), float(w.amplitude[0])) == (1, 1000.0, 150, 10.0)
    assert int(w.onset[0]) == 10 and float(w.dur_ms[0]) == np.float32(43.0)
    assert (w.candidates, w.iterations, w.simplices) == (4096, 20, 186)
    assert not w.calibrated_pulse


def test_batch_workload():
    w = W.batch1024()
    assert w.B == 1024 and np.all(w.fs == 1000.0)
    assert w.L.min() >= 60 and w.L.max() <= 200 and len(np.unique(w.L)) > 100
    assert w.amplitude.min() >= 2.0 and w.amplitude.max() <= 30.0
    assert np.all(w.thetaf > 0) and np.all(w.theta0 == 0) and np.all(w.onset == 10)
    assert _fits_window(w)
    assert (w.candidates, w.iterations, w.simplices) == (65536, 30, 2978)
    assert w.mult.min() >= 0.8 and w.mult.max() <= 1.2
    allnoise = np.concatenate(w.noise)
    assert abs(allnoise.std() - W.NOISE_SIGMA) < 0.002 and abs(allnoise.mean()) < 0.002


def test_uneven_workload():
    w = W.uneven10k()
    assert w.B == 10000
    rates, counts = np.unique(w.fs, return_counts=True)
    assert list(rates) == [250.0, 500.0, 1000.0] and counts.min() > 3000
    assert w.L.min() >= 40 and w.L.max() <= 400
    assert w.amplitude.min() >= 1.0 and w.amplitude.max() <= 40.0
    assert 0.4 < np.mean(w.thetaf > 0) < 0.6          # both directions
    assert _fits_window(w)
    # log-uniform below the cap: ln A spreads over [0, ln cap]; with the
    # uncapped draws, about half lie below sqrt(40)
    uncapped = np.array([W._amax(float(f), int(L)) >= 40.0 for f, L in zip(w.fs, w.L)])
    a = w.amplitude[uncapped]
    assert abs(np.mean(a < math.sqrt(40.0)) - 0.5) < 0.05
    assert (w.candidates, w.iterations, w.simplices) == (16384, 30, 744)


def test_each_saccade_is_seeded_on_its_own():
    small, large = W.batch1024(B=5), W.batch1024(B=40)
    assert np.array_equal(small.L, large.L[:5]) and np.array_equal(small.amplitude, large.amplitude[:5])
    assert np.array_equal(small.mult, large.mult[:5])
    assert all(np.array_equal(a, b) for a, b in zip(small.noise, large.noise[:5]))
    other = W.uneven10k(B=5, config_index=3)
    assert not np.array_equal(other.L, W.uneven10k(B=5).L)


def test_poisson_arrivals():
    for rate in (1000.0, 10000.0):
        t = W.poisson_arrivals(rate, 2.0, seed=int(rate))
        assert np.all(np.diff(t) > 0) and t[-1] < 2.0
        n = len(t)
        assert abs(n - 2.0 * rate) < 4.0 * math.sqrt(2.0 * rate)


def test_raw_stream_recipe():
    n, fs = 600_000, 1000.0
    x, planted = W.raw_stream(n, fs=fs, seed=11)
    assert x.dtype == np.float32 and len(x) == n
    amps = np.array([p[2] for p in planted])
    assert amps.min() >= 1.0 and amps.max() <= 30.0
    # saccade lengths follow the main-sequence duration; fixations between
    # them last 150-1200 ms
    for (k0, k1, a) in planted[:-1]:
        assert k1 - k0 == int(round(float(W.duration_ms(a)) * fs / 1000.0))
    gaps = np.array([planted[i + 1][0] - planted[i][1] for i in range(len(planted) - 1)])
    assert gaps.min() >= 150 and gaps.max() <= 1200
    finite = x[np.isfinite(x)]
    assert np.abs(finite).max() < 20.0 + 0.05
    # blinks: runs of NaN of 80-200 ms at about 0.2 per second
    nan = ~np.isfinite(x)
    starts = np.flatnonzero(nan[1:] & ~nan[:-1]) + 1
    assert 0.1 * n / fs < len(starts) < 0.3 * n / fs
    # fixation noise: 0.005 deg about the fixation position
    k0 = planted[0][1]
    seg = x[k0 + 5:planted[1][0] - 5].astype(np.float64)
    seg = seg[np.isfinite(seg)]
    assert abs(seg.std() - 0.005) < 0.002
