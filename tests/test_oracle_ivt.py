"""Pins of the I-VT front end's reference definition (oracle/ivt.py) on
streams whose saccades are known in closed form: a linear ramp, a step, a
sub-threshold drift, a blink, two saccades, and the 6 ms / 4 deg filters the
paper applies (Sec. 4)."""
import numpy as np

from oracle.ivt import ivt


def _ramp(n, at, length, amp, base=0.0):
    """Fixation at base, a linear ramp of amp deg over length steps starting
    after sample at, fixation at base + amp."""
    x = np.full(n, base, np.float32)
    for i in range(1, length + 1):
        x[at + i] = base + amp * i / length
    x[at + length + 1:] = base + amp
    return x


def test_linear_ramp_gives_one_saccade_with_its_closed_form():
    x = _ramp(400, 100, 12, 12.0)      # 12 deg in 12 ms at 1 kHz: 1000 deg/s
    ev = ivt(x, 1000.0)
    assert len(ev) == 1
    e = ev[0]
    assert (e["onset"], e["end"]) == (100, 112)
    assert e["amplitude"] == np.float32(12.0) and e["duration_ms"] == np.float32(12.0)
    assert abs(e["peak_velocity"] - 1000.0) < 1e-3
    assert (e["window_start"], e["n_samples"], e["onset_index"]) == (90, 63, 10)
    assert (e["theta_start"], e["theta_end"]) == (0.0, 12.0)


def test_step_is_too_short_unless_the_duration_filter_is_off():
    x = _ramp(300, 100, 1, 10.0)
    assert ivt(x, 1000.0) == []
    ev = ivt(x, 1000.0, min_duration_ms=0.0)
    assert len(ev) == 1 and ev[0]["duration_ms"] == np.float32(1.0) and ev[0]["amplitude"] == np.float32(10.0)


def test_subthreshold_drift_and_small_saccades_are_not_saccades():
    drift = _ramp(600, 50, 400, 8.0)   # 20 deg/s < 30 deg/s
    assert ivt(drift, 1000.0) == []
    small = _ramp(300, 100, 10, 3.0)   # 300 deg/s but 3 deg < 4 deg
    assert ivt(small, 1000.0) == []
    assert len(ivt(small, 1000.0, min_amplitude_deg=2.0)) == 1


def test_blink_in_the_window_discards_the_saccade():
    x = _ramp(400, 100, 12, 12.0)
    y = x.copy()
    y[140] = np.nan                    # inside the post window (112 + 40)
    assert ivt(y, 1000.0) == []
    z = x.copy()
    z[200] = np.nan                    # outside it
    assert len(ivt(z, 1000.0)) == 1
    w = x.copy()
    w[95] = 500.0                      # out-of-range sample in the pre window
    assert ivt(w, 1000.0) == []


def test_two_saccades_and_the_window_edges():
    x = _ramp(800, 100, 10, 10.0)
    x[500:] = 10.0 - np.float32(8.0) * np.minimum(np.arange(300, dtype=np.float32) / 8.0, 1.0)
    ev = ivt(x, 1000.0)
    assert [(e["onset"], e["end"]) for e in ev] == [(100, 110), (500, 508)]
    assert ev[1]["amplitude"] == np.float32(8.0)
    # a saccade too close to the stream's start has no complete window
    assert ivt(_ramp(400, 5, 12, 12.0), 1000.0) == []


def test_velocity_scales_with_the_rate():
    x = _ramp(400, 100, 12, 12.0)      # per-sample step 1 deg
    ev = ivt(x, 250.0)                 # 250 deg/s at 250 Hz, 48 ms
    assert len(ev) == 1 and ev[0]["duration_ms"] == np.float32(48.0)
    assert ivt(x, 20.0) == []          # 20 deg/s: below threshold


def test_infinite_samples_are_invalid_even_in_an_unbounded_range():
    """Valid means finite as well as in range: with the range opened to
    (-inf, inf) an infinite sample still breaks its steps and spoils any
    window that holds it, as NaN does."""
    x = _ramp(400, 100, 12, 12.0)
    wide = {"valid_min_deg": -np.inf, "valid_max_deg": np.inf}
    assert len(ivt(x, 1000.0, **wide)) == 1
    for bad in (np.inf, -np.inf, np.nan):
        y = x.copy()
        y[140] = bad                   # inside the post window
        assert ivt(y, 1000.0, **wide) == []
        z = x.copy()
        z[300] = bad                   # outside every window
        assert len(ivt(z, 1000.0, **wide)) == 1
        r = x.copy()
        r[106] = bad                   # inside the run: steps 106 and 107 are not fast
        runs = ivt(r, 1000.0, min_duration_ms=0.0, min_amplitude_deg=0.0, pre_samples=0, post_samples=0, **wide)
        assert [(e["onset"], e["end"]) for e in runs] == [(100, 105), (107, 112)]


def test_planted_saccades_of_a_synthetic_stream_are_recovered():
    """On the seeded raw stream (fixations with 0.005 deg noise, raised-cosine
    saccades of 1-30 deg, blinks of NaN), every kept event lies on a planted
    saccade, and the planted saccades of at least 4.5 deg whose windows are
    free of blinks are found with their amplitude (the raised cosine crosses
    the 30 deg/s threshold within its first and last few percent of
    amplitude, so a planted 4.04 deg saccade may measure just under the 4 deg
    filter)."""
    import workloads as W
    x, planted = W.raw_stream(400_000, seed=3)
    ev = ivt(x, 1000.0)
    assert len(ev) > 100
    starts = np.array([p[0] for p in planted])
    for e in ev:
        i = int(np.searchsorted(starts, e["onset"] + 1, side="right")) - 1
        k0, k1, amp = planted[i]
        assert k0 - 1 <= e["onset"] < e["end"] <= k1, (e, planted[i])
    found = {int(np.searchsorted(starts, e["onset"] + 1, side="right")) - 1: e for e in ev}
    eligible = 0
    for i, (k0, k1, amp) in enumerate(planted):
        lo, hi = k0 - 10 - 5, k1 + 40 + 5
        if amp < 4.5 or lo < 0 or hi >= len(x) or not np.all(np.isfinite(x[lo:hi])):
            continue
        eligible += 1
        assert i in found, (k0, k1, amp)
        assert abs(found[i]["amplitude"] - amp) <= 0.03 * amp + 0.02
    assert eligible > 100
