"""Velocity-threshold (I-VT) saccade detection and cleaning of a raw position
stream: the reference definition for the device front end.

TEST INFRASTRUCTURE ONLY: the product package never imports this module; the
tests, the smoke check and the benchmark's baseline leg do.  It shares no code
with the CUDA path.

The paper segments its recordings with the Velocity-Threshold algorithm and
discards saccades shorter than 6 ms or smaller than 4 deg (Sec. 4); it gives
no velocity threshold and no cleaning rule.  The reading written out here:

* a sample is valid when it is finite and inside [valid_min_deg, valid_max_deg]
  (track loss and blinks show as NaN or out-of-range positions);
* step k (between samples k - 1 and k, k >= 1) is fast when both samples are
  valid and |theta_k - theta_(k-1)| * fs > threshold;
* a saccade is a maximal run of fast steps k in [a, b); its onset sample is
  s = a - 1 (the last sample before the movement) and its end sample
  e = b - 1 (the first sample after it); amplitude |theta_e - theta_s|,
  duration (e - s) / fs, peak velocity the largest |step| * fs in the run;
* it is kept when the duration is at least min_duration_ms, the amplitude at
  least min_amplitude_deg, and the window [s - pre, e + post] lies inside the
  stream with every sample valid (the descriptor for the estimator is that
  window, onset index pre, start fixation theta_s, end fixation theta_e,
  duration (e - s) / fs).

Velocities, amplitudes and durations are computed in float32, the precision
the device takes the same decisions in, so both sides draw every boundary
identically.  Plain loops over the runs (numpy only for the elementwise steps).
"""
from __future__ import annotations

import numpy as np


def ivt(theta, fs, threshold_dps=30.0, min_duration_ms=6.0, min_amplitude_deg=4.0, valid_min_deg=-90.0,
        valid_max_deg=90.0, pre_samples=10, post_samples=40):
    x = np.asarray(theta, dtype=np.float32)
    n = len(x)
    f = np.float32(fs)
    thr = np.float32(threshold_dps)
    valid = np.isfinite(x) & (x >= np.float32(valid_min_deg)) & (x <= np.float32(valid_max_deg))
    fast = np.zeros(n, dtype=bool)
    speed = np.zeros(n, dtype=np.float32)
    if n > 1:
        with np.errstate(invalid="ignore"):
            speed[1:] = np.abs(x[1:] - x[:-1]) * f
        fast[1:] = valid[1:] & valid[:-1] & (speed[1:] > thr)
    events = []
    k = 1
    while k < n:
        if not fast[k]:
            k += 1
            continue
        a = k
        while k < n and fast[k]:
            k += 1
        b = k
        s, e = a - 1, b - 1
        amp = np.float32(abs(x[e] - x[s]))
        dur = np.float32(np.float32(e - s) * np.float32(1000.0) / f)
        peak = np.float32(speed[a:b].max())
        ws, we = s - int(pre_samples), e + int(post_samples)
        keep = (dur >= np.float32(min_duration_ms) and amp >= np.float32(min_amplitude_deg) and ws >= 0
                and we <= n - 1 and bool(valid[ws:we + 1].all()))
        if keep:
            events.append({"onset": s, "end": e, "theta_start": float(x[s]), "theta_end": float(x[e]),
                           "amplitude": float(amp), "duration_ms": float(dur), "peak_velocity": float(peak),
                           "window_start": ws, "n_samples": we - ws + 1, "onset_index": s - ws})
    return events
