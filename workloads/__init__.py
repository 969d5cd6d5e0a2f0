"""Seeded synthetic workloads shared by the oracle and the CUDA path.

This module holds only random draws and bookkeeping: saccade descriptors
(amplitude, direction, sample rate, window length, onset, duration from the
main-sequence rule of thumb), hidden-OPC multipliers and measurement noise.  It
contains none of the plant or estimator arithmetic; each side turns these draws
into traces with its own simulator (hidden OPC = nominal OPC x multiplier, trace
= simulated trajectory + noise).

The paper's recordings (Sec. 3: 32 subjects, 10 deg jumping dot, EyeLink 1000 at
1 kHz, I-VT detection) are not available; these synthetic saccades stand in for
them with the same shape: 1-D position traces in degrees, fixation -> saccade ->
fixation, onset 10 ms into the window, duration 2.2 ms/deg * A + 21 ms.

Every saccade i of workload c is drawn from its own generator seeded with
c * 2**32 + i, so any subset can be regenerated on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NP = 18
NOISE_SIGMA = 0.05          # deg, i.i.d. Gaussian measurement noise
HIDDEN_SPREAD = 0.20        # hidden OPC = nominal * U(1 - 0.2, 1 + 0.2)
ONSET_MS = 10.0             # fixation before the saccade inside the window
TAIL_MS = 20.0              # fixation after the saccade that a window must hold


def duration_ms(amplitude):
    """Main-sequence duration used for the workloads: 2.2 ms/deg * A + 21 ms."""
    return 2.2 * np.asarray(amplitude, dtype=np.float64) + 21.0


def onset_index(fs):
    return int(math.ceil(ONSET_MS * 1e-3 * float(fs) - 1e-9))


@dataclass
class Workload:
    """A batch of synthetic saccades (descriptor fields are float32-exact)."""
    name: str
    config_index: int
    fs: np.ndarray          # [B] float32 sample rate, Hz
    L: np.ndarray           # [B] int32 samples in the window
    onset: np.ndarray       # [B] int32 onset sample
    theta0: np.ndarray      # [B] float32 start fixation, deg
    thetaf: np.ndarray      # [B] float32 end fixation, deg
    dur_ms: np.ndarray      # [B] float32 saccade duration, ms
    amplitude: np.ndarray   # [B] float32 |thetaf - theta0|
    mult: np.ndarray        # [B, 18] float64 hidden OPC multipliers
    noise: list = field(default_factory=list)  # B arrays [L_i] float64, deg
    calibrated_pulse: bool = True
    # estimator settings
    candidates: int = 4096
    iterations: int = 20
    seed: int = 0

    @property
    def B(self) -> int:
        return int(self.fs.shape[0])

    @property
    def simplices(self) -> int:
        """Independent simplices per saccade: the per-iteration candidate
        budget divided by the n + 4 = 22 trial points of one simplex."""
        return self.candidates // (NP + 4)

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        return Workload(self.name + "[sub]", self.config_index, self.fs[idx], self.L[idx],
                        self.onset[idx], self.theta0[idx], self.thetaf[idx], self.dur_ms[idx],
                        self.amplitude[idx], self.mult[idx], [self.noise[i] for i in idx],
                        self.calibrated_pulse, self.candidates, self.iterations, self.seed)


def _rng(config_index: int, i: int) -> np.random.Generator:
    return np.random.default_rng(config_index * 2**32 + i)


def _finish(name, ci, rows, calibrated, candidates, iterations, seed, noise_sigma):
    fs = np.array([r[0] for r in rows], dtype=np.float32)
    L = np.array([r[1] for r in rows], dtype=np.int32)
    amp = np.array([r[2] for r in rows], dtype=np.float32)
    sign = np.array([r[3] for r in rows], dtype=np.float32)
    mult = np.array([r[4] for r in rows], dtype=np.float64).reshape(len(rows), NP)
    noise = [np.asarray(r[5], dtype=np.float64) * (noise_sigma / NOISE_SIGMA) for r in rows]
    onset = np.array([onset_index(f) for f in fs], dtype=np.int32)
    th0 = np.zeros(len(rows), dtype=np.float32)
    thf = (sign * amp).astype(np.float32)
    dur = duration_ms(amp.astype(np.float64)).astype(np.float32)
    return Workload(name, ci, fs, L, onset, th0, thf, dur, amp, mult, noise, calibrated,
                    candidates, iterations, seed)


def _draw_common(g: np.random.Generator, L: int):
    mult = g.uniform(1.0 - HIDDEN_SPREAD, 1.0 + HIDDEN_SPREAD, NP)
    noise = g.normal(0.0, NOISE_SIGMA, L)
    return mult, noise


def single10(noise_sigma: float = NOISE_SIGMA) -> Workload:
    """One horizontal 10 deg saccade at 1 kHz over a 150 ms window, Table 1
    pulse height, 4,096 candidates x 20 iterations, seed 0."""
    g = _rng(0, 0)
    mult, noise = _draw_common(g, 150)
    return _finish("single10", 0, [(1000.0, 150, 10.0, 1.0, mult, noise)], False, 4096, 20, 0,
                   noise_sigma)


def _amax(fs, L):
    win_ms = 1000.0 * L / fs
    on_ms = 1000.0 * onset_index(fs) / fs
    return (win_ms - on_ms - TAIL_MS - 21.0) / 2.2


def batch1024(B: int = 1024, noise_sigma: float = NOISE_SIGMA) -> Workload:
    """Plain batched search: amplitudes U(2, 30) deg (capped so the window
    holds onset + duration + 20 ms), windows U(60, 200) ms at 1 kHz, 65,536
    candidates x 30 iterations per saccade."""
    rows = []
    for i in range(B):
        g = _rng(1, i)
        L = int(g.integers(60, 201))
        amax = min(30.0, _amax(1000.0, L))
        A = float(np.float32(g.uniform(2.0, amax)))
        mult, noise = _draw_common(g, L)
        rows.append((1000.0, L, A, 1.0, mult, noise))
    return _finish("batch1024", 1, rows, True, 65536, 30, 0, noise_sigma)


def uneven10k(B: int = 10000, noise_sigma: float = NOISE_SIGMA, config_index: int = 2) -> Workload:
    """Uneven batch: rates {250, 500, 1000} Hz, both directions, amplitudes
    log-uniform in [1, 40] deg (capped by the window), windows of 40-400
    samples (redrawn until a 1 deg saccade fits), 16,384 candidates x 30."""
    rows = []
    for i in range(B):
        g = _rng(config_index, i)
        fs = float(g.choice([250.0, 500.0, 1000.0]))
        while True:
            L = int(g.integers(40, 401))
            amax = min(40.0, _amax(fs, L))
            if amax >= 1.0:
                break
        A = float(np.float32(math.exp(g.uniform(0.0, math.log(amax)))))
        sign = 1.0 if g.integers(0, 2) == 0 else -1.0
        mult, noise = _draw_common(g, L)
        rows.append((fs, L, A, sign, mult, noise))
    return _finish("uneven10k", config_index, rows, True, 16384, 30, 0, noise_sigma)


def poisson_arrivals(rate_hz: float, seconds: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    g = np.random.default_rng(seed)
    n = int(rate_hz * seconds * 1.2 + 64)
    t = np.cumsum(g.exponential(1.0 / rate_hz, n))
    return t[t < seconds]


def by_name(name: str, **kw) -> Workload:
    return {"single10": single10, "batch1024": batch1024, "uneven10k": uneven10k}[name](**kw)


def raw_stream(n_samples: int, fs: float = 1000.0, seed: int = 7, noise_deg: float = 0.005,
               blink_rate_hz: float = 0.2):
    """Seeded raw horizontal position stream for the I-VT front end: fixations
    (Gaussian noise of noise_deg) at positions uniform in [-20, 20] deg joined
    by saccades of amplitude 1-30 deg whose position follows a raised-cosine
    profile over the main-sequence duration 2.2 ms/deg * A + 21 ms, fixation
    lengths uniform in [150, 1200] ms, and blinks (runs of 80-200 ms of NaN) at
    blink_rate_hz on average.  Returns (stream float32, list of planted
    (start sample, end sample, amplitude))."""
    g = np.random.default_rng(np.random.SeedSequence([0x1F7, seed]))
    x = np.empty(n_samples, np.float32)
    planted = []
    pos = float(g.uniform(-10.0, 10.0))
    k = 0
    while k < n_samples:
        fix = int(g.uniform(0.15, 1.2) * fs)
        m = min(fix, n_samples - k)
        x[k:k + m] = pos + g.normal(0.0, noise_deg, m)
        k += m
        if k >= n_samples:
            break
        while True:
            target = float(g.uniform(-20.0, 20.0))
            A = abs(target - pos)
            if 1.0 <= A <= 30.0:
                break
        dur = int(round(duration_ms(A) * fs / 1000.0))
        m = min(dur, n_samples - k)
        t = (np.arange(1, m + 1) / dur).astype(np.float64)
        x[k:k + m] = pos + (target - pos) * 0.5 * (1.0 - np.cos(np.pi * t)) + g.normal(0.0, noise_deg, m)
        planted.append((k, k + m, abs(target - pos)))
        k += m
        pos = target
    nb = g.poisson(blink_rate_hz * n_samples / fs)
    for _ in range(int(nb)):
        b0 = int(g.integers(0, max(1, n_samples - 1)))
        bl = int(g.uniform(0.08, 0.2) * fs)
        x[b0:b0 + bl] = np.nan
    return x, planted
