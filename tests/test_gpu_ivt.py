"""The I-VT front end on the GPU (opmm_detect_saccades, through the C ABI)
against the reference definition (oracle/ivt.py): both take every decision in
FP32, so the event lists agree exactly: onset and end samples, windows, and
the float fields bit for bit."""
import numpy as np
import pytest

import paper_2007_09884_gb300 as G
import workloads as W
from oracle.ivt import ivt

pytestmark = pytest.mark.gpu

FIELDS = [("onset", "onset"), ("end", "end"), ("window_start", "window_start"), ("n_samples", "n_samples"),
          ("onset_index", "onset_index"), ("theta_start_deg", "theta_start"), ("theta_end_deg", "theta_end"),
          ("amplitude_deg", "amplitude"), ("duration_ms", "duration_ms"), ("peak_velocity_dps", "peak_velocity")]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = G.opmm_create(0)
    yield h
    G.opmm_destroy(h)


def _same(got, want):
    assert len(got) == len(want), (len(got), len(want))
    for g, w in zip(got, want):
        for a, b in FIELDS:
            if a in ("theta_start_deg", "theta_end_deg", "amplitude_deg", "duration_ms", "peak_velocity_dps"):
                assert np.float32(g[a]) == np.float32(w[b]), (a, g[a], w[b])
            else:
                assert int(g[a]) == int(w[b]), (a, g[a], w[b])


def _ramp(n, at, length, amp):
    x = np.zeros(n, np.float32)
    for i in range(1, length + 1):
        x[at + i] = amp * i / length
    x[at + length + 1:] = amp
    return x


def test_closed_form_streams(ctx):
    cases = [_ramp(400, 100, 12, 12.0), _ramp(300, 100, 1, 10.0), _ramp(300, 100, 10, 3.0), _ramp(400, 5, 12, 12.0)]
    blink = _ramp(400, 100, 12, 12.0)
    blink[140] = np.nan
    cases.append(blink)
    for x in cases:
        for kw in ({}, {"min_duration_ms": 0.0, "min_amplitude_deg": 0.0}):
            _same(G.opmm_detect_saccades(ctx, x, 1000.0, **kw), ivt(x, 1000.0, **kw))


@pytest.mark.parametrize("fs", [1000.0, 500.0, 250.0])
def test_synthetic_stream_matches_the_definition(ctx, fs):
    x, planted = W.raw_stream(400_000 if fs == 1000.0 else 150_000, fs=fs, seed=int(fs))
    want = ivt(x, fs)
    got = G.opmm_detect_saccades(ctx, x, fs)
    assert len(want) > 100
    _same(got, want)


def test_tiles_of_many_runs(ctx):
    """Tiles of 8,192 steps holding 64 run starts (the most the count pass
    records; ranked into order from those records), 65 and a noisy stretch
    with hundreds (read again and written in stream order), beside sparse
    tiles: every run is kept (filters off) and the events are the same as
    the definition's."""
    tile = 8192
    n = 5 * tile + 1000
    dx = np.zeros(n, np.float64)
    sign = 1.0
    for first, count, spacing in ((100, 64, 100), (tile + 50, 65, 120), (2 * tile + 7, 63, 128), (4 * tile + 300, 3, 2000)):
        for j in range(count):
            dx[first + j * spacing] = sign      # one fast step: x rises or falls by 1 deg between samples k-1, k
            sign = -sign
    x = np.cumsum(dx).astype(np.float32)
    x[3 * tile:4 * tile] += np.random.default_rng(2).normal(0.0, 0.01, tile).astype(np.float32)
    kw = {"min_duration_ms": 0.0, "min_amplitude_deg": 0.0}
    want = ivt(x, 1000.0, **kw)
    starts = np.array([int(w["onset"]) + 1 for w in want])
    per_tile = np.bincount((starts - 1) // tile, minlength=5)
    assert per_tile[0] == 64 and per_tile[1] == 65 and per_tile[2] == 63 and per_tile[3] > 64, per_tile
    _same(G.opmm_detect_saccades(ctx, x, 1000.0, **kw), want)


def test_degenerate_streams(ctx):
    """A stream of track loss only, the shortest streams (two and three
    samples, one step), with and without filters and margins."""
    streams = (np.full(1000, np.nan, np.float32), np.array([0.0, 10.0], np.float32), np.zeros(2, np.float32),
               np.array([0.0, 10.0, 10.0], np.float32))
    for x in streams:
        for kw in ({}, {"min_duration_ms": 0.0, "min_amplitude_deg": 0.0, "pre_samples": 0, "post_samples": 0}):
            _same(G.opmm_detect_saccades(ctx, x, 1000.0, **kw), ivt(x, 1000.0, **kw))
    # infinite samples are never valid, even with an unbounded valid range
    ramp = np.concatenate([np.zeros(100), np.linspace(0.0, 12.0, 13), np.full(287, 12.0)]).astype(np.float32)
    inf_in, inf_out = ramp.copy(), ramp.copy()
    inf_in[105] = np.inf
    inf_out[300] = -np.inf
    kw = {"valid_min_deg": -np.inf, "valid_max_deg": np.inf, "min_duration_ms": 0.0, "min_amplitude_deg": 0.0}
    for x, kept in ((ramp, 1), (inf_in, 0), (inf_out, 1)):
        want = ivt(x, 1000.0, **kw)
        assert len(want) == kept
        _same(G.opmm_detect_saccades(ctx, x, 1000.0, **kw), want)


def test_device_stream_window_options_and_truncation(ctx):
    torch = pytest.importorskip("torch")
    x, _ = W.raw_stream(200_000, seed=11)
    kw = dict(threshold_dps=45.0, min_duration_ms=10.0, min_amplitude_deg=2.0, pre_samples=25, post_samples=60,
              valid_min_deg=-25.0, valid_max_deg=25.0)
    want = ivt(x, 1000.0, **kw)
    got = G.opmm_detect_saccades(ctx, torch.from_numpy(x).cuda(), 1000.0, **kw)
    _same(got, want)
    few = G.opmm_detect_saccades(ctx, x, 1000.0, max_events=5, **kw)
    _same(few, want[:5])
    # the detected windows are descriptors the estimator takes
    batch = G.batch_from_events(x, got[:8], 1000.0)
    res = G.opmm_fit_batch(ctx, batch, candidates=22 * 8, iterations=4)
    assert np.all(res["status"] == 0)


def test_unaligned_device_stream_takes_the_scalar_path(ctx):
    """A stream starting 4 bytes past a 16-byte boundary is read sample by
    sample (no 16-byte loads); the events are the same."""
    torch = pytest.importorskip("torch")
    x, _ = W.raw_stream(100_003, seed=5)
    full = torch.from_numpy(np.concatenate([np.zeros(1, np.float32), x])).cuda()
    view = full[1:]
    assert view.data_ptr() % 16 != 0
    _same(G.opmm_detect_saccades(ctx, view, 1000.0), ivt(x, 1000.0))


def test_rejected_arguments(ctx):
    x = np.zeros(100, np.float32)
    for bad in (dict(threshold_dps=0.0), dict(pre_samples=-1), dict(valid_min_deg=5.0, valid_max_deg=-5.0)):
        with pytest.raises(G.OpmmError) as e:
            G.opmm_detect_saccades(ctx, x, 1000.0, **bad)
        assert e.value.code == G.OPMM_EINVAL
    with pytest.raises(G.OpmmError) as e:
        G.opmm_detect_saccades(ctx, x[:1], 1000.0)
    assert e.value.code == G.OPMM_EINVAL
