"""opmm_fit_saccade_static: the fit for callers that cannot call cudaMalloc
(a real-time loop that must not stall on an allocation, or a program whose
device memory belongs to another allocator).  Its working memory is a fixed
array inside the library; this test calls it through the C ABI twice in a row
(two different saccades, so leftovers of the first call must not leak into the
second) and checks each result against opmm_fit_batch on the same input, within
the fit tolerance of the parity tests.  Kept in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2007_09884_gb300 as G
import workloads as W
from _support import f32, oracle_inputs, to_batch

pytestmark = pytest.mark.gpu

RMS_TOL = 1e-3


def _result(buf):
    r = G.opmm_fit_result.from_buffer_copy(bytes(buf))
    return G.results_to_numpy((G.opmm_fit_result * 1)(r))


def test_static_fit_matches_fit_batch_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    items = oracle_inputs(W.uneven10k(B=2))
    ctx = G.opmm_create(0)
    try:
        kw = dict(candidates=22 * 40, iterations=8, seed=5)
        dev_batch = to_batch(items, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        nbytes = ctypes.sizeof(G.opmm_fit_result)
        outs = []
        for j in range(2):
            out = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
            rc = G.opmm_fit_saccade_static(dev_batch, out, stream, index=j,
                                           pulse_init=G.OPMM_PULSE_CALIBRATED, **kw)
            assert rc == G.OPMM_OK
            outs.append(_result(out.cpu().numpy()))
        for j, got in enumerate(outs):
            # the batch fit counts saccade j as Philox counter word j; the
            # static call always uses word 0, so compare with a one-saccade batch
            one = G.opmm_fit_batch(ctx, to_batch([items[j]]), pulse_init=G.OPMM_PULSE_CALIBRATED, **kw)
            assert got["status"][0] == 0
            assert abs(got["rms_deg"][0] - one["rms_deg"][0]) <= RMS_TOL
            assert abs(got["f"][0] - one["f"][0]) <= 1e-6 + 1e-5 * one["f"][0]
            np.testing.assert_allclose(got["opc"][0], one["opc"][0], rtol=1e-5)
            assert got["evaluations"][0] == one["evaluations"][0]
    finally:
        G.opmm_destroy(ctx)


def test_static_fit_at_its_longest_trace_after_a_short_batch_fit():
    """A 4,096-sample trace (the largest the fixed array holds: its staged copy
    ends exactly at the array's end) with a caller-given box centre, fitted
    after a batch fit on a short trace has sized the search kernel for that
    short trace; the result must match opmm_fit_batch on the same input."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(4096)
    A, D, L = 10.0, 43.0, 4096
    pn = f32(O.nominal_opc(A, D, calibrated=False))
    ph = f32(pn * rng.uniform(0.8, 1.2, 18))
    y = f32(O.simulate_rk4(ph, L, 1000.0, 10, 0.0, A) + rng.normal(0.0, 0.05, L))
    long_item = dict(y=y, fs=1000.0, onset=10, th0=0.0, thf=A, dur=D, L=L)
    short_items = oracle_inputs(W.uneven10k(B=1))
    kw = dict(candidates=22 * 40, iterations=4, seed=3, init_opc=pn.astype(np.float32),
              pulse_init=G.OPMM_PULSE_TABLE1)
    nbytes = ctypes.sizeof(G.opmm_fit_result)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = G.opmm_create(0)
    try:
        # a static call on the short trace, then a batch fit on it, then the
        # static call on the longest trace
        out = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
        assert G.opmm_fit_saccade_static(to_batch(short_items, device="cuda"), out, stream,
                                         candidates=22 * 8, iterations=2, seed=1) == G.OPMM_OK
        G.opmm_fit_batch(ctx, to_batch(short_items), candidates=22 * 8, iterations=2, seed=1)
        out = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
        rc = G.opmm_fit_saccade_static(to_batch([long_item], device="cuda"), out, stream, **kw)
        assert rc == G.OPMM_OK
        got = _result(out.cpu().numpy())
        one = G.opmm_fit_batch(ctx, to_batch([long_item]), **kw)
        assert got["status"][0] == 0 and one["status"][0] == 0
        assert abs(got["rms_deg"][0] - one["rms_deg"][0]) <= RMS_TOL
        assert abs(got["f"][0] - one["f"][0]) <= 1e-6 + 1e-5 * one["f"][0]
        np.testing.assert_allclose(got["opc"][0], one["opc"][0], rtol=1e-5)
        assert got["evaluations"][0] == one["evaluations"][0]
    finally:
        G.opmm_destroy(ctx)


def test_static_fit_rejects_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    y = torch.zeros(5000, dtype=torch.float32, device="cuda")
    batch = G.make_batch(y, [1000.0], [10], [0.0], [10.0], [43.0], n_samples=[5000], offsets=[0])
    out = torch.zeros(ctypes.sizeof(G.opmm_fit_result), dtype=torch.uint8, device="cuda")
    assert G.opmm_fit_saccade_static(batch, out, 0, candidates=440, iterations=2) == G.OPMM_EINVAL
    y2 = torch.zeros(100, dtype=torch.float32, device="cuda")
    batch2 = G.make_batch(y2, [1000.0], [10], [0.0], [10.0], [43.0], n_samples=[100], offsets=[0])
    assert G.opmm_fit_saccade_static(batch2, out, 0, candidates=70000, iterations=2) == G.OPMM_EINVAL
    # options every fit rejects are rejected here too
    assert G.opmm_fit_saccade_static(batch2, out, 0, candidates=440, iterations=2,
                                     init_step=float("inf")) == G.OPMM_EINVAL
