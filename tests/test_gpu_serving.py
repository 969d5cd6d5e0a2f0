"""The real-time request loop: continuous batching, results independent of
the mix (T12), and the host-side failure paths (T15): admission refused by the
memory budget, queue-full back-pressure, poll deadlines, malformed requests,
stop.  Nothing here faults or hangs the GPU: every failure is made on the host.
"""
import time

import numpy as np
import pytest

import paper_2007_09884_gb300 as G
import workloads as W
from _support import oracle_inputs, to_batch

pytestmark = pytest.mark.gpu

FIT = dict(candidates=22 * 24, iterations=12, seed=3, pulse_init=G.OPMM_PULSE_CALIBRATED)


@pytest.fixture()
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = G.opmm_create(0)
    yield h
    G.opmm_serve_stop(h)
    G.opmm_destroy(h)


def test_result_is_the_same_alone_and_in_a_mix(ctx):
    items = oracle_inputs(W.uneven10k(B=16))
    batch = to_batch(items)
    G.opmm_serve_start(ctx, G.serve_opts(max_slots=64, round_iters=3), **FIT)
    t = G.opmm_serve_submit(ctx, batch, 5)
    alone, _ = G.opmm_serve_poll(ctx, t)
    # the same saccade again, arriving while others are being searched
    tickets = []
    for j in range(16):
        tickets.append(G.opmm_serve_submit(ctx, batch, j))
        if j % 4 == 3:
            time.sleep(0.002)
    mixed = [G.opmm_serve_poll(ctx, tk)[0] for tk in tickets]
    m = mixed[5]
    np.testing.assert_array_equal(m["opc"], alone["opc"])
    assert m["f"] == alone["f"] and m["rms_deg"] == alone["rms_deg"]
    assert m["evaluations"] == alone["evaluations"]
    st = G.opmm_serve_stats_get(ctx)
    assert st["completed"] == 17 and st["submitted"] == 17
    # and equal to the one-shot fit of that saccade (one-saccade batch)
    one = G.opmm_fit_batch(ctx, to_batch([items[5]]), **FIT)
    np.testing.assert_array_equal(one["opc"][0], alone["opc"])
    assert one["rms_deg"][0] == alone["rms_deg"]


def test_admission_refused_when_memory_budget_is_short(ctx):
    with pytest.raises(G.OpmmError) as e:
        G.opmm_serve_start(ctx, G.serve_opts(max_device_bytes=1000), **FIT)
    assert e.value.code == G.OPMM_EBUSY


def test_queue_full_poll_deadlines_and_bad_requests(ctx):
    items = oracle_inputs(W.uneven10k(B=4))
    batch = to_batch(items)
    slow = dict(FIT, candidates=22 * 400, iterations=400)
    G.opmm_serve_start(ctx, G.serve_opts(max_slots=1, max_queue=2, round_iters=1, max_admit_per_round=1), **slow)
    descs, keep = batch.descriptors()
    codes, tickets = [], []
    for j in range(8):
        rc, t = G.opmm_serve_submit_raw(ctx, descs[j % 4])
        codes.append(rc)
        if rc == G.OPMM_OK:
            tickets.append(t)
    assert G.OPMM_EBUSY in codes                      # back-pressure
    assert G.opmm_serve_stats_get(ctx)["rejected"] >= 1
    rc, res, _ = G.opmm_serve_poll_raw(ctx, tickets[-1], 0)
    assert rc == G.OPMM_NOT_READY and res is None
    rc, _, _ = G.opmm_serve_poll_raw(ctx, tickets[-1], 1000)
    assert rc == G.OPMM_ETIMEDOUT
    rc, _, _ = G.opmm_serve_poll_raw(ctx, 987654321, 0)
    assert rc == G.OPMM_EINVAL                         # unknown ticket
    bad = G.make_batch([np.zeros(20, np.float32)], [1000.0], [25], [0.0], [5.0], [30.0])
    d, k2 = bad.descriptors()
    rc, _ = G.opmm_serve_submit_raw(ctx, d[0])
    assert rc == G.OPMM_EINVAL                         # onset outside the window
    G.opmm_serve_stop(ctx)
    rc, _, _ = G.opmm_serve_poll_raw(ctx, tickets[0], 0)
    assert rc == G.OPMM_EINVAL                         # stopped: requests dropped


def test_more_requests_than_slots(ctx):
    """Requests queue while every slot is busy and are admitted as slots free
    up; each still gets exactly its own result."""
    items = oracle_inputs(W.uneven10k(B=8))
    batch = to_batch(items)
    G.opmm_serve_start(ctx, G.serve_opts(max_slots=3, round_iters=4, max_admit_per_round=64), **FIT)
    tickets = [G.opmm_serve_submit(ctx, batch, j % 8) for j in range(24)]
    res = [G.opmm_serve_poll(ctx, t)[0] for t in tickets]
    assert all(r["status"] == 0 for r in res)
    for j in range(8):
        for r in res[j::8]:
            np.testing.assert_array_equal(r["opc"], res[j]["opc"])
    one = G.opmm_fit_batch(ctx, to_batch([items[2]]), **FIT)
    np.testing.assert_array_equal(one["opc"][0], res[2]["opc"])
    st = G.opmm_serve_stats_get(ctx)
    assert st["slots"] == 3 and st["completed"] == 24
