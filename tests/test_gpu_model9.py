"""The 9-parameter model (Sec. 2.2.2, Table 2) on the GPU, through the C ABI,
against the FP64 oracle: the same estimator over nine search coordinates
(shared K_SE and K_LT, neural control signal held at the box centre).
Tolerances as for the 18-parameter fits (1e-3 deg RMS; FP64 re-computation
of the GPU's winner to 1e-9 relative)."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2007_09884_gb300 as G
import workloads as W
from _support import centres, oracle_inputs, to_batch

pytestmark = pytest.mark.gpu

RMS_TOL = 1e-3
HELD = [10, 11, 12, 13, 15, 16, 17]   # activation/deactivation times, pulse heights, width


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = G.opmm_create(0)
    yield h
    G.opmm_destroy(h)


def _fit_both(ctx, items, S, T, **kw):
    res = G.opmm_fit_batch(ctx, to_batch(items), candidates=13 * S, iterations=T, model=G.OPMM_MODEL_9,
                           init_opc=centres(items), **kw)
    refs = [O.fit(it["pn"], it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"], S, T, model=9,
                  sac_index=j, tolx=kw.get("tol_x", 1e-4), tolf=kw.get("tol_f", 1e-4))
            for j, it in enumerate(items)]
    return res, refs


def test_fit_matches_oracle_and_keeps_the_model_structure(ctx):
    w = W.uneven10k(B=6)
    items = oracle_inputs(w)
    S, T = 40, 12
    res, refs = _fit_both(ctx, items, S, T, tol_x=0.0, tol_f=0.0)
    pcs = centres(items)
    for j, it in enumerate(items):
        assert res["status"][j] == 0
        assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL, (j, res["rms_deg"][j], refs[j]["rms"])
        p = res["opc"][j]
        assert p[0] == p[1] and p[2] == p[3]
        np.testing.assert_array_equal(p[HELD], pcs[j][HELD])
        # CPU_check: the oracle's FP64 error of the GPU's own winner
        mse, mae = O.errors(p.astype(np.float64), it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"])
        assert res["rms_deg"][j] == pytest.approx(math.sqrt(mse), rel=1e-9)
        assert res["l1_deg"][j] == pytest.approx(mae, rel=1e-9)
        # no tolerance: every simplex runs every iteration (10 starts + 13 per iteration)
        assert res["evaluations"][j] == S * 10 + T * S * 13
        # one pulse width for every candidate: all or none end inside the window
        assert res["pulse_end_evals"][j] in (0, res["evaluations"][j])


def test_initial_vertices_of_a_large_budget_match_oracle(ctx):
    """16,384 candidates: 1,260 simplices per saccade over several blocks and a
    partial one; with no iterations the winner is the best starting vertex."""
    w = W.uneven10k(B=3)
    items = oracle_inputs(w)
    S = 16384 // 13
    res, refs = _fit_both(ctx, items, S, 0)
    for j in range(len(items)):
        assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL
        bf = refs[j]["best_f_all"]
        assert bf[res["winner"][j]] - bf.min() <= 2.0 * math.sqrt(bf.min()) * 1e-4 + 1e-8 + 1e-6 * bf.min()
        assert res["evaluations"][j] == S * 10


def test_rejected_options(ctx):
    w = W.uneven10k(B=1)
    items = oracle_inputs(w)
    batch = to_batch(items)
    pc = centres(items).copy()
    pc[0, 1] *= 1.25                                # untied series elasticity
    with pytest.raises(G.OpmmError) as e:
        G.opmm_fit_batch(ctx, batch, candidates=130, iterations=2, model=G.OPMM_MODEL_9, init_opc=pc)
    assert e.value.code == G.OPMM_EINVAL
    with pytest.raises(G.OpmmError) as e:
        G.opmm_fit_batch(ctx, batch, candidates=12, iterations=2, model=G.OPMM_MODEL_9)
    assert e.value.code == G.OPMM_EINVAL
    with pytest.raises(G.OpmmError) as e:
        G.opmm_fit_batch(ctx, batch, candidates=130, iterations=2, model=7)
    assert e.value.code == G.OPMM_EINVAL
