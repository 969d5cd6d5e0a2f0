"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here, from the FP32 arithmetic of each quantity):
  * trajectories: 1e-4 deg max abs per sample;
  * objective f (mean squared error): the trajectory bound d gives
    |f_gpu - f_ref| <= 2 sqrt(f) d + d^2, plus FP32 summation noise;
  * fits: |RMS_gpu - RMS_oracle| <= 1e-3 deg (both runs of the same estimator
    from the same seeded starts; FP32 and FP64 may take different branches on
    near-ties, so the parameter vectors are not compared);
  * the FP64 residual the GPU reports for its winner equals the oracle's
    recomputation for that same OPC vector (the OptErr / CPU_check pattern of
    Fig. 4, there ~1e-6 relative; here both are FP64 RK4 of the same vector).
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2007_09884_gb300 as G
import workloads as W
from _support import centres, f32, oracle_inputs, oracle_inputs_parallel, pulse_equilibrium_distance, to_batch

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-4
RMS_TOL = 1e-3


def f_tol(f):
    return 2.0 * math.sqrt(max(f, 0.0)) * TRAJ_TOL + TRAJ_TOL**2 + 1e-6 * f


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = G.opmm_create(0)
    yield h
    G.opmm_destroy(h)


def _random_cases(n, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(n):
        fs = float(rng.choice([250.0, 500.0, 1000.0, 600.0, 120.0]))
        A = float(np.exp(rng.uniform(np.log(0.5), np.log(40.0))))
        D = 2.2 * A + 21.0
        L = int(rng.integers(1, 401))
        if i % 7 == 0:
            on = L - 1
        else:
            on = int(min(L - 1, math.ceil(0.01 * fs)))
        th0 = float(np.float32(rng.uniform(-15, 15)))
        sgn = 1.0 if rng.integers(2) else -1.0
        thf = float(np.float32(th0 + sgn * A))
        box = rng.uniform(0.5, 2.0, 18)
        if i % 11 == 0:
            box[17] = 40.0     # pulse outlasting the window
        p = f32(O.nominal_opc(A, D) * box)
        cases.append(dict(p=p, L=L, fs=fs, onset=on, th0=th0, thf=thf, dur=D))
    return cases


def test_simulate_matches_oracle_10k(ctx):
    """T5: 10^4 random OPC vectors in the [0.5x, 2x] box, rates 120-1000 Hz,
    windows 1-400 samples, both directions, onset at the window edge, pulses
    longer than the window: max abs error <= 1e-4 deg per sample."""
    cases = _random_cases(10000, 11)
    batch = G.make_batch([np.zeros(c["L"], np.float32) for c in cases], [c["fs"] for c in cases],
                         [c["onset"] for c in cases], [c["th0"] for c in cases],
                         [c["thf"] for c in cases], [c["dur"] for c in cases])
    opc = np.stack([c["p"] for c in cases]).astype(np.float32)
    out, offs = G.opmm_simulate(ctx, opc, batch)
    worst = 0.0
    for c, o in zip(cases, offs):
        ref = O.simulate_rk4(c["p"], c["L"], c["fs"], c["onset"], c["th0"], c["thf"])
        got = out[o:o + c["L"]].astype(np.float64)
        worst = max(worst, float(np.max(np.abs(got - ref))))
    assert worst <= TRAJ_TOL, worst


def test_simulate_device_buffers_and_sac_index(ctx):
    torch = pytest.importorskip("torch")
    cases = _random_cases(64, 12)
    batch = G.make_batch([np.zeros(c["L"], np.float32) for c in cases[:4]], [c["fs"] for c in cases[:4]],
                         [c["onset"] for c in cases[:4]], [c["th0"] for c in cases[:4]],
                         [c["thf"] for c in cases[:4]], [c["dur"] for c in cases[:4]])
    idx = np.arange(64, dtype=np.int32) % 4
    opc = np.stack([c["p"] for c in cases]).astype(np.float32)
    host, offs = G.opmm_simulate(ctx, opc, batch, sac_index=idx)
    dev_out = torch.zeros(len(host), dtype=torch.float32, device="cuda")
    dev, _ = G.opmm_simulate(ctx, torch.from_numpy(opc).cuda(), batch, sac_index=idx, out=dev_out)
    np.testing.assert_array_equal(dev.cpu().numpy(), host)


def test_nominal_opc_matches_oracle(ctx):
    """Box centres: Table 1 with W = D - 6 ms; the calibrated agonist pulse
    agrees with the oracle's bisection to 1e-4 relative."""
    amps = np.concatenate([np.linspace(0.5, 45.0, 40), [1.0, 10.0, 20.0, 40.0]]).astype(np.float32)
    n = len(amps)
    D = (2.2 * amps.astype(np.float64) + 21.0).astype(np.float32)
    sg = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    batch = G.make_batch([np.zeros(100, np.float32)] * n, [1000.0] * n, [10] * n, [0.0] * n,
                         sg * amps, D)
    cal = G.opmm_nominal_opc(ctx, batch, G.OPMM_PULSE_CALIBRATED)
    tab = G.opmm_nominal_opc(ctx, batch, G.OPMM_PULSE_TABLE1)
    for i in range(n):
        ref_t = O.nominal_table1(float(D[i]))
        np.testing.assert_allclose(tab[i], ref_t.astype(np.float32), rtol=0, atol=0)
        ref_n = O.calibrate_pulse(float(amps[i]), float(D[i]))
        assert abs(cal[i, 15] - ref_n) <= 1e-4 * ref_n, (amps[i], cal[i, 15], ref_n)


def test_score_matches_oracle(ctx):
    w = W.single10()
    it = oracle_inputs(w)[0]
    batch = to_batch([it])
    rng = np.random.default_rng(3)
    m = 3000
    opc = (it["pn"] * rng.uniform(0.5, 2.0, (m, 18))).astype(np.float32)
    opc[-2] = it["pn"].astype(np.float32) * np.array([1] * 6 + [10.0] + [1] * 2 + [0.1] + [1] * 8,
                                                     dtype=np.float32)   # stiff: refined substeps
    opc[-1] = it["pn"].astype(np.float32) * np.array([1] * 6 + [1000.0] + [1] * 2 + [0.001] + [1] * 8,
                                                     dtype=np.float32)   # too stiff: +inf
    got = G.opmm_score(ctx, opc, batch)
    for i in range(m):
        ref, _ = O.errors(opc[i].astype(np.float64), it["L"], it["fs"], it["onset"], it["th0"],
                          it["thf"], it["y"])
        if math.isinf(ref):
            assert math.isinf(got[i])
        else:
            assert abs(got[i] - ref) <= f_tol(ref), (i, got[i], ref)


def test_grid_argmin_matches_oracle(ctx):
    """T7 on the GPU: a 41 x 41 grid over (passive viscosity, agonist pulse)
    with the other OPCs at the hidden values; the GPU's best grid point is the
    oracle's (or ties with it within the objective tolerance)."""
    w = W.single10()
    it = oracle_inputs(w)[0]
    batch = to_batch([it])
    g = np.linspace(np.log(0.5), np.log(2.0), 41)
    pts = np.array([(a, b) for a in g for b in g])
    base = it["ph"].copy()
    base[6], base[15] = it["pn"][6], it["pn"][15]
    opc = np.repeat(base[None, :], len(pts), axis=0)
    opc[:, 6] *= np.exp(pts[:, 0])
    opc[:, 15] *= np.exp(pts[:, 1])
    opc = opc.astype(np.float32)
    got = G.opmm_score(ctx, opc, batch)
    ref = np.array([O.errors(o.astype(np.float64), it["L"], it["fs"], it["onset"], it["th0"],
                             it["thf"], it["y"])[0] for o in opc])
    kg, kr = int(np.argmin(got)), int(np.argmin(ref))
    assert kg == kr or ref[kg] - ref[kr] <= f_tol(ref[kr])


def _fit_both(ctx, items, S, T, seed=0, nthreads=None, **kw):
    batch = to_batch(items)
    res = G.opmm_fit_batch(ctx, batch, candidates=22 * S, iterations=T, seed=seed,
                           init_opc=centres(items), **kw)
    refs = []
    for j, it in enumerate(items):
        refs.append(O.fit(it["pn"], it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"],
                          S, T, seed=seed, sac_index=j, nthreads=nthreads,
                          box_lo=kw.get("box_lo", 0.5), box_hi=kw.get("box_hi", 2.0),
                          step=kw.get("init_step", 0.05)))
    return res, refs


def test_fit_single10_matches_oracle(ctx):
    """T10/T11 on the single-saccade workload (10 deg, 1 kHz, 150 samples,
    4,096 candidates x 20 iterations, seed 0)."""
    w = W.single10()
    items = oracle_inputs(w)
    res, refs = _fit_both(ctx, items, w.simplices, w.iterations, seed=w.seed)
    it, ref = items[0], refs[0]
    assert res["status"][0] == 0
    assert abs(res["rms_deg"][0] - ref["rms"]) <= RMS_TOL, (res["rms_deg"][0], ref["rms"])
    assert res["rms_deg"][0] < 0.1
    # CPU_check: the oracle's FP64 error of the GPU's own winner
    p = res["opc"][0].astype(np.float64)
    mse, mae = O.errors(p, it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"])
    assert res["rms_deg"][0] == pytest.approx(math.sqrt(mse), rel=1e-9)
    assert res["l1_deg"][0] == pytest.approx(mae, rel=1e-9)
    assert abs(res["f"][0] - mse) <= f_tol(mse)


def test_fit_uneven_batch_matches_oracle(ctx):
    """Mixed rates, both directions, ragged windows, a partial simplex group."""
    w = W.uneven10k(B=12)
    items = oracle_inputs(w)
    res, refs = _fit_both(ctx, items, 19, 8)
    for j in range(len(items)):
        assert res["status"][j] == 0
        assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL, (j, res["rms_deg"][j], refs[j]["rms"])
        p = res["opc"][j].astype(np.float64)
        it = items[j]
        mse, _ = O.errors(p, it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"])
        assert res["rms_deg"][j] == pytest.approx(math.sqrt(mse), rel=1e-9)


def test_fit_zero_iterations_is_best_initial_vertex(ctx):
    w = W.uneven10k(B=3)
    items = oracle_inputs(w)
    res, refs = _fit_both(ctx, items, 5, 0)
    for j in range(3):
        assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL
        assert res["iterations_run"][j] == 0


def test_plan_graph_is_deterministic_and_equals_fit_batch(ctx):
    """A captured plan replays bit-identically and equals the one-shot fit on
    the same launch variant; an autotuned plan agrees within tolerance."""
    w = W.uneven10k(B=6)
    items = oracle_inputs(w)
    batch = to_batch(items)
    kw = dict(candidates=22 * 40, iterations=6, init_opc=centres(items))
    G.opmm_set_search_variant(ctx, 0)
    try:
        a = G.opmm_fit_batch(ctx, batch, **kw)
        plan = G.opmm_plan_create(ctx, batch, **kw)
        b = plan.execute()
        c = plan.execute()
        for k in ("opc", "f", "rms_deg", "winner", "iterations_run", "evaluations"):
            np.testing.assert_array_equal(a[k], b[k])
            np.testing.assert_array_equal(b[k], c[k])
        plan.destroy()
    finally:
        G.opmm_set_search_variant(ctx, -1)
    tuned = G.opmm_plan_create(ctx, batch, **kw)
    d = tuned.execute()
    info = tuned.info()
    assert info["simplices_per_block"] in (8, 16, 32)
    assert np.all(np.abs(d["rms_deg"] - a["rms_deg"]) <= RMS_TOL)
    tuned.destroy()


def test_device_traces_equal_host_traces(ctx):
    w = W.uneven10k(B=5)
    items = oracle_inputs(w)
    kw = dict(candidates=22 * 20, iterations=5, init_opc=centres(items))
    a = G.opmm_fit_batch(ctx, to_batch(items), **kw)
    b = G.opmm_fit_batch(ctx, to_batch(items, device="cuda"), **kw)
    for k in ("opc", "f", "rms_deg", "winner"):
        np.testing.assert_array_equal(a[k], b[k])


def test_calibrated_centres_used_when_none_given(ctx):
    """Without init_opc the GPU computes the calibrated box centre itself; the
    fit then matches an oracle fit centred on the oracle's calibration."""
    w = W.batch1024(B=3)
    items = oracle_inputs(w)
    batch = to_batch(items)
    res = G.opmm_fit_batch(ctx, batch, candidates=22 * 12, iterations=6,
                           pulse_init=G.OPMM_PULSE_CALIBRATED)
    for j, it in enumerate(items):
        ref = O.fit(it["pn"], it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"], 12, 6,
                    sac_index=j)
        assert abs(res["rms_deg"][j] - ref["rms"]) <= RMS_TOL


def test_edge_windows(ctx):
    """A one-sample window, a window that ends at onset, zero amplitude."""
    y1 = np.array([0.3], np.float32)
    y2 = np.linspace(0, 1, 12).astype(np.float32)
    y3 = (0.01 * np.sin(np.arange(80))).astype(np.float32)
    batch = G.make_batch([y1, y2, y3], [1000.0] * 3, [0, 11, 10], [0.0, 0.0, 2.0], [5.0, 8.0, 2.0],
                         [32.0, 38.6, 21.0])
    pc = np.stack([O.nominal_table1(d) for d in (32.0, 38.6, 21.0)]).astype(np.float32)
    res = G.opmm_fit_batch(ctx, batch, candidates=44, iterations=4, init_opc=pc)
    for j, (y, on, t0, tf) in enumerate([(y1, 0, 0.0, 5.0), (y2, 11, 0.0, 8.0), (y3, 10, 2.0, 2.0)]):
        ref = O.fit(pc[j].astype(np.float64), len(y), 1000.0, on, t0, tf, y.astype(np.float64), 2, 4,
                    sac_index=j)
        assert abs(res["rms_deg"][j] - ref["rms"]) <= RMS_TOL


@pytest.mark.parametrize("bad", ["L0", "onset", "fs", "box", "cand", "opc", "dur"])
def test_invalid_arguments_are_rejected(ctx, bad):
    y = np.zeros(50, np.float32)
    L, on, fs, lo, cand = 50, 5, 1000.0, 0.5, 44
    pc = O.nominal_table1(30.0).astype(np.float32)[None, :]
    dur = 30.0
    if bad == "L0":
        L = 0
    elif bad == "onset":
        on = 50
    elif bad == "fs":
        fs = -1.0
    elif bad == "box":
        lo = 1.5
    elif bad == "cand":
        cand = 21
    elif bad == "opc":
        pc = pc.copy()
        pc[0, 9] = -1.0
    elif bad == "dur":
        dur = 4.0
        pc = None
    batch = G.make_batch([y], [fs], [on], [0.0], [5.0], [dur], n_samples=[L])
    with pytest.raises(G.OpmmError) as e:
        G.opmm_fit_batch(ctx, batch, candidates=cand, iterations=2, box_lo=lo, init_opc=pc)
    assert e.value.code == G.OPMM_EINVAL


def test_empty_calls(ctx):
    """An empty batch to fit is OPMM_EINVAL; zero trajectories to simulate,
    candidates to score or centres to compute are no-ops that succeed."""
    import ctypes
    lib = G.load_library()
    o, _ = G.fit_opts(candidates=44, iterations=2)
    res = (G.opmm_fit_result * 1)()
    assert lib.opmm_fit_batch(ctx, None, 0, ctypes.byref(o), res) == G.OPMM_EINVAL
    batch = G.make_batch([np.zeros(50, np.float32)], [1000.0], [5], [0.0], [5.0], [30.0])
    descs, keep = batch.descriptors()
    assert lib.opmm_simulate(ctx, None, 0, descs, 1, None, None, None) == G.OPMM_OK
    assert lib.opmm_score(ctx, None, 0, descs, None) == G.OPMM_OK
    assert lib.opmm_nominal_opc(ctx, None, 0, G.OPMM_PULSE_CALIBRATED, None) == G.OPMM_OK


def test_every_search_variant_matches_oracle(ctx):
    """All launch-shape variants of the search kernel (simplices per block,
    register budget, register-lean schedule) run the same estimator; 70
    simplices fill a 64-simplex unit (waves of 704 candidates, two per
    evaluation thread) and leave a partial one."""
    w = W.uneven10k(B=4)
    items = oracle_inputs(w)
    S, T = 70, 5
    refs = [O.fit(it["pn"], it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"], S, T,
                  sac_index=j) for j, it in enumerate(items)]
    base = None
    try:
        for v in range(G.opmm_search_variants()):
            if G.opmm_search_variant_info(v)[1] != G.OPMM_MODEL_18:
                continue
            G.opmm_set_search_variant(ctx, v)
            res = G.opmm_fit_batch(ctx, to_batch(items), candidates=22 * S, iterations=T,
                                   init_opc=centres(items))
            for j in range(len(items)):
                assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL, (v, j)
            if base is None:
                base = res
            else:
                np.testing.assert_allclose(res["f"], base["f"], rtol=1e-4, atol=1e-7)
    finally:
        G.opmm_set_search_variant(ctx, -1)


@pytest.mark.parametrize("name", ["batch1024", "uneven10k"])
def test_full_size_plan_sampled_against_oracle(ctx, name):
    """The two batched workloads at full size (1,024 saccades at 65,536
    candidates x 30 iterations; 10,000 uneven saccades at 16,384 x 30) in the
    launch configuration the benchmark times: one autotuned, graph-captured
    plan over device-resident traces.  Over every saccade: status 0, the
    winner inside its box, the evaluation count inside the budget.  For 24
    seeded-sampled saccades the oracle recomputes the winner's FP64 error
    (equal to 1e-9 relative), the FP32 objective agrees with it within the
    trajectory bound, and the winner is no worse than the box centre (simplex
    0 starts there and Nelder-Mead never loses its best vertex).  For one
    sampled saccade the oracle runs the same estimator at the full budget
    (same starts: the Philox counter carries the batch index) and the fitted
    RMS agrees within 1e-3 deg."""
    w = W.batch1024() if name == "batch1024" else W.uneven10k()
    items = oracle_inputs_parallel(w)
    assert [it["i"] for it in items] == list(range(w.B))
    batch = to_batch(items, device="cuda")
    pc = centres(items)
    plan = G.Plan(ctx, batch, candidates=w.candidates, iterations=w.iterations, seed=w.seed, init_opc=pc)
    res = plan.execute()
    plan.destroy()
    S = w.candidates // 22
    assert np.all(res["status"] == 0)
    ev = res["evaluations"].astype(np.int64)
    assert np.all(ev >= S * 19) and np.all(ev <= S * (19 + 22 * w.iterations))
    ratio = res["opc"].astype(np.float64) / pc
    assert np.all(ratio >= 0.5 * (1 - 1e-5)) and np.all(ratio <= 2.0 * (1 + 1e-5))
    assert np.mean(res["rms_deg"] <= 0.1) >= 0.8
    rng = np.random.default_rng(20071)
    for j in rng.choice(w.B, 24, replace=False):
        it = items[j]
        p = res["opc"][j].astype(np.float64)
        mse, mae = O.errors(p, it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"])
        assert res["rms_deg"][j] == pytest.approx(math.sqrt(mse), rel=1e-9)
        assert res["l1_deg"][j] == pytest.approx(mae, rel=1e-9)
        assert abs(res["f"][j] - mse) <= f_tol(mse), (j, res["f"][j], mse)
        mse_c, _ = O.errors(it["pn"], it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"])
        assert mse <= mse_c + f_tol(mse_c)
    j = int(rng.integers(w.B))
    it = items[j]
    ref = O.fit(it["pn"], it["L"], it["fs"], it["onset"], it["th0"], it["thf"], it["y"], S, w.iterations,
                seed=w.seed, sac_index=j)
    assert abs(res["rms_deg"][j] - ref["rms"]) <= RMS_TOL, (j, res["rms_deg"][j], ref["rms"])


def test_full_candidate_budget_initial_vertices_match_oracle(ctx):
    """All 2,978 x 19 starting vertices of the 65,536-candidate budget (the
    Philox starts across the whole counter range): with no iterations the
    winner is the best of them, on the GPU as in the oracle."""
    w = W.batch1024(B=3)
    items = oracle_inputs(w)
    S = w.candidates // 22
    res, refs = _fit_both(ctx, items, S, 0)
    for j in range(len(items)):
        assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL
        bf = refs[j]["best_f_all"]
        assert bf[res["winner"][j]] - bf.min() <= f_tol(bf.min())


# In the wide box the plant's modes spread over up to five decades and its
# trajectories over three (a strong pulse against weak tension slopes can
# carry a candidate past 1,000 deg).  The FP32 path keeps the pulse-phase
# state as its deviation from the steady state the pulse heights would hold,
# which there can lie a hundred times beyond the trajectory, and its sample
# updates round at that scale: the bound is 1e-4 deg plus 2e-5 of the larger
# of the reference trajectory's largest |theta| and that distance
# (tests/test_gpu_wide_box.py checks it over 12,288 random candidates).
def wide_traj_tol(ref, p, it):
    scale = max(float(np.max(np.abs(ref))), pulse_equilibrium_distance(p, it["th0"], it["thf"]))
    return TRAJ_TOL + 2e-5 * scale


def test_wide_box_simulation_and_fit_match_oracle(ctx):
    """The paper-scale box [0.1x, 10x] (Fig. 4's rows sit on its bounds):
    stiff candidates integrate with refined substeps on both sides;
    trajectories match within wide_traj_tol and fits in that box match the
    oracle's RMS to 1e-3 deg."""
    w = W.uneven10k(B=4)
    items = oracle_inputs(w)
    rng = np.random.default_rng(11)
    for it in items:
        batch = to_batch([it])
        m = 64
        opc = (it["pn"] * np.exp(rng.uniform(np.log(0.1), np.log(10.0), (m, 18)))).astype(np.float32)
        corner = np.ones(18)
        corner[6], corner[9] = 10.0, 0.1                  # B_P 10x, J 0.1x: 8x the substeps
        opc[0] = (it["pn"] * corner).astype(np.float32)
        traj, offs = G.opmm_simulate(ctx, opc, batch, sac_index=np.zeros(m, np.int32))
        refined = 0
        for i in range(m):
            p = opc[i].astype(np.float64)
            if O.stiff(p, it["fs"]):
                continue
            refined += O.substeps(p, it["fs"]) > O.nsub(it["fs"])
            ref = O.simulate_rk4(p, it["L"], it["fs"], it["onset"], it["th0"], it["thf"])
            got = traj[offs[i]:offs[i] + it["L"]]
            assert np.max(np.abs(got - ref)) <= wide_traj_tol(ref, p, it), (i, np.max(np.abs(got - ref)),
                                                                     np.max(np.abs(ref)))
        assert refined >= 1
    res, refs = _fit_both(ctx, items[:3], 6, 6, box_lo=0.1, box_hi=10.0)
    for j in range(3):
        assert res["status"][j] == 0
        assert abs(res["rms_deg"][j] - refs[j]["rms"]) <= RMS_TOL, (j, res["rms_deg"][j], refs[j]["rms"])
        r = res["opc"][j] / centres(items[:3])[j]
        assert np.all(r >= 0.1 * (1 - 1e-5)) and np.all(r <= 10.0 * (1 + 1e-5))


@pytest.mark.parametrize("box", [(0.5, 2.0), (0.1, 10.0)])
def test_pulse_end_count_of_initial_vertices(ctx, box):
    """pulse_end_evals counts the evaluated candidates whose pulse ends inside
    the window (PW * fs < L - 1 - onset samples after onset, so that the
    interval holding the pulse end is integrated substep by substep).  With no
    iterations the evaluated candidates are exactly the starting vertices,
    which the host rebuilds from the oracle's Philox starts; candidates the
    stiffness rule rejects are not simulated and not counted.  A vertex whose
    pulse ends within 1e-5 of a sample boundary may fall either way in FP32."""
    lo, hi = box
    w = W.uneven10k(B=6)
    items = oracle_inputs(w)
    S, step = 40, 0.05
    res, _ = _fit_both(ctx, items, S, 0, box_lo=lo, box_hi=hi)
    for j, it in enumerate(items):
        ntot = it["L"] - 1 - it["onset"]
        want = near = 0
        for s in range(S):
            c = O.start_centre(18, s, j, 0, lo, hi)
            for v in range(19):
                u = c.copy()
                if v > 0:
                    u[v - 1] += step
                p = O.u_to_p(it["pn"], u, box_lo=lo, box_hi=hi)
                if ntot <= 0 or O.stiff(p, it["fs"]):
                    continue
                x = p[17] * it["fs"] * 1e-3
                want += x < ntot
                near += abs(x - ntot) <= 1e-5 * ntot
        assert res["evaluations"][j] == 19 * S
        assert abs(int(res["pulse_end_evals"][j]) - want) <= near, (j, res["pulse_end_evals"][j], want, near)
    res, _ = _fit_both(ctx, items, 8, 6)
    assert np.all(res["pulse_end_evals"] >= 0) and np.all(res["pulse_end_evals"] <= res["evaluations"])
    assert np.all(res["reserved"] == 0)
