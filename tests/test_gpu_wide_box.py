"""The paper-scale search box [0.1x, 10x] (Fig. 4's rows sit on its bounds) over
a large random sample: 2,048 OPC vectors drawn log-uniformly in the box for
each of two saccades at each sample rate (250, 500, 1000 Hz), simulated by the
library and by the oracle.

Tolerance.  The FP32 path keeps the pulse-phase state as its deviation from
the steady state the pulse heights would hold; in this box (strong pulses,
weak elasticities) that steady state can lie a hundred times beyond the
trajectory, and every FP32 sample update rounds at that scale, which the
FP64 oracle does not.  So a trajectory is held to 1e-4 deg plus 2e-5 of the
larger of its own largest excursion and that distance
(pulse_equilibrium_distance).  The test reports the largest error-to-bound
ratio and the largest error relative to that scale."""
import numpy as np
import pytest

import oracle as O
import paper_2007_09884_gb300 as G
import workloads as W
from _support import oracle_inputs, pulse_equilibrium_distance, to_batch

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-4
REL_TOL = 2e-5
PER_SACCADE = 2048


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = G.opmm_create(0)
    yield h
    G.opmm_destroy(h)


@pytest.mark.parametrize("fs", [250.0, 500.0, 1000.0])
def test_wide_box_trajectories_over_a_large_sample(ctx, fs):
    w = W.uneven10k(B=96)
    picks = [i for i in np.argsort(-w.L) if float(w.fs[i]) == fs][:2]
    items = oracle_inputs(w, idx=picks)
    rng = np.random.default_rng(int(fs))
    worst, worst_rel, refined, stiff, n = 0.0, 0.0, 0, 0, 0
    for it in items:
        opc = (it["pn"] * np.exp(rng.uniform(np.log(0.1), np.log(10.0), (PER_SACCADE, 18)))).astype(np.float32)
        traj, offs = G.opmm_simulate(ctx, opc, to_batch([it]), sac_index=np.zeros(PER_SACCADE, np.int32))
        for i in range(PER_SACCADE):
            p = opc[i].astype(np.float64)
            if O.stiff(p, fs):
                stiff += 1
                continue
            refined += O.substeps(p, fs) > O.nsub(fs)
            ref = O.simulate_rk4(p, it["L"], fs, it["onset"], it["th0"], it["thf"])
            got = traj[offs[i]:offs[i] + it["L"]].astype(np.float64)
            scale = max(float(np.max(np.abs(ref))), pulse_equilibrium_distance(p, it["th0"], it["thf"]))
            err = float(np.max(np.abs(got - ref)))
            worst = max(worst, err / (TRAJ_TOL + REL_TOL * scale))
            worst_rel = max(worst_rel, err / max(scale, 1e-12))
            n += 1
    print(f"fs {fs:.0f} Hz: {n} trajectories ({refined} with refined substeps, {stiff} too stiff), "
          f"largest error / bound {worst:.3f}, largest error / scale {worst_rel:.2e}")
    assert n >= PER_SACCADE
    assert refined >= 1
    assert worst <= 1.0
