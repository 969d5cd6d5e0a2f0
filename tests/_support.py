"""Test helpers: turn seeded workloads into oracle-generated traces and into
batches for the CUDA library (each side simulates with its own code; the GPU
side only ever receives what the oracle generated here)."""
import numpy as np

import oracle as O
import paper_2007_09884_gb300 as G


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def oracle_inputs(w, idx=None, noise=True):
    """Per saccade: box centre pn (float32-exact), hidden OPC, clean and
    recorded trace (float32-exact) for the oracle and the GPU alike."""
    idx = range(w.B) if idx is None else idx
    out = []
    for i in idx:
        A, D = float(w.amplitude[i]), float(w.dur_ms[i])
        pn = f32(O.nominal_opc(A, D, calibrated=w.calibrated_pulse))
        ph = f32(pn * w.mult[i])
        L, fs, on = int(w.L[i]), float(w.fs[i]), int(w.onset[i])
        th0, thf = float(w.theta0[i]), float(w.thetaf[i])
        clean = O.simulate_rk4(ph, L, fs, on, th0, thf)
        y = f32(clean + (w.noise[i] if noise else 0.0))
        out.append(dict(i=i, pn=pn, ph=ph, clean=clean, y=y, L=L, fs=fs, onset=on, th0=th0,
                        thf=thf, dur=D, A=A))
    return out


def to_batch(items, device=None):
    traces = [np.asarray(it["y"], dtype=np.float32) for it in items]
    if device is not None:
        import torch
        packed = np.zeros(sum((len(t) + 3) // 4 * 4 for t in traces), dtype=np.float32)
        offs, o = [], 0
        for t in traces:
            packed[o:o + len(t)] = t
            offs.append(o)
            o += (len(t) + 3) // 4 * 4
        tens = torch.from_numpy(packed).to(device)
        return G.make_batch(tens, [it["fs"] for it in items], [it["onset"] for it in items],
                            [it["th0"] for it in items], [it["thf"] for it in items],
                            [it["dur"] for it in items], n_samples=[it["L"] for it in items],
                            offsets=offs)
    return G.make_batch(traces, [it["fs"] for it in items], [it["onset"] for it in items],
                        [it["th0"] for it in items], [it["thf"] for it in items],
                        [it["dur"] for it in items])


def centres(items):
    return np.stack([it["pn"] for it in items]).astype(np.float32)


def _oracle_chunk(args):
    w, idx = args
    items = oracle_inputs(w)
    for it, i in zip(items, idx):
        it["i"] = int(i)
    return items


def oracle_inputs_parallel(w, procs=None):
    """oracle_inputs over a whole workload in a pool of spawned processes (the
    oracle's traces of 10,000 saccades take minutes on one core).  Spawned, so
    that a CUDA context already open in this process is never forked."""
    import multiprocessing as mp
    import os
    procs = procs or min(16, os.cpu_count() or 1)
    chunks = [c for c in np.array_split(np.arange(w.B), procs * 4) if len(c)]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_oracle_chunk, [(w.subset(c), c) for c in chunks])
    return [it for part in parts for it in part]


def pulse_equilibrium_distance(p, th0, thf):
    """|theta_eq - theta_0| in the saccade's positive frame, where theta_eq is
    the plant's steady state under the pulse heights held (the closed form
    pinned by the oracle tests: (a_g F_a - a_n F_n) / (K_P + a_g K_LT_AG +
    a_n K_LT_ANT), a = K_SE / (K_SE + K_LT), K_P = N_C_AG + N_C_ANT).  The
    FP32 path keeps the pulse-phase state as its deviation from that steady
    state, so this is the scale its rounding acts on."""
    p = np.asarray(p, dtype=np.float64)
    ag = p[0] / (p[0] + p[2])
    an = p[1] / (p[1] + p[3])
    th_eq = (ag * p[15] - an * p[16]) / (p[4] + p[5] + ag * p[2] + an * p[3])
    sign = -1.0 if thf < th0 else 1.0
    return abs(th_eq - sign * th0)
