"""Benchmark: batched OPMM estimation on GB300.

One step = one complete fit of the workload's batch (trace gather, box centres,
persistent parallel Nelder-Mead search, FP64 check), every row of the hot path.
Default workload: 1,024 synthetic saccades, 65,536 candidates x 30 iterations
each (the plain batched-search configuration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch1024|uneven10k|single10]
  python bench.py --workload surrogate   # plain vs surrogate-seeded search, 10,000 uneven saccades
  python bench.py --workload serve       # Poisson arrivals, p50/p99 latency, plain vs seeded
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

At N=1 the default line also carries:
  uneven10k  the 10,000-saccade uneven workload (250/500/1000 Hz, 16,384 x 30)
             through an autotuned graph-captured plan: candidate sims/s, the
             search kernel's FP32 roofline fraction, the autotuner's choice;
  surrogate  the learned network trained on 10 M generated saccades, then
             saccades fitted/s at <= 0.1 deg RMS on the uneven workload for
             the plain search and for the seeded search with plain fallback;
  serve      the request loop under 1 s of Poisson arrivals at 1k, 10k and
             50k/s, plain and seeded: p50/p99 latency, throughput, refusals;
  single10   the single 10 deg saccade (4,096 x 20) fitted on the GPU and,
             in the CPU-baseline leg, by the oracle: seconds and RMS;
  refine, ivt  the refinement after the search and the I-VT front end.

Prints one JSON line (rank 0).  value = candidate OPC simulations per second
over the whole job (all ranks), inputs resident in HBM; e2e = the same metric
through the C ABI with host buffers (H2D of traces and D2H of results inside
the timed region).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "OPC candidate sims/s (% FP32 peak); saccades fitted/s at <=0.1 deg RMS; p99 latency"
FP32_LANES_PER_SM = 128
RESULT_BYTES = 120


# ------------------------------------------------------------------ algorithmic work
def pow_products(n: int) -> int:
    """Matrix products of the binary powering of the RK4 step matrix."""
    if n <= 1:
        return 0
    return (n.bit_length() - 1) + (bin(n).count("1") - 1)


def flops_per_sim(L: int, onset: int, nsub: int) -> int:
    """Algorithmic FP32 FLOPs of one candidate simulation + score in the
    propagator formulation (FMA = 2): parameter map and stiffness guard (46),
    plant coefficients (24), single-step RK4 increment matrices of both phases
    (560), binary powering to one sample interval (332 per product),
    equilibria (68), finish (2), and per integrated sample a 6x6 block update
    plus the residual term (55).  A candidate whose pulse ends inside the
    window adds pulse_end_flops(nsub) on top (counted per candidate by the
    kernel).  Candidates refined to a finer substep are credited at the base
    substep (their extra work is not counted)."""
    n_int = max(0, L - 1 - onset)
    return 46 + 24 + 560 + 332 * pow_products(nsub) + 68 + 2 + 55 * n_int


def pulse_end_flops(nsub: int) -> int:
    """Extra FLOPs of the sample interval that holds the pulse end, over the
    52 of the one-sample update already counted for it: nsub - 1 single-substep
    block updates (52 each), two RK4 steps around the switch (4 levels of the
    A-apply, 19, plus 6 FMAs, and 3 for the level coefficients: 127 each), the
    two split step lengths (2) and the equilibrium shift (6)."""
    return 52 * (nsub - 1) + 2 * 127 + 2 + 6 - 52


def rk4_stage_flops_per_sim(L: int, nsub: int) -> int:
    """Same trajectory integrated stage by stage (168 FLOP per RK4 substep)."""
    return 168 * max(0, L - 1) * nsub


def nsub_for(fs: float) -> int:
    return max(1, int(math.floor(1.0e4 / fs + 0.5)))


# ------------------------------------------------------------------ peaks / clocks
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"opmm_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return parse_clock_samples(f)


def parse_clock_samples(lines):
    """Summary of nvidia-smi samples (the ClockSampler fields, csv, no header,
    no units): median SM clock, the maximum SM clock, and the throttle reasons
    seen active in any sample."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax = float(parts[2])
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup(n_gpus: int):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def dist_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ workloads
def make_workload(name: str, rank: int, quick: bool, saccades: int = 0):
    if name == "batch1024":
        w = W.batch1024(B=saccades or (64 if quick else 1024))
    elif name == "uneven10k":
        w = W.uneven10k(B=saccades or (256 if quick else 10000))
    elif name == "single10":
        w = W.single10()
    else:
        raise SystemExit(f"unknown workload {name}")
    if rank > 0 and name != "single10":
        # weak scaling: every rank fits its own batch of the same size
        g = W.batch1024 if name == "batch1024" else W.uneven10k
        full = g(B=w.B * (rank + 1))
        w = full.subset(np.arange(w.B * rank, w.B * (rank + 1)))
    return w


def workload_config(w, scaling_note: str, coords: int = 18):
    """coords: search coordinates, 18 (the OPC entries) or 9 (the 9-parameter
    model of Sec. 2.2.2, fitted to the same traces)."""
    return {"workload": w.name + ("" if coords == 18 else "_9p"), "saccades": int(w.B),
            "candidates_per_iteration": int(w.candidates), "iterations": int(w.iterations),
            "search_coordinates": int(coords), "simplices_per_saccade": int(w.candidates // (coords + 4)),
            "sample_rates_hz": sorted({float(x) for x in w.fs}),
            "window_samples": [int(w.L.min()), int(w.L.max())],
            "pulse_init": "calibrated" if w.calibrated_pulse else "table1",
            "l2": scaling_note}


# ------------------------------------------------------------------ our arm
def gpu_inputs(G, ctx, w):
    """Traces synthesised on the GPU by the library itself: hidden OPC =
    centre x multiplier, trajectory by opmm_simulate, plus the seeded noise."""
    n = w.B
    descs = G.make_batch([np.zeros(int(L), np.float32) for L in w.L], w.fs, w.onset, w.theta0,
                         w.thetaf, w.dur_ms)
    pulse = G.OPMM_PULSE_CALIBRATED if w.calibrated_pulse else G.OPMM_PULSE_TABLE1
    centre = G.opmm_nominal_opc(ctx, descs, pulse)
    hidden = (centre.astype(np.float64) * w.mult).astype(np.float32)
    traj, offs = G.opmm_simulate(ctx, hidden, descs)
    traces = []
    for i in range(n):
        L = int(w.L[i])
        traces.append((traj[offs[i]:offs[i] + L].astype(np.float64) + w.noise[i]).astype(np.float32))
    return traces, pulse


def packed(traces):
    offs, o = [], 0
    for t in traces:
        offs.append(o)
        o += (len(t) + 3) // 4 * 4
    buf = np.zeros(o, np.float32)
    for t, of in zip(traces, offs):
        buf[of:of + len(t)] = t
    return buf, np.array(offs, np.int64)


def profile_traffic(kernel_src_hash: str):
    """DRAM bytes per search launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "search_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_sha256") == kernel_src_hash:
            return d
    except Exception:
        pass
    return None


def source_code_digest(texts):
    """sha256 of source texts with their // comments, trailing blanks and
    blank lines removed: a comment edit leaves it unchanged, any code edit
    changes it."""
    h = hashlib.sha256()
    for t in texts:
        lines = (ln.split("//", 1)[0].rstrip() for ln in t.splitlines())
        h.update("\n".join(ln for ln in lines if ln).encode())
        h.update(b"\0")
    return h.hexdigest()


def kernel_hash():
    """Digest of the search kernel's sources (the key of the committed DRAM
    traffic record)."""
    texts = []
    for f in ("kernels.cu", "plant.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2007_09884_gb300", "csrc", f), encoding="utf-8") as fh:
            texts.append(fh.read())
    return source_code_digest(texts)


def search_flops(w, r):
    """Algorithmic FLOPs of one search over workload w with results r (the
    per-saccade evaluation and pulse-end counts), and the same work counted
    as stage-by-stage RK4."""
    flops = 0.0
    rk4_eq = 0.0
    for i in range(w.B):
        nsub = nsub_for(float(w.fs[i]))
        e = float(r["evaluations"][i])
        flops += e * flops_per_sim(int(w.L[i]), int(w.onset[i]), nsub)
        flops += float(r["pulse_end_evals"][i]) * pulse_end_flops(nsub)
        rk4_eq += e * rk4_stage_flops_per_sim(int(w.L[i]), nsub)
    return flops, rk4_eq


def fp32_peak_tflops(local, clk=None):
    import torch
    props = torch.cuda.get_device_properties(local)
    mp = measured_peaks()
    sm_max = (mp or {}).get("sm_max_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * float(sm_max) * 1e6 / 1e12
    return peak, f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (of nominal max clock)"


def uneven_measure(G, ctx, local, quick=False, steps=2):
    """The uneven workload (10,000 saccades at 250/500/1000 Hz, both
    directions, 1-40 deg, 40-400 samples, 16,384 candidates x 30 iterations):
    one autotuned, graph-captured plan over device-resident traces, one
    warm-up execute, then `steps` timed executes with L2 flushed before each.
    Candidate simulations per second over the whole execute, and the search
    kernel's FLOP rate (same accounting as the default line) against the FP32
    peak."""
    import torch
    w = W.uneven10k(B=512 if quick else 10000)
    traces, pulse = gpu_inputs(G, ctx, w)
    buf, offs = packed(traces)
    dev = torch.from_numpy(buf).cuda()
    batch = G.make_batch(dev, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms, n_samples=w.L, offsets=offs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = G.Plan(ctx, batch, candidates=w.candidates, iterations=w.iterations, seed=w.seed, pulse_init=pulse)
    plan_s = time.perf_counter() - t0
    plan.execute_raw()
    flush = torch.empty((256 << 20) // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    step_ms, search_ms = [], []
    res = None
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = plan.execute_raw()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        search_ms.append(plan.last_search_ms())
    r = G.results_to_numpy(res)
    info, probes = plan.info(), plan.tuning()
    plan.destroy()
    evals = float(np.sum(r["evaluations"].astype(np.float64)))
    flops, _ = search_flops(w, r)
    mean_step, mean_search = statistics.mean(step_ms), statistics.mean(search_ms)
    peak, basis = fp32_peak_tflops(local)
    achieved = flops / (mean_search * 1e-3) / 1e12
    ok = (r["rms_deg"] <= 0.1) & (r["status"] == 0)
    return {"workload": w.name, "saccades": int(w.B), "candidates_per_iteration": int(w.candidates),
            "iterations": int(w.iterations), "sample_rates_hz": sorted({float(x) for x in w.fs}),
            "window_samples": [int(w.L.min()), int(w.L.max())], "timed_steps": steps,
            "candidate_sims_per_s": evals / (mean_step * 1e-3), "step_ms": mean_step, "search_ms": mean_search,
            "saccades_fitted_per_s_at_0p1deg": float(ok.sum()) / (mean_step * 1e-3),
            "fraction_fitted_at_0p1deg": float(ok.mean()), "median_rms_deg": float(np.median(r["rms_deg"])),
            "roofline": {"bound": "alu", "kernel": "k_search", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "peak_basis": basis},
            "launch_shape": info, "autotuner_probes": probes, "plan_build_s": plan_s,
            "l2": "L2 flushed (256 MB write) before every timed execute"}


def run_ours(args, ws, rank, local):
    import torch
    import paper_2007_09884_gb300 as G

    torch.cuda.set_device(local)
    w = make_workload(args.workload, rank, args.quick, args.saccades)
    ctx = G.opmm_create(local)
    stream = torch.cuda.current_stream()
    G.opmm_set_stream(ctx, stream.cuda_stream)
    traces, pulse = gpu_inputs(G, ctx, w)
    buf, offs = packed(traces)
    dev = torch.from_numpy(buf).cuda()
    batch_dev = G.make_batch(dev, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms, n_samples=w.L, offsets=offs)
    opts = dict(candidates=w.candidates, iterations=w.iterations, seed=w.seed, pulse_init=pulse, model=args.model)
    plan = G.Plan(ctx, batch_dev, **opts)
    info = plan.info()
    info["autotuner_probes"] = plan.tuning()
    for _ in range(args.warmup):
        plan.execute_raw()
    torch.cuda.synchronize()

    l2_bytes = 256 << 20
    flush = torch.empty(l2_bytes // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(torch.cuda.current_device())
    step_ms, search_ms = [], []
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    res = None
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = plan.execute_raw()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        search_ms.append(plan.last_search_ms())
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(ws)
    r = G.results_to_numpy(res)
    evals_rank = float(np.sum(r["evaluations"].astype(np.float64)))
    fitted_rank = float(np.sum((r["rms_deg"] <= 0.1) & (r["status"] == 0)))
    total_ms = sum(step_ms)
    t_max = dist_max(total_ms, ws)
    evals_all = dist_sum(evals_rank, ws) * args.steps
    fitted_all = dist_sum(fitted_rank, ws) * args.steps
    value = evals_all / (t_max * 1e-3)

    # algorithmic FLOPs of this rank's search launch
    flops, rk4_eq = search_flops(w, r)
    mean_search_ms = statistics.mean(search_ms)
    if not mean_search_ms > 0.0:
        raise SystemExit("search kernel events returned no time")
    achieved = flops / (mean_search_ms * 1e-3) / 1e12
    peak, peak_basis = fp32_peak_tflops(local, clk)
    prof = profile_traffic(kernel_hash())

    # end to end through the C ABI with host buffers
    batch_host = G.make_batch(traces, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms)
    plan_h = G.Plan(ctx, batch_host, **opts)
    for _ in range(max(1, min(args.warmup, 2))):
        plan_h.execute_raw()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rh = plan_h.execute_raw()
    e2e_s = time.perf_counter() - t0
    e2e_s = dist_max(e2e_s, ws)
    rh = G.results_to_numpy(rh)
    e2e_value = dist_sum(float(np.sum(rh["evaluations"].astype(np.float64))), ws) * args.steps / e2e_s
    h2d = int(buf.nbytes)
    d2h = int(w.B * RESULT_BYTES + 4)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "candidate sims/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded OPMM-simulated saccades + Gaussian noise; no dataset)",
        "config": workload_config(w, "L2 flushed (256 MB write) before every timed step", args.model),
        "impl": "ours",
        "saccades_fitted_per_s_at_0p1deg": fitted_all / (t_max * 1e-3),
        "fraction_fitted_at_0p1deg": fitted_rank / w.B,
        "median_rms_deg": float(np.median(r["rms_deg"])),
        "step_ms_p50": statistics.median(step_ms),
        "step_ms_p99": float(np.percentile(step_ms, 99)),
        "search_ms_mean": mean_search_ms,
        "rk4_stage_equivalent_tflops": rk4_eq / (mean_search_ms * 1e-3) / 1e12,
        "launch_shape": info,
        "roofline": {"bound": "alu", "kernel": "k_search (persistent Nelder-Mead + plant)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "peak_basis": peak_basis,
                     "traffic": (prof["dram_bytes_per_launch"] if prof else None),
                     "traffic_basis": (prof.get("basis") if prof else "no ncu capture of the current kernel")},
        "e2e": {"value": e2e_value, "unit": "candidate sims/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(info["kernels_per_execute"]) * args.steps,
        "clocks": clk,
    }
    plan.destroy()
    plan_h.destroy()
    if rank == 0 and ws == 1 and not args.no_refine:
        out["refine"] = refine_after_search(G, ctx, batch_dev, r, args, pulse, w)
    if rank == 0 and ws == 1 and not args.no_ivt:
        out["ivt"] = ivt_measure(G, ctx, 1 << (22 if args.quick else 26), with_oracle=not args.no_cpu_baseline)
    headline = rank == 0 and ws == 1 and args.workload == "batch1024" and args.model == 18
    if headline and not args.no_uneven:
        out["uneven10k"] = uneven_measure(G, ctx, local, args.quick)
    if headline and not args.no_surrogate:
        out["surrogate"] = surrogate_compare(G, ctx, args.quick)
    if headline and not args.no_serve:
        out["serve"] = serve_measure(G, ctx, args.rates, seconds=args.serve_seconds_line,
                                     trained=not args.no_surrogate, quick=args.quick)
    if headline:
        out["single10"] = single10_measure(G, ctx)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget, model=args.model)
        if "single10" in out:
            out["single10"]["oracle"] = cpu_baseline_single10(out["single10"])
    G.opmm_destroy(ctx)
    return out


def refine_after_search(G, ctx, batch, r, args, pulse, w=None, iterations=10):
    """Levenberg-Marquardt refinement (opmm_refine_batch) of the timed step's
    search results on the same saccades: wall time of the call (staging,
    refinement kernel, FP64 check, results), trajectories simulated, and the
    fit before and after; beside it the oracle's refinement of the first few
    of the same saccades from the same starts on one host core."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = G.opmm_refine_batch(ctx, batch, r["opc"], iterations=iterations, model=args.model, pulse_init=pulse)
    dt = time.perf_counter() - t0
    sims = float(np.sum(ref["evaluations"].astype(np.float64)))
    ok0 = (r["status"] == 0) & (r["rms_deg"] <= 0.1)
    ok1 = (ref["status"] == 0) & (ref["rms_deg"] <= 0.1)
    out = {"iterations": iterations, "seconds": dt, "saccades_per_s": len(ref["status"]) / dt,
           "trajectories_per_s": sims / dt, "accepted_steps_mean": float(np.mean(ref["iterations_run"])),
           "median_rms_deg_before": float(np.median(r["rms_deg"])),
           "median_rms_deg_after": float(np.median(ref["rms_deg"])),
           "fraction_fitted_at_0p1deg_before": float(np.mean(ok0)),
           "fraction_fitted_at_0p1deg_after": float(np.mean(ok1))}
    if w is not None and not args.no_cpu_baseline:
        import oracle as O
        nb = min(6, w.B)
        t0 = time.perf_counter()
        osims = 0
        for i in range(nb):
            A, D = float(w.amplitude[i]), float(w.dur_ms[i])
            pn = np.float32(O.nominal_opc(A, D, calibrated=w.calibrated_pulse)).astype(np.float64)
            ph = np.float32(pn * w.mult[i]).astype(np.float64)
            L, fs, on = int(w.L[i]), float(w.fs[i]), int(w.onset[i])
            th0, thf = float(w.theta0[i]), float(w.thetaf[i])
            y = np.float32(O.simulate_rk4(ph, L, fs, on, th0, thf) + w.noise[i]).astype(np.float64)
            coords = list(range(18)) if args.model == 18 else [0, 2, 7, 8, 6, 4, 5, 9, 14]
            u0 = np.log(r["opc"][i].astype(np.float64)[coords] / pn[coords])
            o = O.refine(pn, L, fs, on, th0, thf, y, u0, iterations, model=args.model)
            osims += o["evaluations"]
        odt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": nb / odt, "unit": "saccades refined/s", "cores": 1, "kind": "oracle",
                               "sample": f"saccades 0-{nb - 1} of {w.name}, {iterations} iterations from the same "
                                         f"starts ({osims} FP64 trajectories, {odt:.2f} s)"}
    return out


def ivt_measure(G, ctx, n, reps=5, with_oracle=True):
    """The I-VT front end (opmm_detect_saccades) on device-resident raw
    streams of n samples at 1 kHz (larger than L2), each call timed whole on
    the host: a stream with saccades (two passes over it, the per-run pass,
    the event copy) and the same length of fixation alone (the scan passes
    with nothing to report: the front end's HBM rate).  Beside it the
    reference definition (numpy, one core) on a 4 M-sample slice."""
    import torch

    def timed(dev):
        for _ in range(2):
            ev = G.opmm_detect_saccades(ctx, dev, 1000.0)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            ev = G.opmm_detect_saccades(ctx, dev, 1000.0)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts), ev

    x, planted = W.raw_stream(n)
    t, ev = timed(torch.from_numpy(x).cuda())
    quiet = (np.random.default_rng(3).normal(0.0, 0.005, n) + 5.0).astype(np.float32)
    tq, evq = timed(torch.from_numpy(quiet).cuda())
    mp = measured_peaks() or {}
    hbm = float(mp.get("hbm_gbs") or 6800.0)
    out = {"samples": n, "stream_bytes": 4 * n, "planted_saccades": len(planted), "saccades_kept": int(len(ev)),
           "seconds_median": t, "samples_per_s": n / t,
           "fixation_only": {"seconds_median": tq, "samples_per_s": n / tq, "stream_gbs": 4.0 * n / tq / 1e9,
                             "frac_of_hbm_peak": 4.0 * n / tq / 1e9 / hbm, "hbm_peak_gbs": hbm,
                             "events": int(len(evq))},
           "note": "whole calls timed on the host; the fixation-only stream has no run to report, so its call is the "
                   "scan over the stream plus one small copy"}
    if with_oracle:
        from oracle.ivt import ivt
        m = min(n, 1 << 22)
        t0 = time.perf_counter()
        ivt(x[:m], 1000.0)
        odt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": m / odt, "unit": "samples/s", "cores": 1, "kind": "oracle",
                               "sample": f"first {m} samples of the same stream ({odt:.2f} s)"}
    return out


def run_ivt(args):
    """The I-VT front end alone (--workload ivt): one JSON line for a raw
    stream of 2^26 samples (2^22 with --quick)."""
    import torch
    import paper_2007_09884_gb300 as G
    torch.cuda.set_device(0)
    ctx = G.opmm_create(0)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    r = ivt_measure(G, ctx, 1 << (22 if args.quick else 26), reps=max(3, args.steps),
                    with_oracle=not args.no_cpu_baseline)
    clk = clocks.stop()
    G.opmm_destroy(ctx)
    out = {"metric": "raw stream samples/s through I-VT detection (saccade windows out)", "value": r["samples_per_s"],
           "unit": "samples/s", "n_gpus": 1, "steps": max(3, args.steps), "warmup": 2,
           "ms_per_step": 1e3 * r["seconds_median"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic raw stream (workloads.raw_stream)",
           "config": {"workload": "ivt_stream", "samples": r["samples"], "sample_rate_hz": 1000.0,
                      "l2": "stream larger than L2"},
           "impl": "ours", "ivt": r, "clocks": clk}
    if "cpu_baseline" in r:
        out["cpu_baseline"] = r["cpu_baseline"]
    return out


def run_gemm(args):
    """The surrogate's tensor-core GEMM (opmm_gemm_bf16: tcgen05, TMEM
    accumulator, TMA ring) alone (--workload gemm): D = A.B^T in BF16 with FP32
    accumulation at the surrogate's layer shape (4,096 x 512 x 512) and at a
    large square shape, each call timed with CUDA events on the library's
    stream (the call also clears and reads back the error word), against the
    measured BF16 peak; cuBLAS (torch.matmul) on the same shapes beside it."""
    import torch
    import paper_2007_09884_gb300 as G
    torch.cuda.set_device(0)
    ctx = G.opmm_create(0)
    stream = torch.cuda.current_stream()
    G.opmm_set_stream(ctx, stream.cuda_stream)
    mp = measured_peaks() or {}
    peak = float(mp.get("bf16_tflops") or 1900.0)
    rows = []
    g = torch.Generator(device="cuda").manual_seed(0)
    for (M, N, K) in ((4096, 512, 512), (8192, 8192, 8192)):
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        D = torch.empty(M, N, device="cuda", dtype=torch.float32)
        reps = max(3, args.steps) * (20 if M * N * K < 1 << 32 else 2)
        for _ in range(3):
            G.opmm_gemm_bf16(ctx, A, Bm, out=D)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            G.opmm_gemm_bf16(ctx, A, Bm, out=D)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        ref = (A.float() @ Bm.float().t())
        err = float((D - ref).abs().max() / ref.abs().max())
        for _ in range(3):
            torch.matmul(A, Bm.t())
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            torch.matmul(A, Bm.t())
        e1.record(stream)
        torch.cuda.synchronize()
        ms_cublas = e0.elapsed_time(e1) / reps
        fl = 2.0 * M * N * K
        rows.append({"M": M, "N": N, "K": K, "ms": ms, "tflops": fl / ms / 1e9, "frac_of_bf16_peak": fl / ms / 1e9 / peak,
                     "max_rel_err_vs_fp32_product": err, "cublas_ms": ms_cublas, "cublas_tflops": fl / ms_cublas / 1e9})
    G.opmm_destroy(ctx)
    big = rows[-1]
    return {"metric": "BF16 tensor-core GEMM TFLOP/s (surrogate layer primitive)", "value": big["tflops"],
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": 3, "ms_per_step": big["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (normal random operands)", "config": {"workload": "gemm", "shapes": [r["M"] for r in rows]},
            "impl": "ours",
            "roofline": {"bound": "tensor", "achieved": big["tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": big["tflops"] / peak, "peak_basis": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)"},
            "rows": rows}


# ------------------------------------------------------------------ serving
def serve_run(G, ctx, traces_desc, arrivals, fit, cfg):
    """Submit saccades at the given arrival times (s), collect every result;
    returns per-request latency (ms), RMS, and counts."""
    import threading
    G.opmm_serve_start(ctx, cfg, **fit)
    descs, keep = traces_desc.descriptors()
    n_desc = len(traces_desc)
    tickets, rejected = [], 0
    lock = threading.Lock()
    done = {"lat": [], "rms": [], "status": []}
    stop = {"flag": False}

    def collector():
        i = 0
        while True:
            with lock:
                have = i < len(tickets)
                t = tickets[i] if have else None
            if not have:
                if stop["flag"]:
                    break
                time.sleep(0.0005)
                continue
            rc, res, lat = G.opmm_serve_poll_raw(ctx, t, 2_000_000)
            if rc == G.OPMM_OK:
                done["lat"].append(lat / 1000.0)
                done["rms"].append(res["rms_deg"])
                done["status"].append(res["status"])
                i += 1
            elif rc == G.OPMM_ETIMEDOUT:
                continue
            else:
                i += 1

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    k = 0
    n = len(arrivals)
    while k < n:
        now = time.perf_counter() - t0
        while k < n and arrivals[k] <= now:
            rc, t = G.opmm_serve_submit_raw(ctx, descs[k % n_desc])
            if rc == G.OPMM_OK:
                with lock:
                    tickets.append(t)
            elif rc == G.OPMM_EBUSY:
                rejected += 1
            k += 1
        time.sleep(0.0002)
    t_submit_end = time.perf_counter() - t0
    stop["flag"] = True
    th.join()
    t_all = time.perf_counter() - t0
    stats = G.opmm_serve_stats_get(ctx)
    G.opmm_serve_stop(ctx)
    lat = np.array(done["lat"]) if done["lat"] else np.array([float("nan")])
    rms = np.array(done["rms"]) if done["rms"] else np.array([float("nan")])
    return {"offered": n, "completed": len(done["lat"]), "rejected": rejected,
            "duration_s": t_all, "submit_window_s": t_submit_end,
            "throughput_per_s": len(done["lat"]) / t_all,
            "fitted_per_s_at_0p1deg": float(np.sum(rms <= 0.1)) / t_all,
            "fraction_fitted_at_0p1deg": float(np.mean(rms <= 0.1)),
            "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
            "slots": stats["slots"], "rounds": stats["rounds"]}


# ------------------------------------------------------------------ learned surrogate
# 2,441 steps of 4,096 generated saccades = 10 M training samples
SURROGATE_SCHEDULE = [(800, 2e-3), (800, 1e-3), (500, 5e-4), (341, 2.5e-4)]
SEEDED_FIT = dict(candidates=1024, iterations=20, box_lo=0.95, box_hi=1.05, init_step=0.025)
# the plain search that re-fits the seeded search's misses (> 0.1 deg)
FALLBACK_FIT = dict(candidates=4096, iterations=30)
# Network arithmetic per training sample, as the training step performs it:
# forward 2 (4 x 512 x 512 + 18 x 512); backward: the output layer's weight
# gradient and dH3 (2 x 2 x 18 x 512), the four hidden weight gradients and
# the three error products of layers 3, 2, 1 (2 x 7 x 512 x 512; no error
# product is formed for the input layer)
MLP_TRAIN_FLOP_PER_SAMPLE = 2 * (4 * 512 * 512 + 18 * 512) + 2 * 2 * 18 * 512 + 2 * 7 * 512 * 512


def train_surrogate(G, ctx, quick=False):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G.opmm_surrogate_init(ctx, 1)
    base = 0
    last = None
    for steps, lr in (SURROGATE_SCHEDULE if not quick else [(100, 2e-3)]):
        last = G.opmm_surrogate_train(ctx, steps, batch=4096, lr=lr, weight_decay=1e-4, data_seed=7,
                                      sample_base=base)
        base += steps * 4096
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"samples": base, "seconds": dt, "final_loss_mean_last_50": float(np.mean(last[-50:])),
            "tflops_wall": base * MLP_TRAIN_FLOP_PER_SAMPLE / dt / 1e12}


def surrogate_compare(G, ctx, quick=False):
    """10,000 uneven saccades (250/500/1000 Hz, both directions, 1-40 deg,
    40-400 samples): plain search at 16,384 x 30 against the surrogate-seeded
    search at 1,024 x 20 in a +-5% box whose misses (> 0.1 deg) fall back to
    the plain search; each followed by the Levenberg-Marquardt refinement as
    variants; plus the network alone on 100,000 held-out saccades."""
    import torch
    training = train_surrogate(G, ctx, quick)
    w = W.uneven10k(B=512 if quick else 10000)
    traces, pulse = gpu_inputs(G, ctx, w)
    batch = G.make_batch(traces, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms)
    plain = dict(candidates=w.candidates, iterations=w.iterations, seed=w.seed, pulse_init=pulse)
    seeded = dict(SEEDED_FIT, seed=w.seed, pulse_init=pulse)
    warm = W.uneven10k(B=64, config_index=7)
    wt, _ = gpu_inputs(G, ctx, warm)
    wb = G.make_batch(wt, warm.fs, warm.onset, warm.theta0, warm.thetaf, warm.dur_ms)
    G.opmm_fit_batch(ctx, wb, **plain)
    G.opmm_fit_batch_seeded(ctx, wb, seeded, plain, 0.1)
    torch.cuda.synchronize()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    fallback = dict(FALLBACK_FIT, seed=w.seed, pulse_init=pulse)

    def row(r, t, nfb=None):
        ok = (r["rms_deg"] <= 0.1) & (r["status"] == 0)
        out = {"seconds": t, "fitted_per_s_at_0p1deg": float(ok.sum()) / t,
               "fraction_fitted_at_0p1deg": float(ok.mean()), "median_rms_deg": float(np.median(r["rms_deg"])),
               "evaluations_per_saccade": float(np.mean(r["evaluations"].astype(np.float64)))}
        if nfb is not None:
            out["fallbacks"] = int(nfb)
            out["kept_from_fallback"] = int(np.sum(r["source"] == G.OPMM_SOURCE_FALLBACK))
        return out

    rp, tp = timed(lambda: G.opmm_fit_batch(ctx, batch, **plain))
    plain_row = row(rp, tp)
    (rs, nfb), ts = timed(lambda: G.opmm_fit_batch_seeded(ctx, batch, seeded, fallback, 0.1))
    seeded_row = row(rs, ts, nfb)
    # the same with no fallback, with the full plain budget as fallback, and
    # with a box of +-10% instead of +-5%
    r1, t1 = timed(lambda: G.opmm_fit_batch(ctx, batch, use_surrogate=True, **seeded))
    (r2, n2), t2 = timed(lambda: G.opmm_fit_batch_seeded(ctx, batch, seeded, plain, 0.1))
    wide = dict(seeded, box_lo=0.9, box_hi=1.1, init_step=0.05)
    (r3, n3), t3 = timed(lambda: G.opmm_fit_batch_seeded(ctx, batch, wide, fallback, 0.1))
    # Levenberg-Marquardt refinement (10 iterations) of each search's results
    rpr, tpr = timed(lambda: G.opmm_refine_batch(ctx, batch, rp["opc"], iterations=10, pulse_init=pulse))
    rsr, tsr = timed(lambda: G.opmm_refine_batch(ctx, batch, rs["opc"], iterations=10, pulse_init=pulse))
    r1r, t1r = timed(lambda: G.opmm_refine_batch(ctx, batch, r1["opc"], iterations=10, pulse_init=pulse))
    variants = {"seeded_only": row(r1, t1), "seeded_full_budget_fallback": dict(row(r2, t2, n2), fallback=plain),
                "seeded_box_10pct": dict(row(r3, t3, n3), search=wide),
                "plain_then_refine": dict(row(rpr, tp + tpr), refine_seconds=tpr, refine_iterations=10),
                "seeded_with_fallback_then_refine": dict(row(rsr, ts + tsr), refine_seconds=tsr,
                                                         refine_iterations=10),
                "seeded_only_then_refine": dict(row(r1r, t1 + t1r), refine_seconds=t1r, refine_iterations=10)}

    # the network alone on held-out saccades (drawn by the numpy generator;
    # training draws its saccades on the device)
    h = W.uneven10k(B=2000 if quick else 100000, config_index=5)
    htr, _ = gpu_inputs(G, ctx, h)
    hb = G.make_batch(htr, h.fs, h.onset, h.theta0, h.thetaf, h.dur_ms)
    nominal = G.opmm_nominal_opc(ctx, hb, pulse)
    hidden = nominal.astype(np.float64) * h.mult
    (pred,), tpred = timed(lambda: (G.opmm_surrogate_predict(ctx, hb, pulse),))

    def traj_rms(opc):
        traj, offs = G.opmm_simulate(ctx, opc.astype(np.float32), hb)
        return np.array([math.sqrt(np.mean((traj[offs[i]:offs[i] + len(htr[i])] - htr[i]) ** 2))
                         for i in range(h.B)])

    # share of the log-OPC target variance the network explains (targets
    # y = ln(hidden / nominal) / 0.2, estimate ln(pred / nominal) / 0.2)
    yt = np.log(hidden / nominal.astype(np.float64))
    ye = np.log(pred.astype(np.float64) / nominal.astype(np.float64))
    ss_res = np.sum((yt - ye) ** 2, axis=0)
    ss_tot = np.sum((yt - yt.mean(axis=0)) ** 2, axis=0)
    held = {"saccades": int(h.B), "predict_seconds": tpred,
            "explained_variance_log_opc": float(1.0 - ss_res.sum() / ss_tot.sum()),
            "explained_variance_per_parameter": [float(x) for x in 1.0 - ss_res / ss_tot],
            "median_abs_log_error_nominal": float(np.median(np.abs(np.log(nominal / hidden)))),
            "median_abs_log_error_surrogate": float(np.median(np.abs(np.log(pred / hidden)))),
            "median_trace_rms_deg_nominal": float(np.median(traj_rms(nominal))),
            "median_trace_rms_deg_surrogate": float(np.median(traj_rms(pred)))}
    return {"workload": w.name, "saccades": int(w.B), "plain": dict(plain_row, search=plain),
            "seeded_with_fallback": dict(seeded_row, search=seeded, fallback=fallback, fallback_rms_deg=0.1),
            "fitted_per_s_ratio": seeded_row["fitted_per_s_at_0p1deg"] / plain_row["fitted_per_s_at_0p1deg"],
            "variants": variants,
            "training": training, "held_out": held}


def serve_measure(G, ctx, rates, seconds=1.0, trained=True, quick=False):
    """The request loop for about `seconds` of Poisson arrivals per rate,
    plain search (16,384 x 30) and surrogate-seeded search (1,024 x 20 in
    +-5%) on the same saccades (uneven distribution): p50/p99 latency from
    submit to result, throughput, refusals, share fitted to <= 0.1 deg.  The
    queue holds a quarter second of arrivals, so an overloaded plain search
    refuses the rest instead of building minutes of backlog."""
    if not trained:
        train_surrogate(G, ctx, quick)
    w = W.uneven10k(B=2048, config_index=4)
    traces, pulse = gpu_inputs(G, ctx, w)
    batch = G.make_batch(traces, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms)
    plain = dict(candidates=16384, iterations=30, seed=0, pulse_init=pulse)
    seeded = dict(SEEDED_FIT, seed=0, pulse_init=pulse, use_surrogate=True)
    rows = []
    for rate in rates:
        arr = W.poisson_arrivals(rate, seconds, seed=int(rate))
        for name, fit, ri in (("plain", plain, 10), ("surrogate", seeded, 5)):
            cfg = G.serve_opts(max_slots=4096, max_queue=max(1000, int(rate * 0.25)), max_samples=400,
                               round_iters=ri, max_admit_per_round=4096)
            r = serve_run(G, ctx, batch, arr, fit, cfg)
            r.update({"rate_per_s": rate, "search": name})
            rows.append(r)
    return {"workload": "serve (Poisson arrivals of single saccades, uneven distribution)",
            "seconds_of_arrivals_per_rate": seconds, "plain": plain,
            "surrogate": {k: v for k, v in seeded.items()}, "rows": rows}


_SINGLE10 = {}


def single10_measure(G, ctx):
    """The single 10 deg saccade (1 kHz, 150 samples, Table 1's 55 g pulse),
    4,096 candidates x 20 iterations: the GPU fit through opmm_fit_batch with
    host buffers, wall time after one warm-up call (plan, autotune)."""
    w = W.single10()
    traces, pulse = gpu_inputs(G, ctx, w)
    batch = G.make_batch(traces, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms)
    opts = dict(candidates=w.candidates, iterations=w.iterations, seed=w.seed, pulse_init=pulse)
    G.opmm_fit_batch(ctx, batch, **opts)
    t0 = time.perf_counter()
    r = G.opmm_fit_batch(ctx, batch, **opts)
    dt = time.perf_counter() - t0
    _SINGLE10.update(w=w, y=traces[0])
    return {"workload": w.name, "candidates_per_iteration": int(w.candidates), "iterations": int(w.iterations),
            "simplices": int(w.candidates // 22), "gpu_seconds": dt, "gpu_rms_deg": float(r["rms_deg"][0]),
            "gpu_evaluations": int(r["evaluations"][0]), "gpu_status": int(r["status"][0])}


def cpu_baseline_single10(g):
    """The oracle's full fit of the same saccade (same trace, same budget,
    same seed) on the host cores: seconds and RMS beside the GPU's."""
    import oracle as O
    w, y = _SINGLE10["w"], _SINGLE10["y"]
    A, D = float(w.amplitude[0]), float(w.dur_ms[0])
    pn = np.float32(O.nominal_opc(A, D, calibrated=w.calibrated_pulse)).astype(np.float64)
    nthreads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ro = O.fit(pn, int(w.L[0]), float(w.fs[0]), int(w.onset[0]), float(w.theta0[0]), float(w.thetaf[0]),
               np.asarray(y, np.float64), w.candidates // 22, w.iterations, seed=w.seed, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "rms_deg": ro["rms"], "cores": nthreads, "kind": "oracle (FP64)",
            "abs_rms_difference_deg": abs(ro["rms"] - g["gpu_rms_deg"]), "speedup_gpu": dt / g["gpu_seconds"]}


def run_surrogate(args):
    import paper_2007_09884_gb300 as G
    ctx = G.opmm_create(0)
    cmp_ = surrogate_compare(G, ctx, args.quick)
    G.opmm_destroy(ctx)
    s = cmp_["seeded_with_fallback"]
    return {"metric": "saccades fitted/s at <=0.1 deg RMS (surrogate-seeded search with plain fallback)",
            "value": s["fitted_per_s_at_0p1deg"], "unit": "saccades/s", "n_gpus": 1, "higher_is_better": True,
            "vs_baseline": None, "dtype": "f32 search, bf16 network", "data": "synthetic",
            "config": {"workload": cmp_["workload"], "saccades": cmp_["saccades"],
                       "l2": "inputs resident; one timed pass per arm"},
            "surrogate": cmp_}


def run_serve(args):
    import paper_2007_09884_gb300 as G
    ctx = G.opmm_create(0)
    w = W.uneven10k(B=2048, config_index=4)
    traces, pulse = gpu_inputs(G, ctx, w)
    batch = G.make_batch(traces, w.fs, w.onset, w.theta0, w.thetaf, w.dur_ms)
    training = train_surrogate(G, ctx)
    train_s, base = training["seconds"], training["samples"]
    plain = dict(candidates=16384, iterations=30, seed=0, pulse_init=pulse)
    seeded = dict(SEEDED_FIT, seed=0, pulse_init=pulse, use_surrogate=True)
    rows = []
    for rate in args.rates:
        arr = W.poisson_arrivals(rate, args.serve_seconds, seed=int(rate))
        for name, fit, ri in (("plain", plain, 10), ("surrogate", seeded, 5)):
            cfg = G.serve_opts(max_slots=args.serve_slots, max_queue=max(1000, int(rate * 2)), max_samples=400,
                               round_iters=ri, max_admit_per_round=4096)
            r = serve_run(G, ctx, batch, arr, fit, cfg)
            r.update({"rate_per_s": rate, "search": name})
            rows.append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    G.opmm_destroy(ctx)
    head = [r for r in rows if r["search"] == "surrogate"]
    best = max(head, key=lambda r: r["fitted_per_s_at_0p1deg"])
    return {"metric": "saccades fitted/s at <=0.1 deg RMS with p50/p99 fit latency (real-time serving)",
            "value": best["fitted_per_s_at_0p1deg"], "unit": "saccades/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic (Poisson arrivals)",
            "config": {"workload": "serve", "rates_per_s": args.rates, "seconds_per_rate": args.serve_seconds,
                       "plain": plain, "surrogate": {k: v for k, v in seeded.items()},
                       "surrogate_training_s": train_s, "surrogate_training_samples": base},
            "rows": rows}


# ------------------------------------------------------------------ oracle arm
def oracle_sample(w, budget_s: float, nthreads: int, model: int = 18):
    """Oracle fit of saccade 0 at the workload's full iteration cap on a
    bounded number of simplices, sized to about budget_s of host time, over
    the model's search coordinates (18, or 9)."""
    import oracle as O
    i = 0
    A, D = float(w.amplitude[i]), float(w.dur_ms[i])
    pn = np.float32(O.nominal_opc(A, D, calibrated=w.calibrated_pulse)).astype(np.float64)
    ph = np.float32(pn * w.mult[i]).astype(np.float64)
    L, fs, on = int(w.L[i]), float(w.fs[i]), int(w.onset[i])
    th0, thf = float(w.theta0[i]), float(w.thetaf[i])
    y = np.float32(O.simulate_rk4(ph, L, fs, on, th0, thf) + w.noise[i]).astype(np.float64)
    # probe: one simplex per thread, 2 iterations
    t0 = time.perf_counter()
    nv, nt = model + 1, model + 4
    O.fit(pn, L, fs, on, th0, thf, y, nthreads, 2, seed=w.seed, nthreads=nthreads, model=model)
    probe = time.perf_counter() - t0
    per_sim = probe / (nthreads * (nv + 2 * nt)) * nthreads      # wall seconds per sim per thread
    sims_per_simplex = nv + nt * w.iterations
    S = int(max(nthreads, min(w.candidates // nt, budget_s / (per_sim / nthreads * sims_per_simplex))))
    S = max(nthreads, (S // nthreads) * nthreads)
    t0 = time.perf_counter()
    r = O.fit(pn, L, fs, on, th0, thf, y, S, w.iterations, seed=w.seed, nthreads=nthreads, model=model)
    dt = time.perf_counter() - t0
    sims = S * nv + nt * float(np.sum(r["iters"]))
    return sims, dt, S


def cpu_baseline(w, budget_s=12.0, model=18):
    nthreads = os.cpu_count() or 1
    sims, dt, S = oracle_sample(w, budget_s, nthreads, model)
    return {"value": sims / dt, "unit": "candidate sims/s", "cores": nthreads, "kind": "oracle",
            "sample": f"saccade 0 of {w.name}: {S} of {w.candidates // (model + 4)} simplices x {w.iterations} "
                      f"iterations ({int(sims)} simulations, {dt:.1f} s, FP64 RK4 stages)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    w = make_workload(args.workload, 0, args.quick)
    nthreads = os.cpu_count() or 1
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(w, budget / 2, nthreads, args.model)
    tot_sims, tot_t, S = 0.0, 0.0, 0
    for _ in range(args.steps):
        sims, dt, S = oracle_sample(w, budget, nthreads, args.model)
        tot_sims += sims
        tot_t += dt
    v = tot_sims / tot_t
    return {
        "metric": METRIC, "value": v, "unit": "candidate sims/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded OPMM-simulated saccades + Gaussian noise; no dataset)",
        "config": workload_config(w, "CPU run", args.model), "impl": "reference",
        "cpu_baseline": {"value": v, "unit": "candidate sims/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"per step: saccade 0 of {w.name}, {S} simplices x {w.iterations} iterations"},
        "e2e": {"value": v, "unit": "candidate sims/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch1024",
                    choices=["batch1024", "uneven10k", "single10", "serve", "surrogate", "ivt", "gemm"])
    ap.add_argument("--no-surrogate", action="store_true", help="leave the surrogate comparison out of the line")
    ap.add_argument("--rates", type=float, nargs="+", default=[1000.0, 10000.0, 50000.0])
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--serve-seconds-line", type=float, default=1.0,
                    help="seconds of arrivals per rate for the serve object of the default line")
    ap.add_argument("--no-serve", action="store_true", help="leave the request-loop measurement out of the line")
    ap.add_argument("--no-uneven", action="store_true", help="leave the uneven 10,000-saccade search out of the line")
    ap.add_argument("--serve-slots", type=int, default=4096)
    ap.add_argument("--quick", action="store_true", help="small batch (smoke of the bench itself)")
    ap.add_argument("--saccades", type=int, default=0,
                    help="batch size of the batch1024 / uneven10k workload (profiling runs; 0 = the workload's own)")
    ap.add_argument("--model", type=int, default=18, choices=[18, 9],
                    help="search coordinates: the 18-parameter OPMM or the 9-parameter model (Sec. 2.2.2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-refine", action="store_true", help="leave the refinement after the search out of the line")
    ap.add_argument("--no-ivt", action="store_true", help="leave the I-VT front-end measurement out of the line")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    args = ap.parse_args()
    if args.model == 9 and args.workload in ("serve", "surrogate"):
        ap.error("--model 9 applies to the batched fit workloads (the request loop and the surrogate are 18-parameter)")
    if args.warmup < 3 and not args.quick:
        args.warmup = 3
    ws, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    elif args.workload == "serve":
        out = run_serve(args) if rank == 0 else None
    elif args.workload == "surrogate":
        out = run_surrogate(args) if rank == 0 else None
    elif args.workload == "ivt":
        out = run_ivt(args) if rank == 0 else None
    elif args.workload == "gemm":
        out = run_gemm(args) if rank == 0 else None
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
