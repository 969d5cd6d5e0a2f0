"""Python binding of the GB300 OPMM library (include/opmm.h).

Argument marshalling only: every step of the estimation path runs in the CUDA
kernels of libopmm.so.  Functions keep the C names (opmm_create,
opmm_simulate, opmm_score, opmm_nominal_opc, opmm_fit_batch, opmm_plan_*,
...); arrays may be numpy (host) or torch CUDA tensors (device), passed to the
library as plain pointers.  There is no CPU fallback: if the library cannot be
loaded, or no CUDA device is usable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libopmm.so")

OPMM_OK = 0
OPMM_NOT_READY = 1
OPMM_EINVAL = -1
OPMM_ENOMEM = -2
OPMM_ECUDA = -3
OPMM_ETIMEDOUT = -4
OPMM_EBUSY = -5
OPMM_NPARAM = 18
OPMM_MODEL_18 = 18
OPMM_MODEL_9 = 9
OPMM_SOURCE_REFINED = 3
OPMM_PULSE_TABLE1 = 0
OPMM_SOURCE_PLAIN, OPMM_SOURCE_SEEDED, OPMM_SOURCE_FALLBACK = 0, 1, 2
OPMM_PULSE_CALIBRATED = 1
OPMM_WALK_SCALAR, OPMM_WALK_PACKED, OPMM_WALK_LEAN = 0, 1, 2
WALK_NAMES = {OPMM_WALK_SCALAR: "scalar", OPMM_WALK_PACKED: "packed", OPMM_WALK_LEAN: "lean"}

PARAM_NAMES = ["SE_ag", "SE_ant", "LT_ag", "LT_ant", "PE_ag", "PE_ant", "Vis", "FV_ag", "FV_ant",
               "Inert", "Act_ag", "Act_ant", "Deact_ag", "Deact_ant", "Step", "H_ag", "H_ant", "W"]

# Every symbol include/opmm.h declares.
EXPORTS = ["opmm_create", "opmm_destroy", "opmm_last_error", "opmm_set_stream", "opmm_set_search_variant",
           "opmm_search_variants", "opmm_search_variant_walk", "opmm_simulate",
           "opmm_score", "opmm_nominal_opc", "opmm_fit_batch", "opmm_plan_create",
           "opmm_plan_execute", "opmm_plan_info", "opmm_plan_variant", "opmm_plan_tuning", "opmm_plan_last_search_ms",
           "opmm_plan_destroy",
           "opmm_fit_saccade_static", "opmm_surrogate_init", "opmm_surrogate_num_params",
           "opmm_surrogate_get_params", "opmm_surrogate_set_params", "opmm_surrogate_grad", "opmm_surrogate_apply_grad",
           "opmm_surrogate_train", "opmm_surrogate_predict", "opmm_surrogate_save", "opmm_surrogate_load", "opmm_featurize",
           "opmm_gemm_bf16", "opmm_serve_start", "opmm_serve_submit", "opmm_serve_poll",
           "opmm_serve_stats_get", "opmm_serve_stop"]


class OpmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"OPMM error {code}: {msg}")
        self.code = code


class opmm_saccade(ctypes.Structure):
    _fields_ = [("trace_deg", ctypes.c_void_p), ("n_samples", ctypes.c_int32),
                ("sample_rate_hz", ctypes.c_float), ("onset_index", ctypes.c_int32),
                ("theta_start_deg", ctypes.c_float), ("theta_end_deg", ctypes.c_float),
                ("duration_ms", ctypes.c_float)]


class opmm_fit_opts(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("box_lo", ctypes.c_float),
                ("box_hi", ctypes.c_float), ("init_step", ctypes.c_float),
                ("tol_x", ctypes.c_float), ("tol_f", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("pulse_init", ctypes.c_int32), ("use_surrogate", ctypes.c_int32),
                ("init_opc", ctypes.c_void_p)]


class opmm_serve_opts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_device_bytes", ctypes.c_uint64),
                ("max_queue", ctypes.c_int32), ("max_samples", ctypes.c_int32),
                ("round_iters", ctypes.c_int32), ("max_admit_per_round", ctypes.c_int32)]


class opmm_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("queued", ctypes.c_int32), ("active", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class opmm_fit_result(ctypes.Structure):
    _fields_ = [("opc", ctypes.c_float * 18), ("f", ctypes.c_float),
                ("iterations_run", ctypes.c_int32), ("rms_deg", ctypes.c_double),
                ("l1_deg", ctypes.c_double), ("status", ctypes.c_int32), ("winner", ctypes.c_int32),
                ("evaluations", ctypes.c_int32), ("source", ctypes.c_int32),
                ("pulse_end_evals", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libopmm.so (building it first if missing).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64p = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)
    lib.opmm_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
    lib.opmm_destroy.argtypes = [vp]
    lib.opmm_destroy.restype = None
    lib.opmm_last_error.argtypes = [vp]
    lib.opmm_last_error.restype = ctypes.c_char_p
    lib.opmm_set_stream.argtypes = [vp, vp]
    lib.opmm_set_search_variant.argtypes = [vp, i32]
    lib.opmm_search_variants.argtypes = [ctypes.POINTER(i32)]
    lib.opmm_search_variant_info.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.opmm_search_variant_walk.argtypes = [i32, ctypes.POINTER(i32)]
    lib.opmm_simulate.argtypes = [vp, vp, i32, ctypes.POINTER(opmm_saccade), i32, vp, i64p, vp]
    lib.opmm_score.argtypes = [vp, vp, i32, ctypes.POINTER(opmm_saccade), vp]
    lib.opmm_nominal_opc.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32, i32, vp]
    lib.opmm_refine_batch.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32, vp, ctypes.POINTER(opmm_refine_opts),
                                      ctypes.POINTER(opmm_fit_result)]
    lib.opmm_detect_saccades.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.POINTER(opmm_ivt_opts), vp,
                                         i32, ctypes.POINTER(i32)]
    lib.opmm_fit_batch_seeded.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32, ctypes.POINTER(opmm_fit_opts),
                                          ctypes.POINTER(opmm_fit_opts), ctypes.c_float,
                                          ctypes.POINTER(opmm_fit_result), ctypes.POINTER(ctypes.c_int32)]
    lib.opmm_fit_batch.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32,
                                   ctypes.POINTER(opmm_fit_opts), ctypes.POINTER(opmm_fit_result)]
    lib.opmm_plan_create.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32,
                                     ctypes.POINTER(opmm_fit_opts), ctypes.POINTER(vp)]
    lib.opmm_plan_execute.argtypes = [vp, ctypes.POINTER(opmm_fit_result)]
    lib.opmm_plan_info.argtypes = [vp] + [ctypes.POINTER(i32)] * 4
    lib.opmm_plan_variant.argtypes = [vp, ctypes.POINTER(i32)]
    lib.opmm_plan_last_search_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.opmm_plan_tuning.argtypes = [vp] + [vp] * 5 + [i32, ctypes.POINTER(i32)]
    lib.opmm_plan_destroy.argtypes = [vp]
    lib.opmm_plan_destroy.restype = None
    lib.opmm_fit_saccade_static.argtypes = [ctypes.POINTER(opmm_saccade), ctypes.POINTER(opmm_fit_opts),
                                            vp, vp]
    lib.opmm_surrogate_init.argtypes = [vp, ctypes.c_uint64]
    lib.opmm_surrogate_num_params.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    lib.opmm_surrogate_get_params.argtypes = [vp, vp]
    lib.opmm_surrogate_set_params.argtypes = [vp, vp]
    lib.opmm_surrogate_grad.argtypes = [vp, vp, vp, i32, ctypes.POINTER(ctypes.c_float), vp, vp]
    lib.opmm_surrogate_apply_grad.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float]
    lib.opmm_surrogate_train.argtypes = [vp, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                         ctypes.c_int64, vp]
    lib.opmm_surrogate_predict.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32, i32, vp]
    lib.opmm_surrogate_save.argtypes = [vp, ctypes.c_char_p]
    lib.opmm_surrogate_load.argtypes = [vp, ctypes.c_char_p]
    lib.opmm_featurize.argtypes = [vp, ctypes.POINTER(opmm_saccade), i32, vp]
    lib.opmm_gemm_bf16.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    lib.opmm_serve_start.argtypes = [vp, ctypes.POINTER(opmm_serve_opts), ctypes.POINTER(opmm_fit_opts)]
    lib.opmm_serve_submit.argtypes = [vp, ctypes.POINTER(opmm_saccade), ctypes.POINTER(ctypes.c_uint64)]
    lib.opmm_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(opmm_fit_result), i32,
                                    ctypes.POINTER(ctypes.c_double)]
    lib.opmm_serve_stats_get.argtypes = [vp, ctypes.POINTER(opmm_serve_stats)]
    lib.opmm_serve_stop.argtypes = [vp]
    for name in ["opmm_create", "opmm_set_stream", "opmm_set_search_variant", "opmm_search_variants", "opmm_simulate", "opmm_score", "opmm_nominal_opc",
                 "opmm_fit_batch", "opmm_fit_batch_seeded", "opmm_plan_create", "opmm_plan_execute", "opmm_plan_info",
                 "opmm_plan_last_search_ms", "opmm_fit_saccade_static", "opmm_plan_tuning",
                 "opmm_surrogate_init", "opmm_surrogate_num_params", "opmm_surrogate_get_params",
                 "opmm_surrogate_set_params", "opmm_surrogate_grad", "opmm_surrogate_train",
                 "opmm_surrogate_predict", "opmm_surrogate_save", "opmm_surrogate_load",
                 "opmm_featurize", "opmm_gemm_bf16", "opmm_serve_start", "opmm_serve_submit",
                 "opmm_serve_poll", "opmm_serve_stats_get", "opmm_serve_stop"]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ------------------------------------------------------------------ pointers
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=np.float32):
    """(pointer, keepalive) of a host numpy array or a torch tensor."""
    if x is None:
        return None, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a


# ------------------------------------------------------------------ batches
@dataclass
class SaccadeBatch:
    """Descriptors of n recorded saccades plus the storage their traces live in.

    `traces` is either one packed array (numpy host array or torch CUDA tensor)
    with `offsets[i]` the first sample of saccade i, or a list of per-saccade
    arrays."""
    traces: object
    offsets: Optional[np.ndarray]
    n_samples: np.ndarray
    sample_rate_hz: np.ndarray
    onset_index: np.ndarray
    theta_start_deg: np.ndarray
    theta_end_deg: np.ndarray
    duration_ms: np.ndarray

    def __len__(self):
        return int(len(self.n_samples))

    def descriptors(self):
        n = len(self)
        arr = (opmm_saccade * n)()
        keep = []
        if isinstance(self.traces, (list, tuple)):
            bases = []
            for t in self.traces:
                p, k = _ptr(t)
                keep.append(k)
                bases.append(p.value)
        else:
            p, k = _ptr(self.traces)
            keep.append(k)
            esz = 4
            bases = [p.value + int(o) * esz for o in self.offsets]
        for i in range(n):
            arr[i].trace_deg = bases[i]
            arr[i].n_samples = int(self.n_samples[i])
            arr[i].sample_rate_hz = float(self.sample_rate_hz[i])
            arr[i].onset_index = int(self.onset_index[i])
            arr[i].theta_start_deg = float(self.theta_start_deg[i])
            arr[i].theta_end_deg = float(self.theta_end_deg[i])
            arr[i].duration_ms = float(self.duration_ms[i])
        return arr, keep


def make_batch(traces, sample_rate_hz, onset_index, theta_start_deg, theta_end_deg, duration_ms,
               n_samples=None, offsets=None) -> SaccadeBatch:
    n = len(sample_rate_hz)
    if n_samples is None:
        n_samples = [len(t) for t in traces]
    return SaccadeBatch(traces, None if offsets is None else np.asarray(offsets, np.int64),
                        np.asarray(n_samples, np.int32), np.asarray(sample_rate_hz, np.float32),
                        np.asarray(onset_index, np.int32), np.asarray(theta_start_deg, np.float32),
                        np.asarray(theta_end_deg, np.float32),
                        np.asarray(duration_ms if duration_ms is not None else [0.0] * n, np.float32))


def fit_opts(candidates=4096, iterations=20, box_lo=0.5, box_hi=2.0, init_step=0.05, tol_x=1e-4,
             tol_f=1e-4, seed=0, pulse_init=OPMM_PULSE_CALIBRATED, use_surrogate=False,
             init_opc=None, model=OPMM_MODEL_18):
    o = opmm_fit_opts()
    o.model = int(model)
    o.candidates, o.iterations = int(candidates), int(iterations)
    o.box_lo, o.box_hi, o.init_step = float(box_lo), float(box_hi), float(init_step)
    o.tol_x, o.tol_f, o.seed = float(tol_x), float(tol_f), int(seed)
    o.pulse_init, o.use_surrogate = int(pulse_init), int(bool(use_surrogate))
    keep = None
    if init_opc is not None:
        keep = np.ascontiguousarray(init_opc, dtype=np.float32)
        o.init_opc = keep.ctypes.data
    return o, keep


def results_to_numpy(res) -> dict:
    n = len(res)
    buf = np.frombuffer(bytes(res), dtype=np.dtype([("opc", "<f4", (18,)), ("f", "<f4"),
                                                     ("iterations_run", "<i4"), ("rms_deg", "<f8"),
                                                     ("l1_deg", "<f8"), ("status", "<i4"),
                                                     ("winner", "<i4"), ("evaluations", "<i4"),
                                                     ("source", "<i4"), ("pulse_end_evals", "<i4"),
                                                     ("reserved", "<i4")]), count=n)
    return {k: buf[k].copy() for k in buf.dtype.names}


# ------------------------------------------------------------------ C names
def _check(ctx, rc):
    if rc < 0:
        lib = load_library()
        msg = lib.opmm_last_error(ctx).decode(errors="replace") if ctx else "no context"
        raise OpmmError(rc, msg)
    return rc


def opmm_create(device: int = 0):
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.opmm_create(int(device), ctypes.byref(h))
    if rc != OPMM_OK:
        raise OpmmError(rc, "opmm_create failed (no usable CUDA device?)")
    return h


def opmm_destroy(ctx):
    _IVT_OUT.pop(_ctx_key(ctx), None)
    load_library().opmm_destroy(ctx)


def opmm_last_error(ctx) -> str:
    return load_library().opmm_last_error(ctx).decode(errors="replace")


def opmm_set_stream(ctx, stream_handle: int):
    _check(ctx, load_library().opmm_set_stream(ctx, ctypes.c_void_p(int(stream_handle) or None)))


def opmm_set_search_variant(ctx, variant: int):
    _check(ctx, load_library().opmm_set_search_variant(ctx, int(variant)))


def opmm_search_variants() -> int:
    n = ctypes.c_int32()
    load_library().opmm_search_variants(ctypes.byref(n))
    return int(n.value)


def opmm_search_variant_info(variant: int):
    """(simplices per block, model) of a search variant."""
    g, m = ctypes.c_int32(), ctypes.c_int32()
    rc = load_library().opmm_search_variant_info(int(variant), ctypes.byref(g), ctypes.byref(m))
    if rc != OPMM_OK:
        raise OpmmError(rc, "search variant out of range")
    return int(g.value), int(m.value)


def opmm_search_variant_walk(variant: int) -> int:
    """How a search variant integrates a candidate (OPMM_WALK_*)."""
    w = ctypes.c_int32()
    rc = load_library().opmm_search_variant_walk(int(variant), ctypes.byref(w))
    if rc != OPMM_OK:
        raise OpmmError(rc, "search variant out of range")
    return int(w.value)


def opmm_simulate(ctx, opc, batch: SaccadeBatch, sac_index=None, out=None):
    """Trajectories [n][L_i] packed; returns (out, offsets)."""
    lib = load_library()
    n = int(opc.shape[0])
    sidx = np.arange(n, dtype=np.int32) if sac_index is None else np.asarray(sac_index, np.int32)
    L = np.asarray(batch.n_samples, np.int64)[sidx]
    offs = np.concatenate([[0], np.cumsum(L)[:-1]]).astype(np.int64)
    if out is None:
        out = np.zeros(int(L.sum()), dtype=np.float32)
    descs, keep = batch.descriptors()
    po, ko = _ptr(opc)
    pout, kout = _ptr(out)
    rc = lib.opmm_simulate(ctx, po, n, descs, len(batch),
                           None if sac_index is None else sidx.ctypes.data_as(ctypes.c_void_p),
                           offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), pout)
    _check(ctx, rc)
    return out, offs


def opmm_score(ctx, opc, batch: SaccadeBatch, index: int = 0, out=None):
    lib = load_library()
    m = int(opc.shape[0])
    if out is None:
        out = np.zeros(m, dtype=np.float32)
    descs, keep = batch.descriptors()
    po, ko = _ptr(opc)
    pf, kf = _ptr(out)
    _check(ctx, lib.opmm_score(ctx, po, m, ctypes.byref(descs[index]), pf))
    return out


def opmm_nominal_opc(ctx, batch: SaccadeBatch, pulse_init=OPMM_PULSE_CALIBRATED) -> np.ndarray:
    lib = load_library()
    out = np.zeros((len(batch), 18), dtype=np.float32)
    descs, keep = batch.descriptors()
    _check(ctx, lib.opmm_nominal_opc(ctx, descs, len(batch), int(pulse_init),
                                     out.ctypes.data_as(ctypes.c_void_p)))
    return out


def opmm_fit_batch(ctx, batch: SaccadeBatch, **opts) -> dict:
    lib = load_library()
    o, keep_o = fit_opts(**opts)
    descs, keep = batch.descriptors()
    res = (opmm_fit_result * len(batch))()
    _check(ctx, lib.opmm_fit_batch(ctx, descs, len(batch), ctypes.byref(o), res))
    return results_to_numpy(res)


class opmm_refine_opts(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("iterations", ctypes.c_int32), ("box_lo", ctypes.c_float),
                ("box_hi", ctypes.c_float), ("fd_step", ctypes.c_float), ("lambda0", ctypes.c_float),
                ("pulse_init", ctypes.c_int32), ("centre_opc", ctypes.c_void_p)]


def opmm_refine_batch(ctx, batch: SaccadeBatch, start_opc, iterations=10, box_lo=0.5, box_hi=2.0, fd_step=1e-2,
                      lambda0=1e-3, model=OPMM_MODEL_18, pulse_init=OPMM_PULSE_CALIBRATED, centre_opc=None) -> dict:
    """Levenberg-Marquardt refinement of start_opc ([n][18]) on each saccade."""
    lib = load_library()
    o = opmm_refine_opts()
    o.model, o.iterations = int(model), int(iterations)
    o.box_lo, o.box_hi, o.fd_step, o.lambda0 = float(box_lo), float(box_hi), float(fd_step), float(lambda0)
    o.pulse_init = int(pulse_init)
    keep_c = None
    if centre_opc is not None:
        keep_c = np.ascontiguousarray(centre_opc, dtype=np.float32)
        o.centre_opc = keep_c.ctypes.data
    start = np.ascontiguousarray(start_opc, dtype=np.float32)
    descs, keep = batch.descriptors()
    res = (opmm_fit_result * len(batch))()
    _check(ctx, lib.opmm_refine_batch(ctx, descs, len(batch), start.ctypes.data, ctypes.byref(o), res))
    return results_to_numpy(res)


class opmm_ivt_opts(ctypes.Structure):
    _fields_ = [("threshold_dps", ctypes.c_float), ("min_duration_ms", ctypes.c_float),
                ("min_amplitude_deg", ctypes.c_float), ("valid_min_deg", ctypes.c_float),
                ("valid_max_deg", ctypes.c_float), ("pre_samples", ctypes.c_int32), ("post_samples", ctypes.c_int32)]


IVT_EVENT_DTYPE = np.dtype([("onset", "<i8"), ("end", "<i8"), ("window_start", "<i8"), ("n_samples", "<i4"),
                            ("onset_index", "<i4"), ("theta_start_deg", "<f4"), ("theta_end_deg", "<f4"),
                            ("amplitude_deg", "<f4"), ("duration_ms", "<f4"), ("peak_velocity_dps", "<f4"),
                            ("reserved", "<i4")])


_IVT_OUT = {}


def _ctx_key(ctx) -> int:
    return ctypes.cast(ctx, ctypes.c_void_p).value or 0


def opmm_detect_saccades(ctx, stream, sample_rate_hz, threshold_dps=30.0, min_duration_ms=6.0,
                         min_amplitude_deg=4.0, valid_min_deg=-90.0, valid_max_deg=90.0, pre_samples=10,
                         post_samples=40, max_events=None) -> np.ndarray:
    """I-VT detection on a position stream (numpy host array or torch CUDA
    tensor of float32); returns the kept events (IVT_EVENT_DTYPE) in onset
    order."""
    lib = load_library()
    o = opmm_ivt_opts(float(threshold_dps), float(min_duration_ms), float(min_amplitude_deg), float(valid_min_deg),
                      float(valid_max_deg), int(pre_samples), int(post_samples))
    if _is_torch(stream) and stream.dtype.__repr__() != "torch.float32":
        raise ValueError("stream tensor must be float32")
    ptr, keep = _ptr(stream)
    n = int(stream.numel()) if _is_torch(stream) else int(keep.size)
    cap = int(max_events) if max_events is not None else max(16, n // 64)
    # the event array is kept per context and reused (its pages are touched
    # once); the caller gets a copy of the events found
    out = _IVT_OUT.get(_ctx_key(ctx))
    if out is None or out.size < cap:
        out = np.zeros(cap, dtype=IVT_EVENT_DTYPE)
        _IVT_OUT[_ctx_key(ctx)] = out
    found = ctypes.c_int32()
    _check(ctx, lib.opmm_detect_saccades(ctx, ptr, ctypes.c_int64(n), ctypes.c_float(sample_rate_hz),
                                         ctypes.byref(o), out.ctypes.data, cap, ctypes.byref(found)))
    if found.value > cap and max_events is None:
        return opmm_detect_saccades(ctx, stream, sample_rate_hz, threshold_dps, min_duration_ms, min_amplitude_deg,
                                    valid_min_deg, valid_max_deg, pre_samples, post_samples, found.value)
    return out[:min(found.value, cap)].copy()


def batch_from_events(stream, events, sample_rate_hz) -> SaccadeBatch:
    """Descriptors and host traces of detected saccades (the event windows)."""
    x = np.asarray(stream, dtype=np.float32)
    traces = [x[int(e["window_start"]):int(e["window_start"]) + int(e["n_samples"])].copy() for e in events]
    n = len(events)
    return make_batch(traces, [float(sample_rate_hz)] * n, events["onset_index"], events["theta_start_deg"],
                      events["theta_end_deg"], events["duration_ms"])


def opmm_fit_batch_seeded(ctx, batch: SaccadeBatch, seeded: dict, plain: dict, fallback_rms_deg=0.1):
    """Surrogate-seeded fit; saccades it leaves above fallback_rms_deg are
    fitted again with the plain search.  Returns (results, n_fallback)."""
    lib = load_library()
    so, keep_s = fit_opts(**dict(seeded, use_surrogate=True))
    po, keep_p = fit_opts(**dict(plain, use_surrogate=False))
    descs, keep = batch.descriptors()
    res = (opmm_fit_result * len(batch))()
    nfb = ctypes.c_int32(0)
    _check(ctx, lib.opmm_fit_batch_seeded(ctx, descs, len(batch), ctypes.byref(so), ctypes.byref(po),
                                          ctypes.c_float(fallback_rms_deg), res, ctypes.byref(nfb)))
    return results_to_numpy(res), int(nfb.value)


class Plan:
    """opmm_plan_*: a graph-captured fit of a fixed batch (traces re-read on
    every execute)."""

    def __init__(self, ctx, batch: SaccadeBatch, **opts):
        self.lib = load_library()
        self.ctx = ctx
        o, self._keep_o = fit_opts(**opts)
        self._descs, self._keep = batch.descriptors()
        self.n = len(batch)
        self.h = ctypes.c_void_p()
        _check(ctx, self.lib.opmm_plan_create(ctx, self._descs, self.n, ctypes.byref(o),
                                              ctypes.byref(self.h)))
        self._res = (opmm_fit_result * self.n)()

    def execute(self) -> dict:
        _check(self.ctx, self.lib.opmm_plan_execute(self.h, self._res))
        return results_to_numpy(self._res)

    def execute_raw(self):
        _check(self.ctx, self.lib.opmm_plan_execute(self.h, self._res))
        return self._res

    def info(self) -> dict:
        v = [ctypes.c_int32() for _ in range(4)]
        _check(self.ctx, self.lib.opmm_plan_info(self.h, *[ctypes.byref(x) for x in v]))
        var = ctypes.c_int32()
        _check(self.ctx, self.lib.opmm_plan_variant(self.h, ctypes.byref(var)))
        return {"variant": var.value, "walk": WALK_NAMES[opmm_search_variant_walk(var.value)],
                "simplices_per_block": v[0].value, "threads": v[1].value,
                "blocks_per_sm": v[2].value, "kernels_per_execute": v[3].value}

    def tuning(self) -> list:
        cap = 32
        arrs = [np.zeros(cap, np.int32) for _ in range(4)]
        ms = np.zeros(cap, np.float32)
        cnt = ctypes.c_int32()
        _check(self.ctx, self.lib.opmm_plan_tuning(self.h, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                                   ms.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(cnt)))
        n = min(cnt.value, cap)
        return [{"variant": int(arrs[0][i]), "simplices_per_block": int(arrs[1][i]),
                 "walk": WALK_NAMES[opmm_search_variant_walk(int(arrs[0][i]))],
                 "min_blocks": int(arrs[2][i]), "blocks_per_sm": int(arrs[3][i]),
                 "probe_ms": float(ms[i])} for i in range(n)]

    def last_search_ms(self) -> float:
        ms = ctypes.c_float()
        _check(self.ctx, self.lib.opmm_plan_last_search_ms(self.h, ctypes.byref(ms)))
        return float(ms.value)

    def destroy(self):
        if self.h:
            self.lib.opmm_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def opmm_plan_create(ctx, batch: SaccadeBatch, **opts) -> Plan:
    return Plan(ctx, batch, **opts)


def opmm_plan_execute(plan: Plan) -> dict:
    return plan.execute()


def opmm_plan_info(plan: Plan) -> dict:
    return plan.info()


def opmm_plan_destroy(plan: Plan):
    plan.destroy()


def opmm_fit_saccade_static(batch: SaccadeBatch, out_device, stream_handle: int = 0, index: int = 0,
                            **opts) -> int:
    """Allocation-free fit of saccade `index` of a batch whose traces are in
    device memory; writes one opmm_fit_result into `out_device` (a device
    tensor of at least sizeof(opmm_fit_result) bytes).  Returns the status
    code (no context, so no error text)."""
    lib = load_library()
    o, keep_o = fit_opts(**opts)
    descs, keep = batch.descriptors()
    po, ko = _ptr(out_device)
    return int(lib.opmm_fit_saccade_static(ctypes.byref(descs[index]), ctypes.byref(o), po,
                                           ctypes.c_void_p(int(stream_handle) or None)))


# ------------------------------------------------------------------ surrogate
def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def opmm_surrogate_init(ctx, seed: int = 0):
    _check(ctx, load_library().opmm_surrogate_init(ctx, int(seed)))


def opmm_surrogate_num_params() -> int:
    n = ctypes.c_int64()
    load_library().opmm_surrogate_num_params(ctypes.byref(n))
    return int(n.value)


def opmm_surrogate_get_params(ctx) -> np.ndarray:
    out = np.zeros(opmm_surrogate_num_params(), np.float32)
    _check(ctx, load_library().opmm_surrogate_get_params(ctx, _vp(out)))
    return out


def opmm_surrogate_set_params(ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, load_library().opmm_surrogate_set_params(ctx, _vp(p)))


def opmm_surrogate_grad(ctx, x, t):
    """(loss, grad[n_params], y[m][18]) for features x [m][512], targets t [m][18]."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    m = x.shape[0]
    g = np.zeros(opmm_surrogate_num_params(), np.float32)
    y = np.zeros((m, 18), np.float32)
    loss = ctypes.c_float()
    _check(ctx, load_library().opmm_surrogate_grad(ctx, _vp(x), _vp(t), m, ctypes.byref(loss), _vp(g), _vp(y)))
    return float(loss.value), g, y


def opmm_surrogate_apply_grad(ctx, grad, lr, weight_decay=0.0):
    """One AdamW step of the surrogate's parameters with gradient grad [n_params]."""
    g = np.ascontiguousarray(grad, dtype=np.float32)
    if g.shape != (opmm_surrogate_num_params(),):
        raise ValueError("gradient must have one entry per parameter")
    _check(ctx, load_library().opmm_surrogate_apply_grad(ctx, _vp(g), float(lr), float(weight_decay)))


def opmm_surrogate_train(ctx, steps, batch=4096, lr=1e-3, weight_decay=1e-4, data_seed=1, sample_base=0):
    losses = np.zeros(max(1, steps), np.float32)
    _check(ctx, load_library().opmm_surrogate_train(ctx, int(steps), int(batch), float(lr),
                                                     float(weight_decay), int(data_seed),
                                                     int(sample_base), _vp(losses)))
    return losses[:steps]


def opmm_surrogate_predict(ctx, batch: SaccadeBatch, pulse_init=OPMM_PULSE_CALIBRATED) -> np.ndarray:
    out = np.zeros((len(batch), 18), np.float32)
    descs, keep = batch.descriptors()
    _check(ctx, load_library().opmm_surrogate_predict(ctx, descs, len(batch), int(pulse_init), _vp(out)))
    return out


def opmm_surrogate_save(ctx, path: str):
    _check(ctx, load_library().opmm_surrogate_save(ctx, path.encode()))


def opmm_surrogate_load(ctx, path: str):
    _check(ctx, load_library().opmm_surrogate_load(ctx, path.encode()))


def opmm_featurize(ctx, batch: SaccadeBatch) -> np.ndarray:
    out = np.zeros((len(batch), 512), np.float32)
    descs, keep = batch.descriptors()
    _check(ctx, load_library().opmm_featurize(ctx, descs, len(batch), _vp(out)))
    return out


def opmm_gemm_bf16(ctx, A, B, out=None):
    """D = A . B^T for torch bfloat16 CUDA tensors A [M][K], B [N][K]; returns D (float32)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(ctx, load_library().opmm_gemm_bf16(ctx, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                               int(M), int(N), int(K), ctypes.c_void_p(out.data_ptr())))
    return out


# ------------------------------------------------------------------ serving
def serve_opts(max_slots=4096, max_device_bytes=0, max_queue=100000, max_samples=400, round_iters=5,
               max_admit_per_round=4096):
    o = opmm_serve_opts()
    o.max_slots, o.max_device_bytes, o.max_queue = int(max_slots), int(max_device_bytes), int(max_queue)
    o.max_samples, o.round_iters, o.max_admit_per_round = int(max_samples), int(round_iters), int(max_admit_per_round)
    return o


def opmm_serve_start(ctx, cfg: opmm_serve_opts, **fit):
    o, keep = fit_opts(**fit)
    _check(ctx, load_library().opmm_serve_start(ctx, ctypes.byref(cfg), ctypes.byref(o)))


def opmm_serve_submit_raw(ctx, desc) -> tuple:
    """(status, ticket) for one opmm_saccade (no exception on EBUSY)."""
    t = ctypes.c_uint64()
    rc = load_library().opmm_serve_submit(ctx, ctypes.byref(desc), ctypes.byref(t))
    return int(rc), int(t.value)


def opmm_serve_submit(ctx, batch: SaccadeBatch, index: int = 0) -> int:
    descs, keep = batch.descriptors()
    rc, t = opmm_serve_submit_raw(ctx, descs[index])
    _check(ctx, rc)
    return t


def opmm_serve_poll_raw(ctx, ticket: int, timeout_us: int = 0):
    """(status, result-dict or None, latency_us)."""
    r = opmm_fit_result()
    lat = ctypes.c_double()
    rc = load_library().opmm_serve_poll(ctx, ctypes.c_uint64(int(ticket)), ctypes.byref(r), int(timeout_us),
                                        ctypes.byref(lat))
    if rc != OPMM_OK:
        return int(rc), None, None
    return OPMM_OK, {k: v[0] for k, v in results_to_numpy((opmm_fit_result * 1)(r)).items()}, float(lat.value)


def opmm_serve_poll(ctx, ticket: int, timeout_us: int = 10_000_000):
    rc, res, lat = opmm_serve_poll_raw(ctx, ticket, timeout_us)
    _check(ctx, rc)
    if rc != OPMM_OK:
        raise OpmmError(rc, "result not ready")
    return res, lat


def opmm_serve_stats_get(ctx) -> dict:
    s = opmm_serve_stats()
    _check(ctx, load_library().opmm_serve_stats_get(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}


def opmm_serve_stop(ctx):
    _check(ctx, load_library().opmm_serve_stop(ctx))
