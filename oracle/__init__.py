"""FP64 CPU oracle of the OPMM estimation path (ctypes wrapper over opmm_oracle.c).

TEST INFRASTRUCTURE ONLY.  The product package never imports this module; only
the tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares no
code with the CUDA path.  See opmm_oracle.c for the model reading and the paper
passages each function follows (Sec. 2.1-3.4, Table 1, Algorithm 1, Fig. 4).

Parity status: the plant equations are a reading of a paper that prints none,
so agreement with the authors' unpublished implementation is parity unpinned;
the integrator, objective and estimator are pinned by the tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NP = 18
NAMES = ["SE_ag", "SE_ant", "LT_ag", "LT_ant", "PE_ag", "PE_ant", "Vis", "FV_ag",
         "FV_ant", "Inert", "Act_ag", "Act_ant", "Deact_ag", "Deact_ant", "Step",
         "H_ag", "H_ant", "W"]
ALL_FREE = (1 << NP) - 1
# 9-parameter model (Sec. 2.2.2, Table 2): its parameters in the table's order
NAMES9 = ["K_SE", "K_LT", "B_AG", "B_ANT", "B_P", "N_C_AG", "N_C_ANT", "J", "N_C_FIX"]


def model_dim(model: int) -> int:
    return {18: NP, 9: 9}[int(model)]


def _mask(model: int, free_mask) -> int:
    return (1 << model_dim(model)) - 1 if free_mask is None else int(free_mask)

_d = ctypes.c_double
_i = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_philox4x32_10.argtypes = [ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                                             ctypes.POINTER(_u32)]
            lib.or_nsub.argtypes = [_d]
            lib.or_nsub.restype = _i
            lib.or_step_ag.argtypes = [_dp, _d]
            lib.or_step_ag.restype = _d
            lib.or_step_ant.argtypes = [_dp, _d]
            lib.or_step_ant.restype = _d
            lib.or_rest_state.argtypes = [_dp, _d, _dp]
            lib.or_simulate_rk4.argtypes = [_dp, _i, _d, _i, _d, _d, _dp, _dp]
            lib.or_simulate_rk4.restype = _i
            lib.or_simulate_exact.argtypes = [_dp, _i, _d, _i, _d, _d, _dp]
            lib.or_simulate_exact.restype = _i
            lib.or_integrate_const.argtypes = [_dp, _dp, _d, _d, _d, _d, _d, ctypes.c_long]
            lib.or_deriv.argtypes = [_dp, _dp, _d, _d, _d, _d, _dp]
            lib.or_expm7.argtypes = [_dp, _dp]
            lib.or_stiff.argtypes = [_dp, _d]
            lib.or_stiff.restype = _i
            lib.or_substeps.argtypes = [_dp, _d]
            lib.or_substeps.restype = _i
            lib.or_errors.argtypes = [_dp, _i, _d, _i, _d, _d, _dp, _dp, _dp]
            lib.or_errors.restype = _i
            lib.or_nominal_table1.argtypes = [_d, _dp]
            lib.or_calibrate_pulse.argtypes = [_d, _d]
            lib.or_calibrate_pulse.restype = _d
            lib.or_nm_testfn.argtypes = [_i, _i, _dp, _i, _d, _d, _dp, _ip]
            lib.or_nm_testfn.restype = _i
            lib.or_nm_one_step_testfn.argtypes = [_i, _i, _dp, _dp]
            lib.or_nm_one_step_testfn.restype = _i
            lib.or_start_centre.argtypes = [_i, _i, _u32, _u64, _d, _d, _dp]
            lib.or_fit.argtypes = [_dp, _i, _u32, _i, _d, _i, _d, _d, _dp, _i, _i, _d, _d, _d,
                                   _d, _d, _u64, _u32, _i, _dp, _dp, _ip, _ip]
            lib.or_fit.restype = _i
            lib.or_score.argtypes = [_dp, _i, _u32, _i, _d, _i, _d, _d, _dp, _d, _d, _dp, _i, _dp]
            lib.or_score.restype = _i
            lib.or_u_to_p.argtypes = [_dp, _i, _u32, _d, _d, _dp, _dp]
            lib.or_refine.argtypes = [_dp, _i, _u32, _i, _d, _i, _d, _d, _dp, _d, _d, _dp, _i, _d, _d,
                                      _dp, _ip, ctypes.POINTER(ctypes.c_long)]
            lib.or_refine.restype = _i
            lib.or_lm_testfn.argtypes = [_i, _dp, _i, _d, _d, _d, _d, _dp, _ip]
            lib.or_lm_testfn.restype = _i
            lib.or_u_to_p.restype = _i
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = (_u32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (_u32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (_u32 * 4)()
    lib.or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def nsub(fs: float) -> int:
    return int(_load().or_nsub(float(fs)))


def step_levels(p, theta: float):
    p = _f64(p)
    lib = _load()
    return lib.or_step_ag(_dptr(p), float(theta)), lib.or_step_ant(_dptr(p), float(theta))


def rest_state(p, theta: float) -> np.ndarray:
    p = _f64(p)
    s = np.zeros(6)
    _load().or_rest_state(_dptr(p), float(theta), _dptr(s))
    return s


def deriv(p, s, na, nn, ta, tn) -> np.ndarray:
    p, s = _f64(p), _f64(s)
    ds = np.zeros(6)
    _load().or_deriv(_dptr(p), _dptr(s), na, nn, ta, tn, _dptr(ds))
    return ds


def integrate_const(p, s, na, nn, ta, tn, h, nsteps) -> np.ndarray:
    p = _f64(p)
    s = _f64(s).copy()
    _load().or_integrate_const(_dptr(p), _dptr(s), na, nn, ta, tn, h, int(nsteps))
    return s


def expm7(m) -> np.ndarray:
    m = _f64(m).reshape(7, 7)
    e = np.zeros((7, 7))
    _load().or_expm7(_dptr(m), _dptr(e))
    return e


def simulate_rk4(p, L, fs, onset, th0, thf, return_state=False):
    p = _f64(p)
    th = np.zeros(int(L))
    st = np.zeros((int(L), 6)) if return_state else None
    rc = _load().or_simulate_rk4(_dptr(p), int(L), float(fs), int(onset), float(th0),
                                 float(thf), _dptr(th), _dptr(st) if return_state else None)
    if rc != 0:
        raise ValueError("bad saccade descriptor")
    return (th, st) if return_state else th


def simulate_exact(p, L, fs, onset, th0, thf) -> np.ndarray:
    p = _f64(p)
    th = np.zeros(int(L))
    rc = _load().or_simulate_exact(_dptr(p), int(L), float(fs), int(onset), float(th0),
                                   float(thf), _dptr(th))
    if rc != 0:
        raise ValueError("bad saccade descriptor")
    return th


def stiff(p, fs) -> bool:
    return bool(_load().or_stiff(_dptr(_f64(p)), float(fs)))


def substeps(p, fs) -> int:
    """RK4 substeps per sample for candidate p (the base count, doubled for
    stiff candidates)."""
    return int(_load().or_substeps(_dptr(_f64(p)), float(fs)))


def errors(p, L, fs, onset, th0, thf, y):
    """(MSE, mean absolute error) of the RK4 trajectory against y."""
    p, y = _f64(p), _f64(y)
    mse, mae = _d(), _d()
    _load().or_errors(_dptr(p), int(L), float(fs), int(onset), float(th0), float(thf),
                      _dptr(y), ctypes.byref(mse), ctypes.byref(mae))
    return mse.value, mae.value


def nominal_table1(dur_ms: float) -> np.ndarray:
    p = np.zeros(NP)
    _load().or_nominal_table1(float(dur_ms), _dptr(p))
    return p


def calibrate_pulse(amplitude: float, dur_ms: float) -> float:
    return float(_load().or_calibrate_pulse(float(amplitude), float(dur_ms)))


def nominal_opc(amplitude: float, dur_ms: float, calibrated: bool = True) -> np.ndarray:
    """Table 1 vector for a saccade of the given amplitude and duration; the
    agonist pulse height is calibrated to the amplitude when asked."""
    p = nominal_table1(dur_ms)
    if calibrated:
        p[15] = calibrate_pulse(abs(float(amplitude)), dur_ms)
    return p


# ---------------------------------------------------------------- Nelder-Mead
def nm_testfn(fn_id: int, verts, max_iter: int, tolx: float, tolf: float):
    """Minimise test function 0 (weighted quadratic, minimum at 1) or 1 (2-D
    Rosenbrock) from the given initial simplex.  Returns (simplex, f, iters,
    branches)."""
    v = _f64(verts).copy()
    n = v.shape[1]
    f = np.zeros(n + 1)
    br = np.zeros(max(max_iter, 1), dtype=np.int32)
    it = _load().or_nm_testfn(int(fn_id), n, _dptr(v), int(max_iter), float(tolx),
                              float(tolf), _dptr(f), br.ctypes.data_as(_ip))
    return v, f, int(it), br[:it]


def nm_one_step(fn_id: int, verts):
    v = _f64(verts).copy()
    n = v.shape[1]
    f = np.zeros(n + 1)
    b = _load().or_nm_one_step_testfn(int(fn_id), n, _dptr(v), _dptr(f))
    return int(b), v, f


def start_centre(n, s, sac_index, seed, box_lo, box_hi) -> np.ndarray:
    c = np.zeros(n)
    _load().or_start_centre(int(n), int(s), int(sac_index), int(seed), float(np.log(box_lo)),
                            float(np.log(box_hi)), _dptr(c))
    return c


def fit(pc, L, fs, onset, th0, thf, y, S, T, *, model=18, free_mask=None, box_lo=0.5, box_hi=2.0,
        step=0.05, tolx=1e-4, tolf=1e-4, seed=0, sac_index=0, nthreads=None):
    """Multi-start parallel Nelder-Mead fit of one saccade (Algorithm 1) over
    the search coordinates of the 18- or 9-parameter model (Sec. 2.2)."""
    pc, y = _f64(pc), _f64(y)
    mask = _mask(model, free_mask)
    n = bin(mask).count("1")
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    bu = np.zeros((S, n))
    bf = np.zeros(S)
    it = np.zeros(S, dtype=np.int32)
    w = _i()
    rc = _load().or_fit(_dptr(pc), int(model), mask, int(L), float(fs), int(onset), float(th0),
                        float(thf), _dptr(y), int(S), int(T), float(box_lo), float(box_hi),
                        float(step), float(tolx), float(tolf), int(seed), int(sac_index),
                        int(nthreads), _dptr(bu), _dptr(bf), it.ctypes.data_as(_ip),
                        ctypes.byref(w))
    if rc != 0:
        raise ValueError("bad fit arguments")
    win = w.value
    p = u_to_p(pc, bu[win], model=model, free_mask=mask, box_lo=box_lo, box_hi=box_hi)
    mse, mae = errors(p, L, fs, onset, th0, thf, y)
    return {"u": bu[win].copy(), "p": p, "f": float(bf[win]), "rms": float(np.sqrt(mse)),
            "l1": float(mae), "winner": win, "iters": it, "best_f_all": bf, "best_u_all": bu}


def score(pc, L, fs, onset, th0, thf, y, u, *, model=18, free_mask=None, box_lo=0.5, box_hi=2.0):
    pc, y, u = _f64(pc), _f64(y), _f64(u)
    m = u.shape[0]
    f = np.zeros(m)
    rc = _load().or_score(_dptr(pc), int(model), _mask(model, free_mask), int(L), float(fs), int(onset),
                          float(th0), float(thf), _dptr(y), float(box_lo), float(box_hi), _dptr(u), m, _dptr(f))
    if rc != 0:
        raise ValueError("bad score arguments")
    return f


def u_to_p(pc, u, *, model=18, free_mask=None, box_lo=0.5, box_hi=2.0) -> np.ndarray:
    """Full OPC vector of search point u (the objective's clamp applied)."""
    pc, u = _f64(pc), _f64(u)
    p = np.zeros(NP)
    rc = _load().or_u_to_p(_dptr(pc), int(model), _mask(model, free_mask), float(box_lo), float(box_hi),
                           _dptr(u), _dptr(p))
    if rc != 0:
        raise ValueError("bad model or centre")
    return p


def refine(pc, L, fs, onset, th0, thf, y, u0, K, *, model=18, free_mask=None, box_lo=0.5, box_hi=2.0,
           delta=1e-2, lambda0=1e-3):
    """Levenberg-Marquardt refinement of search point u0 (Sec. 5's gradient
    alternative): K iterations, central-difference Jacobian of step delta
    (ln units), damping lambda0.  Returns u, p, f (MSE), rms, accepted steps
    and residual evaluations."""
    pc, y = _f64(pc), _f64(y)
    u = _f64(u0).copy()
    f = _d()
    acc = _i()
    nres = ctypes.c_long()
    rc = _load().or_refine(_dptr(pc), int(model), _mask(model, free_mask), int(L), float(fs), int(onset),
                           float(th0), float(thf), _dptr(y), float(box_lo), float(box_hi), _dptr(u), int(K),
                           float(delta), float(lambda0), ctypes.byref(f), ctypes.byref(acc), ctypes.byref(nres))
    if rc != 0:
        raise ValueError("bad refine arguments")
    p = u_to_p(pc, u, model=model, free_mask=free_mask, box_lo=box_lo, box_hi=box_hi)
    mse, mae = errors(p, L, fs, onset, th0, thf, y)
    return {"u": u, "p": p, "f": float(f.value), "rms": float(np.sqrt(mse)), "l1": float(mae),
            "accepted": int(acc.value), "evaluations": int(nres.value)}


def lm_testfn(fn_id: int, u0, K: int, lo=-np.inf, hi=np.inf, delta=1e-6, lambda0=1e-3):
    """Levenberg-Marquardt on a textbook residual (0: linear least squares,
    1: Rosenbrock)."""
    u = _f64(u0).copy()
    f = _d()
    acc = _i()
    rc = _load().or_lm_testfn(int(fn_id), _dptr(u), int(K), float(lo), float(hi), float(delta), float(lambda0),
                              ctypes.byref(f), ctypes.byref(acc))
    if rc != 0:
        raise ValueError("bad test function")
    return u, float(f.value), int(acc.value)
