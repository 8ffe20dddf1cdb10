"""FP64 CPU oracle for the per-day GradABM step (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only users.  The product path (the CUDA
library and its Python binding) never imports this package, and this package
imports nothing from the product.

``gabm_oracle.c`` holds the simulator, written in FP64 in the order of the
paper's Sec. 3.1 update (Eq. 1-3), assumptions A1-A6 (App. A) and the
unrolled-loop adjoint (App. B).  This module compiles it with gcc and exposes
numpy-level wrappers.  ``brute`` (exact enumeration on tiny graphs) and
``meanfield`` (mean-field recurrence and final-size relation) are independent
computations used to pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

NEVER = 32767
NUM_AGES = 9

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gabm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgabm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (IEEE FP64, OpenMP over pull loops)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64, u64, u32, i32, f64 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_int, ctypes.c_double)
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_hash.argtypes = [u64, u32, u32, u32, u32]
            L.orc_hash.restype = u32
            L.orc_uniform.argtypes = [u64, u32, u32, u32, u32]
            L.orc_uniform.restype = f64
            L.orc_uniform_array.argtypes = [u64, i64, P, u32, u32, u32, P]
            L.orc_select_seeds.argtypes = [i64, P, u64, u32, i64, P]
            L.orc_mean_weighted_degree.argtypes = [i64, P, P]
            L.orc_mean_weighted_degree.restype = f64
            L.orc_day_hard.argtypes = [i64, P, P, P, P, P, i32, i32, P, u64, u32, f64, i32, f64,
                                       P, P, P, P, P, P, P, P, P]
            L.orc_forward_hard.argtypes = [i64, P, P, P, P, P, i32, i32, P, u64, u32, i32, i32,
                                           P, P, P, i64, P, P, P, P, P, P, P, P]
            L.orc_backward_hard.argtypes = [i64, P, P, P, P, P, i32, i32, P, u64, u32, i32,
                                            P, P, P, P, P, P, P, P, P, P]
            L.orc_forward_soft.argtypes = [i64, P, P, P, P, P, i32, i32, P, u64, u32, i32,
                                           P, P, P, i64, P, P, P, P, P, P, P]
            L.orc_backward_soft.argtypes = [i64, P, P, P, P, i32, i32, P, i32, P, P, P, P,
                                            P, P, P, P, P, P, P, P, P, P]
            L.orc_mse.argtypes = [i32, P, P, P, P]
            L.orc_dy_dlambda.argtypes = [f64, f64]
            L.orc_dy_dlambda.restype = f64
            L.orc_y_soft.argtypes = [f64, f64]
            L.orc_y_soft.restype = f64
            L.orc_num_threads.restype = i32
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _arr(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


class Model:
    """Model constants shared by every call: stage durations, infectiousness table, Philox key."""

    def __init__(self, tau_EI: int, tau_IR: int, c, seed: int = 0):
        self.tau_EI = int(tau_EI)
        self.tau_IR = int(tau_IR)
        self.L = self.tau_EI + self.tau_IR
        self.c = np.ascontiguousarray(c, dtype=np.float32)
        assert self.c.shape == (self.L,)
        self.seed = int(seed)


def _graph_args(pop, orig_id):
    rowptr = _arr(pop.rowptr, np.uint64)
    col = _arr(pop.col, np.uint32)
    w = _arr(pop.w, np.float32)
    age = _arr(pop.age, np.uint8)
    oid = _arr(orig_id, np.uint32)
    keep = (rowptr, col, w, age, oid)
    return keep, [ctypes.c_int64(pop.n), _p(rowptr), _p(col), _p(w), _p(age), _p(oid)]


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(seed: int, ids, day: int, inst: int = 0, stream: int = 0) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.zeros(ids.size, np.float64)
    lib().orc_uniform_array(seed, ids.size, _p(ids), day, inst, stream, _p(out))
    return out


def hash_words(seed: int, ids, day: int, inst: int = 0, stream: int = 0) -> np.ndarray:
    return np.array([lib().orc_hash(seed, int(i), day, inst, stream) for i in ids], np.uint32)


def select_seeds(n: int, seed: int, inst: int, n_seed: int, orig_id=None) -> np.ndarray:
    oid = _arr(orig_id, np.uint32)
    out = np.zeros(max(n_seed, 1), np.int64)
    rc = lib().orc_select_seeds(n, _p(oid), seed, inst, n_seed, _p(out))
    if rc:
        raise ValueError(f"orc_select_seeds failed ({rc})")
    return out[:n_seed]


def mean_weighted_degree(pop) -> float:
    rowptr = _arr(pop.rowptr, np.uint64)
    w = _arr(pop.w, np.float32)
    return lib().orc_mean_weighted_degree(pop.n, _p(rowptr), _p(w))


def day_hard(pop, model: Model, t: int, R_t: float, S_age, e_in, inst: int = 0, orig_id=None):
    """One synchronous hard day from state ``e_in``; returns e_out, Lam, p, u, newRM, counts, margin."""
    keep, g = _graph_args(pop, orig_id)
    S = _arr(S_age, np.float32)
    e_in = _arr(e_in, np.int16)
    n = pop.n
    e_out = np.zeros(n, np.int16)
    Lam = np.zeros(n); p = np.zeros(n); u = np.zeros(n)
    nrm = np.zeros(1, np.int64); counts = np.zeros(4, np.int64); mg = np.zeros(1)
    Dbar = mean_weighted_degree(pop)
    lib().orc_day_hard(*g, model.tau_EI, model.tau_IR, _p(model.c), model.seed, inst, Dbar, t,
                       float(R_t), _p(S), _p(e_in), _p(e_out), _p(Lam), _p(p), _p(u), _p(nrm),
                       _p(counts), _p(mg))
    return dict(e_out=e_out, Lam=Lam, p=p, u=u, newRM=int(nrm[0]), counts=counts, margin=float(mg[0]))


def forward_hard(pop, model: Model, R, m, S_age, n_seed: int = 0, e0=None, t0: int = 0,
                 inst: int = 0, orig_id=None, want_hist: bool = False, want_Lam: bool = False):
    """Hard forward over days t0..T-1 (T = len(R)).  Returns e_final, D, counts, newRM, margin
    and optionally e_hist [(T+1), n] and Lam_hist [T, n]."""
    keep, g = _graph_args(pop, orig_id)
    R = _arr(R, np.float32); m = _arr(m, np.float32); S = _arr(S_age, np.float32)
    T = int(R.size)
    n = pop.n
    e0 = _arr(e0, np.int16)
    e_final = np.zeros(n, np.int16)
    D = np.zeros(T); counts = np.zeros((T, 4), np.int64); newRM = np.zeros(T, np.int64)
    e_hist = np.zeros((T + 1, n), np.int16) if want_hist else None
    Lam_hist = np.zeros((T, n)) if want_Lam else None
    mg = np.zeros(1)
    rc = lib().orc_forward_hard(*g, model.tau_EI, model.tau_IR, _p(model.c), model.seed, inst, T, t0,
                                _p(R), _p(m), _p(S), n_seed, _p(e0), _p(e_final), _p(D), _p(counts),
                                _p(newRM), _p(e_hist), _p(Lam_hist), _p(mg))
    if rc:
        raise RuntimeError(f"orc_forward_hard failed ({rc})")
    return dict(e_final=e_final, D=D, counts=counts, newRM=newRM, e_hist=e_hist, Lam_hist=Lam_hist,
                margin=float(mg[0]))


def backward_hard(pop, model: Model, R, m, S_age, E, gD, inst: int = 0, orig_id=None, want_gl=False):
    """Hard/straight-through adjoint of the trajectory encoded by the final state ``E``.
    ``dc`` [L] is dL/dc[k], the adjoint of the infectiousness table (dc[0] = 0: c[0] is fixed)."""
    keep, g = _graph_args(pop, orig_id)
    R = _arr(R, np.float32); m = _arr(m, np.float32); S = _arr(S_age, np.float32)
    E = _arr(E, np.int16); gD = _arr(gD, np.float64)
    T = int(R.size)
    dR = np.zeros(T); dm = np.zeros(T); dS = np.zeros(NUM_AGES)
    gl = np.zeros((T, pop.n)) if want_gl else None
    dc = np.zeros(model.tau_EI + model.tau_IR)
    rc = lib().orc_backward_hard(*g, model.tau_EI, model.tau_IR, _p(model.c), model.seed, inst, T,
                                 _p(R), _p(m), _p(S), _p(E), _p(gD), _p(dR), _p(dm), _p(dS), _p(gl),
                                 _p(dc))
    if rc:
        raise RuntimeError(f"orc_backward_hard failed ({rc})")
    return dict(dR=dR, dm=dm, dS=dS, gl=gl, dc=dc)


def forward_soft(pop, model: Model, R, m, S_age, n_seed: int = 0, e0=None, inst: int = 0, orig_id=None):
    """Fixed-noise soft relaxation forward; returns D, newRM and the histories its adjoint needs."""
    keep, g = _graph_args(pop, orig_id)
    R = _arr(R, np.float32); m = _arr(m, np.float32); S = _arr(S_age, np.float32)
    T = int(R.size)
    n = pop.n
    e0 = _arr(e0, np.int16)
    D = np.zeros(T); newRM = np.zeros(T)
    s_hist = np.zeros((T + 1, n)); y_hist = np.zeros((T, n)); dydl = np.zeros((T, n)); Lam = np.zeros((T, n))
    rc = lib().orc_forward_soft(*g, model.tau_EI, model.tau_IR, _p(model.c), model.seed, inst, T,
                                _p(R), _p(m), _p(S), n_seed, _p(e0), _p(D), _p(newRM), _p(s_hist),
                                _p(y_hist), _p(dydl), _p(Lam))
    if rc:
        raise RuntimeError(f"orc_forward_soft failed ({rc})")
    return dict(D=D, newRM=newRM, s_hist=s_hist, y_hist=y_hist, dydl_hist=dydl, Lam_hist=Lam)


def backward_soft(pop, model: Model, R, m, S_age, gD, s_hist, y_hist, dydl_hist, Lam_hist, newRM, e0=None):
    """Adjoint of the relaxed model from its histories (hard values give the ST adjoint).
    ``e0``: the initial exposure days (seeds negative), needed for the seeds' share of
    ``dc`` [L] = dL/dc[k] (dc[0] = 0)."""
    rowptr = _arr(pop.rowptr, np.uint64); col = _arr(pop.col, np.uint32)
    w = _arr(pop.w, np.float32); age = _arr(pop.age, np.uint8)
    R = _arr(R, np.float32); m = _arr(m, np.float32); S = _arr(S_age, np.float32)
    gD = _arr(gD, np.float64)
    arrs = [_arr(a, np.float64) for a in (s_hist, y_hist, dydl_hist, Lam_hist, newRM)]
    T = int(R.size)
    dR = np.zeros(T); dm = np.zeros(T); dS = np.zeros(NUM_AGES)
    dc = np.zeros(model.tau_EI + model.tau_IR)
    e0 = _arr(e0, np.int16)
    rc = lib().orc_backward_soft(pop.n, _p(rowptr), _p(col), _p(w), _p(age), model.tau_EI,
                                 model.tau_IR, _p(model.c), T, _p(R), _p(m), _p(S), _p(gD),
                                 *[_p(a) for a in arrs], _p(dR), _p(dm), _p(dS), _p(e0), _p(dc))
    if rc:
        raise RuntimeError(f"orc_backward_soft failed ({rc})")
    return dict(dR=dR, dm=dm, dS=dS, dc=dc)


def mse(D, y):
    """MSE on daily deaths: loss = mean((D - y)^2), gD = 2 (D - y) / T."""
    D = _arr(D, np.float64); y = _arr(y, np.float64)
    T = int(D.size)
    loss = np.zeros(1); gD = np.zeros(T)
    lib().orc_mse(T, _p(D), _p(y), _p(loss), _p(gD))
    return float(loss[0]), gD


def dy_dlambda(lam: float, u: float) -> float:
    return lib().orc_dy_dlambda(float(lam), float(u))


def y_soft(lam: float, u: float) -> float:
    return lib().orc_y_soft(float(lam), float(u))


def num_threads() -> int:
    return lib().orc_num_threads()
