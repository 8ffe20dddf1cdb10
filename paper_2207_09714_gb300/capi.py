"""Thin Python binding of the C ABI in ``include/gabm.h`` (same function names).

Argument marshalling only: every step of the simulation and of its adjoint
runs in the CUDA library ``_build/libgabm.so``.  Arrays may be CUDA tensors
(the call runs with GABM_DEVICE) or numpy arrays / CPU tensors (GABM_HOST);
one call takes all of its arrays from the same side.  PyTorch is used for
device memory and the CUDA stream.  There is no CPU fallback: if the library
has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgabm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gabm.h")

GABM_OK, GABM_EINVAL, GABM_ENOMEM, GABM_ECUDA, GABM_ESTATE = 0, 1, 2, 3, 4
GABM_ETIMEOUT, GABM_ECANCELLED, GABM_EUNSUPPORTED = 5, 6, 7
GABM_DEVICE, GABM_HOST = 0, 1
GABM_HARD_ST, GABM_SOFT = 0, 1
GABM_STORE_LAMBDA, GABM_RECOMPUTE = 0, 1
GABM_ORDER_INPUT, GABM_ORDER_BFS, GABM_ORDER_COMMUNITY = 0, 1, 2
GABM_NEVER = 32767
GABM_NUM_AGES = 9
STATUS_NAMES = {0: "GABM_OK", 1: "GABM_EINVAL", 2: "GABM_ENOMEM", 3: "GABM_ECUDA", 4: "GABM_ESTATE",
                5: "GABM_ETIMEOUT", 6: "GABM_ECANCELLED", 7: "GABM_EUNSUPPORTED"}


class GabmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _GraphDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("w", ctypes.c_void_p), ("age", ctypes.c_void_p),
                ("mem_space", ctypes.c_int)]


class _BipartiteDesc(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int64), ("n_locations", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("loc", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("age", ctypes.c_void_p)]


class _ModelDesc(ctypes.Structure):
    _fields_ = [("tau_EI", ctypes.c_int), ("tau_IR", ctypes.c_int), ("c", ctypes.c_void_p),
                ("gumbel_tau", ctypes.c_float), ("relax_mode", ctypes.c_int),
                ("lambda_policy", ctypes.c_int), ("seed", ctypes.c_uint64), ("agent_order", ctypes.c_int),
                ("tau_IM", ctypes.c_int), ("p_IR", ctypes.c_void_p), ("tau_RS", ctypes.c_int)]


class _Schedule(ctypes.Structure):
    _fields_ = [("fwd_sets_per_lane", ctypes.c_int), ("bwd_sets_per_lane", ctypes.c_int),
                ("fwd_smem_bitmap", ctypes.c_int), ("bwd_sets_per_launch", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgabm.so (built by ``paper_2207_09714_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run `python -m paper_2207_09714_gb300.build`)")
        L = ctypes.CDLL(path)
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        L.gabm_create.argtypes = [ctypes.POINTER(_GraphDesc), i32, i32, ctypes.POINTER(_ModelDesc), P,
                                  ctypes.POINTER(P)]
        L.gabm_forward.argtypes = [P, i32, P, P, P, P, P, P, i32]
        L.gabm_create_bipartite.argtypes = [ctypes.POINTER(_BipartiteDesc), i32, ctypes.POINTER(_ModelDesc), P,
                                            ctypes.POINTER(P)]
        L.gabm_mse_loss.argtypes = [P, P, P, P, i32]
        L.gabm_backward.argtypes = [P, P, P, P, P, i32]
        L.gabm_backward_table.argtypes = [P, P, P, P, P, P, i32]
        L.gabm_set_infectiousness.argtypes = [P, P]
        L.gabm_get_state.argtypes = [P, P, i32]
        L.gabm_set_state.argtypes = [P, i32, P, i32]
        L.gabm_get_lambda.argtypes = [P, i32, P, i32]
        L.gabm_mem_stats.argtypes = [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
        L.gabm_launch_count.argtypes = [P]
        L.gabm_launch_count.restype = u64
        L.gabm_set_profiling.argtypes = [P, i32]
        L.gabm_get_profile.argtypes = [P, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        L.gabm_philox.argtypes = [u64, P, P, i64, P]
        L.gabm_last_error.argtypes = [P]
        L.gabm_last_error.restype = ctypes.c_char_p
        L.gabm_destroy.argtypes = [P]
        L.gabm_destroy.restype = None
        L.gabm_version.restype = ctypes.c_char_p
        L.gabm_seed_state_noalloc.argtypes = [u64, i64, i32, P, i32, P, P]
        L.gabm_seed_state_noalloc.restype = ctypes.c_int
        L.gabm_noalloc_last_error.restype = ctypes.c_char_p
        L.gabm_get_schedule.argtypes = [P, ctypes.POINTER(_Schedule)]
        L.gabm_set_schedule.argtypes = [P, ctypes.POINTER(_Schedule)]
        L.gabm_autotune.argtypes = [P, i32]
        L.gabm_agent_layout.argtypes = [ctypes.POINTER(_GraphDesc), i32, i32, P]
        for name in ("gabm_create", "gabm_create_bipartite", "gabm_forward", "gabm_mse_loss", "gabm_backward", "gabm_backward_table",
                     "gabm_set_infectiousness",
                     "gabm_get_state",
                     "gabm_set_state", "gabm_get_lambda", "gabm_mem_stats", "gabm_set_profiling",
                     "gabm_get_profile", "gabm_philox", "gabm_get_schedule", "gabm_set_schedule",
                     "gabm_autotune", "gabm_agent_layout"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def header_functions(path: str = HEADER):
    """Names of the functions include/gabm.h declares."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gabm_[a-z_0-9]+)\s*\(", src)))


# --------------------------------------------------------------------------- marshalling
def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _space(*arrays) -> int:
    present = [a for a in arrays if a is not None]
    kinds = {_is_cuda(a) for a in present}
    if len(kinds) > 1:
        raise ValueError("all arrays of one call must be CUDA tensors, or all host arrays")
    return GABM_DEVICE if kinds == {True} else GABM_HOST


def _ptr(x, dtype=None):
    """Pointer to a contiguous array of the given numpy dtype (validated, never converted)."""
    if x is None:
        return None
    if _is_cuda(x) or hasattr(x, "data_ptr"):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                np.int16: torch.int16, np.uint8: torch.uint8, np.uint32: torch.uint32,
                np.uint64: torch.uint64}.get(dtype)
        if want is not None and x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray):
        raise TypeError(f"unsupported array type {type(x)}")
    if dtype is not None and x.dtype != np.dtype(dtype):
        raise TypeError(f"expected {np.dtype(dtype)}, got {x.dtype}")
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _shape(x, want, name):
    if x is not None and tuple(x.shape) != tuple(want):
        raise ValueError(f"{name} must have shape {tuple(want)}, got {tuple(x.shape)}")


def _check(status: int, handle=None):
    if status != GABM_OK:
        msg = load_library().gabm_last_error(handle).decode(errors="replace")
        raise GabmError(status, msg)


def _empty(shape, np_dtype, cuda: bool, device=None):
    if cuda:
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
               np.int16: torch.int16}[np_dtype]
        return torch.empty(shape, dtype=tdt, device=device)
    return np.empty(shape, dtype=np_dtype)


@dataclasses.dataclass
class ModelDesc:
    """Model constants of a ctx (mirrors gabm_model_desc)."""
    tau_EI: int
    tau_IR: int
    c: np.ndarray
    seed: int = 0
    lambda_policy: int = GABM_STORE_LAMBDA
    gumbel_tau: float = 1.0
    relax_mode: int = GABM_HARD_ST
    agent_order: int = GABM_ORDER_COMMUNITY
    tau_IM: int = 0          # > 0: the sampled R/M split (c then has tau_EI + max(tau_IR, tau_IM) entries)
    p_IR: np.ndarray = None  # [tau_IR] pmf of a per-agent I-stage duration 1..tau_IR, or None
    tau_RS: int = 0          # > 0: SIRS reinfection, back to S tau_RS days after entering RM

    @property
    def L(self) -> int:
        return int(self.tau_EI) + max(int(self.tau_IR), int(self.tau_IM))


class GabmCtx:
    """Owning handle of a gabm_ctx (destroyed with the object)."""

    def __init__(self, handle, graphs, sets, model, device, stream):
        self.handle = handle
        self.num_graphs = len(graphs)
        self.sets = sets
        self.instances = len(graphs) * sets
        self.n_per_graph = [int(g.n) for g in graphs]
        self.n_total = sum(self.n_per_graph)
        self.model = model
        self.device = device
        self.stream = stream
        self.T = None
        self._lib = load_library()

    def close(self):
        if self.handle:
            self._lib.gabm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- ABI
def gabm_version() -> str:
    return load_library().gabm_version().decode()


def _model_struct(model: ModelDesc, c: np.ndarray) -> _ModelDesc:
    if c.size != model.L:
        raise ValueError(f"c must have tau_EI + max(tau_IR, tau_IM) = {model.L} entries, got {c.size}")
    p = None
    if model.p_IR is not None:
        p = np.ascontiguousarray(np.asarray(model.p_IR, np.float32).reshape(-1))
        if p.size != int(model.tau_IR):
            raise ValueError(f"p_IR must have tau_IR = {model.tau_IR} entries, got {p.size}")
    md = _ModelDesc(int(model.tau_EI), int(model.tau_IR), _ptr(c, np.float32), float(model.gumbel_tau),
                    int(model.relax_mode), int(model.lambda_policy), int(model.seed), int(model.agent_order),
                    int(model.tau_IM), _ptr(p, np.float32), int(model.tau_RS))
    md._keep = p   # alive for as long as the descriptor
    return md


def gabm_create_bipartite(graphs, model: ModelDesc, stream=None) -> GabmCtx:
    """Create a ctx over agent-location graphs (one, or a list; objects with n, n_loc,
    rowptr [n+1], loc, w, age as host numpy arrays): agents interact through shared
    locations, the pair weight being sum_l w_il w_jl.  One set per graph; store-lambda
    hard mode."""
    L = load_library()
    graphs = list(graphs) if isinstance(graphs, (list, tuple)) else [graphs]
    descs = (_BipartiteDesc * len(graphs))()
    keep = []
    for i, graph in enumerate(graphs):
        rowptr = np.ascontiguousarray(graph.rowptr, np.uint64)
        loc = np.ascontiguousarray(graph.loc, np.uint32)
        w = np.ascontiguousarray(graph.w, np.float32)
        age = np.ascontiguousarray(graph.age, np.uint8)
        keep.append((rowptr, loc, w, age))
        descs[i] = _BipartiteDesc(int(graph.n), int(graph.n_loc), int(loc.shape[0]), _ptr(rowptr, np.uint64),
                                  _ptr(loc, np.uint32), _ptr(w, np.float32), _ptr(age, np.uint8))
    c = np.ascontiguousarray(model.c, dtype=np.float32)
    md = _model_struct(model, c)
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    s = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    device = getattr(stream, "device", None) or torch.device("cuda", torch.cuda.current_device())
    out = ctypes.c_void_p()
    st = L.gabm_create_bipartite(descs, len(graphs), ctypes.byref(md), s, ctypes.byref(out))
    _check(st, None)
    return GabmCtx(out, graphs, 1, model, device, stream)


def gabm_agent_layout(graph, agent_order: int = GABM_ORDER_COMMUNITY, sets_per_graph: int = 1) -> np.ndarray:
    """The device order gabm_create gives one graph's agents (host arrays, host work only):
    order[r] = the caller's id of device row r."""
    rowptr = np.ascontiguousarray(graph.rowptr, np.uint64)
    col = np.ascontiguousarray(graph.col, np.uint32)
    w = np.ascontiguousarray(graph.w, np.float32)
    age = np.ascontiguousarray(graph.age, np.uint8)
    desc = _GraphDesc(int(graph.n), int(col.shape[0]), _ptr(rowptr, np.uint64), _ptr(col, np.uint32),
                      _ptr(w, np.float32), _ptr(age, np.uint8), GABM_HOST)
    out = np.empty(int(graph.n), np.uint32)
    _check(load_library().gabm_agent_layout(ctypes.byref(desc), int(agent_order), int(sets_per_graph),
                                            out.ctypes.data_as(ctypes.c_void_p)), None)
    return out


def gabm_create(graphs, model: ModelDesc, sets_per_graph: int = 1, stream=None) -> GabmCtx:
    """Create a ctx from graphs (objects with n, rowptr, col, w, age) and a ModelDesc."""
    L = load_library()
    keep = []
    descs = (_GraphDesc * max(len(graphs), 1))()
    device = None
    for i, g in enumerate(graphs):
        ms = _space(g.rowptr, g.col, g.w, g.age)
        if ms == GABM_DEVICE:
            device = g.rowptr.device
        descs[i] = _GraphDesc(int(g.n), int(g.col.shape[0]), _ptr(g.rowptr, np.uint64), _ptr(g.col, np.uint32),
                              _ptr(g.w, np.float32), _ptr(g.age, np.uint8), ms)
        keep.append(g)
    c = np.ascontiguousarray(model.c, dtype=np.float32)
    md = _model_struct(model, c)
    s = None
    if stream is not None:
        s = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        device = device or getattr(stream, "device", None)
    try:
        import torch
        if torch.cuda.is_available():
            if stream is None:
                stream = torch.cuda.current_stream()
                s = ctypes.c_void_p(stream.cuda_stream)
            device = device or torch.device("cuda", torch.cuda.current_device())
    except ImportError:
        pass
    out = ctypes.c_void_p()
    st = L.gabm_create(descs, len(graphs), int(sets_per_graph), ctypes.byref(md), s, ctypes.byref(out))
    _check(st, None)
    return GabmCtx(out, graphs, int(sets_per_graph), model, device, stream)


def gabm_forward(ctx: GabmCtx, T: int, R, m, S_age, n_seed=None, D=None, counts=None, want_counts=False):
    """Run the forward over T days; returns (D [I,T] float64, counts [I,T,4] int32 or None)."""
    ms = _space(R, m, S_age, D, counts)
    cuda = ms == GABM_DEVICE
    I = ctx.instances
    _shape(R, (I, T), "R")
    _shape(m, (I, T), "m")
    _shape(S_age, (I, GABM_NUM_AGES), "S_age")
    _shape(D, (I, T), "D")
    _shape(counts, (I, T, 4), "counts")
    if D is None:
        D = _empty((I, T), np.float64, cuda, ctx.device)
    if counts is None and want_counts:
        counts = _empty((I, T, 4), np.int32, cuda, ctx.device)
    seeds = None
    if n_seed is not None:
        seeds = np.ascontiguousarray(np.broadcast_to(np.asarray(n_seed, dtype=np.int32), (I,)))
    st = load_library().gabm_forward(ctx.handle, int(T), _ptr(R, np.float32), _ptr(m, np.float32),
                                     _ptr(S_age, np.float32), _ptr(seeds, np.int32), _ptr(D, np.float64),
                                     _ptr(counts, np.int32), ms)
    _check(st, ctx.handle)
    ctx.T = int(T)
    return D, counts


def gabm_mse_loss(ctx: GabmCtx, y, loss=None, gD=None):
    """MSE of the last forward's daily deaths against y [I,T]; returns (loss [I], gD [I,T])."""
    ms = _space(y, loss, gD)
    cuda = ms == GABM_DEVICE
    I, T = ctx.instances, (ctx.T if ctx.T is not None else int(y.shape[-1]))
    _shape(y, (I, T), "y")
    _shape(loss, (I,), "loss")
    _shape(gD, (I, T), "gD")
    if loss is None:
        loss = _empty((I,), np.float64, cuda, ctx.device)
    if gD is None:
        gD = _empty((I, T), np.float64, cuda, ctx.device)
    st = load_library().gabm_mse_loss(ctx.handle, _ptr(y, np.float64), _ptr(loss, np.float64),
                                      _ptr(gD, np.float64), ms)
    _check(st, ctx.handle)
    return loss, gD


def gabm_backward(ctx: GabmCtx, gD, dR=None, dm=None, dS_age=None):
    """Straight-through adjoint; returns (dR [I,T], dm [I,T], dS_age [I,9]) in float64."""
    ms = _space(gD, dR, dm, dS_age)
    cuda = ms == GABM_DEVICE
    I, T = ctx.instances, (ctx.T if ctx.T is not None else int(gD.shape[-1]))
    _shape(gD, (I, T), "gD")
    _shape(dR, (I, T), "dR")
    _shape(dm, (I, T), "dm")
    _shape(dS_age, (I, GABM_NUM_AGES), "dS_age")
    if dR is None:
        dR = _empty((I, T), np.float64, cuda, ctx.device)
    if dm is None:
        dm = _empty((I, T), np.float64, cuda, ctx.device)
    if dS_age is None:
        dS_age = _empty((I, GABM_NUM_AGES), np.float64, cuda, ctx.device)
    st = load_library().gabm_backward(ctx.handle, _ptr(gD, np.float64), _ptr(dR, np.float64),
                                      _ptr(dm, np.float64), _ptr(dS_age, np.float64), ms)
    _check(st, ctx.handle)
    return dR, dm, dS_age


def gabm_backward_table(ctx: GabmCtx, gD, dR=None, dm=None, dS_age=None, dc=None):
    """``gabm_backward`` plus the adjoint of the infectiousness table; returns
    (dR [I,T], dm [I,T], dS_age [I,9], dc [I,L]) in float64 (dc[:, 0] = 0)."""
    ms = _space(gD, dR, dm, dS_age, dc)
    cuda = ms == GABM_DEVICE
    I, T = ctx.instances, (ctx.T if ctx.T is not None else int(gD.shape[-1]))
    L = ctx.model.L
    _shape(gD, (I, T), "gD")
    _shape(dR, (I, T), "dR")
    _shape(dm, (I, T), "dm")
    _shape(dS_age, (I, GABM_NUM_AGES), "dS_age")
    _shape(dc, (I, L), "dc")
    if dR is None:
        dR = _empty((I, T), np.float64, cuda, ctx.device)
    if dm is None:
        dm = _empty((I, T), np.float64, cuda, ctx.device)
    if dS_age is None:
        dS_age = _empty((I, GABM_NUM_AGES), np.float64, cuda, ctx.device)
    if dc is None:
        dc = _empty((I, L), np.float64, cuda, ctx.device)
    st = load_library().gabm_backward_table(ctx.handle, _ptr(gD, np.float64), _ptr(dR, np.float64),
                                            _ptr(dm, np.float64), _ptr(dS_age, np.float64),
                                            _ptr(dc, np.float64), ms)
    _check(st, ctx.handle)
    return dR, dm, dS_age, dc


def gabm_set_infectiousness(ctx: GabmCtx, c):
    """Replace the model's infectiousness table c [L] (c[0] = 0) for the following forwards."""
    L = ctx.model.L
    c = np.ascontiguousarray(np.asarray(c, np.float32).reshape(-1))
    if c.size != L:
        raise ValueError(f"c must have {L} entries, got {c.size}")
    st = load_library().gabm_set_infectiousness(ctx.handle, c.ctypes.data_as(ctypes.c_void_p))
    _check(st, ctx.handle)
    ctx.model = dataclasses.replace(ctx.model, c=c.copy())


def gabm_get_state(ctx: GabmCtx, out=None, device: bool = False):
    """Exposure days [sets, n_total] int16 (host numpy unless device=True or out is a CUDA tensor)."""
    cuda = _is_cuda(out) if out is not None else device
    if out is None:
        out = _empty((ctx.sets, ctx.n_total), np.int16, cuda, ctx.device)
    st = load_library().gabm_get_state(ctx.handle, _ptr(out, np.int16), GABM_DEVICE if cuda else GABM_HOST)
    _check(st, ctx.handle)
    return out


def gabm_set_state(ctx: GabmCtx, day: int, e):
    if tuple(e.shape) not in ((ctx.sets, ctx.n_total),) + (((ctx.n_total,),) if ctx.sets == 1 else ()):
        raise ValueError(f"e must have shape ({ctx.sets}, {ctx.n_total}), got {tuple(e.shape)}")
    st = load_library().gabm_set_state(ctx.handle, int(day), _ptr(e, np.int16), _space(e))
    _check(st, ctx.handle)


def gabm_get_lambda(ctx: GabmCtx, t: int, out=None, device: bool = False):
    cuda = _is_cuda(out) if out is not None else device
    if out is None:
        out = _empty((ctx.sets, ctx.n_total), np.float32, cuda, ctx.device)
    st = load_library().gabm_get_lambda(ctx.handle, int(t), _ptr(out, np.float32), GABM_DEVICE if cuda else GABM_HOST)
    _check(st, ctx.handle)
    return out


def gabm_mem_stats(ctx: GabmCtx):
    cur, peak = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load_library().gabm_mem_stats(ctx.handle, ctypes.byref(cur), ctypes.byref(peak)), ctx.handle)
    return int(cur.value), int(peak.value)


def gabm_get_schedule(ctx: GabmCtx) -> dict:
    sc = _Schedule()
    _check(load_library().gabm_get_schedule(ctx.handle, ctypes.byref(sc)), ctx.handle)
    return {k: int(getattr(sc, k)) for k, _ in _Schedule._fields_}


def gabm_set_schedule(ctx: GabmCtx, fwd_sets_per_lane=0, bwd_sets_per_lane=0, fwd_smem_bitmap=0,
                      bwd_sets_per_launch=0):
    sc = _Schedule(int(fwd_sets_per_lane), int(bwd_sets_per_lane), int(fwd_smem_bitmap), int(bwd_sets_per_launch))
    _check(load_library().gabm_set_schedule(ctx.handle, ctypes.byref(sc)), ctx.handle)


def gabm_autotune(ctx: GabmCtx, repetitions: int = 1) -> dict:
    """Time every schedule on the last forward's workload, keep the fastest; returns it."""
    _check(load_library().gabm_autotune(ctx.handle, int(repetitions)), ctx.handle)
    return gabm_get_schedule(ctx)


def gabm_create_order_tuned(graphs, model: ModelDesc, R, m, S_age, n_seed, sets_per_graph: int = 1,
                            stream=None, orders=(GABM_ORDER_COMMUNITY, GABM_ORDER_BFS), repetitions: int = 2):
    """gabm_create with the device layout of the agents chosen by timing: a ctx is built for
    each agent order in `orders` (the model's own agent_order is ignored), each runs this
    workload's forward (R, m, S_age as gabm_forward takes them, n_seed per instance) and a
    backward with dL/dD = 1 once untimed and then `repetitions` times under CUDA events on
    the ctx stream; the fastest ctx is returned and the others are destroyed.  Results do
    not depend on the order beyond fp32 summation order (ids stay the caller's), so the
    choice is free.  Returns (ctx, {order: ms per forward + backward})."""
    import dataclasses
    import torch
    T = int(R.shape[-1])
    best, best_ms, times = None, None, {}
    for order in orders:
        ctx = gabm_create(graphs, dataclasses.replace(model, agent_order=int(order)), sets_per_graph, stream)
        s = ctx.stream
        if not hasattr(s, "cuda_stream"):
            s = torch.cuda.ExternalStream(int(s)) if s is not None else torch.cuda.current_stream()
        gD = None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(1 + repetitions):
            if rep == 1:
                e0.record(s)
            D, _ = gabm_forward(ctx, T, R, m, S_age, n_seed)
            if gD is None:
                gD = torch.ones_like(D)
            gabm_backward(ctx, gD)
        e1.record(s)
        e1.synchronize()
        times[int(order)] = e0.elapsed_time(e1) / repetitions
        if best is None or times[int(order)] < best_ms:
            if best is not None:
                gabm_destroy(best)
            best, best_ms = ctx, times[int(order)]
        else:
            gabm_destroy(ctx)
    return best, times


def gabm_launch_count(ctx: GabmCtx) -> int:
    return int(load_library().gabm_launch_count(ctx.handle))


def gabm_set_profiling(ctx: GabmCtx, enable: bool):
    _check(load_library().gabm_set_profiling(ctx.handle, int(bool(enable))), ctx.handle)


def gabm_get_profile(ctx: GabmCtx, kind: int):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load_library().gabm_get_profile(ctx.handle, int(kind), ctypes.byref(ms), ctypes.byref(n)), ctx.handle)
    return float(ms.value), int(n.value)


def gabm_philox(seed: int, ctr, out=None, stream=None):
    """Device Philox4x32-10 on counters ctr [count, 4] (uint32 CUDA tensor)."""
    import torch
    if out is None:
        out = torch.empty_like(ctr)
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    st = load_library().gabm_philox(int(seed), _ptr(ctr, np.uint32), _ptr(out, np.uint32), int(ctr.shape[0]), s)
    _check(st, None)
    return out


def gabm_destroy(ctx: GabmCtx):
    ctx.close()


def gabm_seed_state_noalloc(seed: int, n: int, n_seed, tau_EI: int, e_out, stream=None):
    """Day-0 state of len(n_seed) instances into e_out [instances, n] (int16 CUDA tensor the
    caller allocated).  The library allocates nothing for this call."""
    import torch
    seeds = np.ascontiguousarray(np.asarray(n_seed, dtype=np.int32).reshape(-1))
    if not _is_cuda(e_out):
        raise ValueError("e_out must be a CUDA tensor")
    _shape(e_out, (seeds.size, int(n)), "e_out")
    # the C side works on the current device's scratch: make e_out's device current
    with torch.cuda.device(e_out.device):
        strm = stream or torch.cuda.current_stream()
        if strm.device != e_out.device:
            raise ValueError("stream and e_out must be on the same device")
        st = load_library().gabm_seed_state_noalloc(int(seed), int(n), int(seeds.size), _ptr(seeds, np.int32),
                                                    int(tau_EI), _ptr(e_out, np.int16),
                                                    ctypes.c_void_p(strm.cuda_stream))
    if st != GABM_OK:
        raise GabmError(st, load_library().gabm_noalloc_last_error().decode(errors="replace"))
    return e_out
