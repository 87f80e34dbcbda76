"""GB300-native PCDN (Parallel Coordinate Descent Newton, arXiv:1306.4080) for L1-regularised
logistic regression and L2-loss SVM.

This module is a thin ctypes binding of the C ABI declared in ``include/pcdn.h``: every
function here has the C name, marshals its arguments (numpy host arrays or device pointers
from PyTorch tensors) and calls ``libpcdn.so``.  All arithmetic of the method runs in that
library's CUDA kernels.  There is no CPU fallback: if the library is not built, or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcdn.so")

PCDN_OK = 0
PCDN_EINVAL = -1
PCDN_ENOMEM = -2
PCDN_ECUDA = -3
PCDN_ENUMERIC = -4
PCDN_ETIMEOUT = -5
PCDN_ENOTCONVERGED = 1

LOSSES = {"logistic": 0, "l2svm": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
LAYOUTS = {"auto": 0, "scatter": 1, "rows": 2}
LAYOUT_NAMES = {v: k for k, v in LAYOUTS.items()}

SYMBOLS = ["pcdn_default_opts", "pcdn_create", "pcdn_create_device", "pcdn_solve", "pcdn_bundle_step",
           "pcdn_set_w", "pcdn_get_w", "pcdn_objective", "pcdn_kkt", "pcdn_permutation", "pcdn_memory",
           "pcdn_destroy", "pcdn_last_error", "pcdn_objective_noalloc", "pcdn_set_C", "pcdn_set_penalty",
           "pcdn_default_batch_opts", "pcdn_solve_batch", "pcdn_autotune", "pcdn_default_server_opts",
           "pcdn_server_create", "pcdn_server_submit", "pcdn_server_submit_borrowed", "pcdn_server_wait", "pcdn_server_stats",
           "pcdn_server_destroy"]
PCDN_NOALLOC_MAX_SAMPLES = 262144


_NOT_FINISHED = -12345  # a status no call returns


class PcdnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pcdn error {code}: {msg}")
        self.code = code


class pcdn_csc(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("n_features", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class pcdn_opts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("nu", ctypes.c_double), ("q_max", ctypes.c_int32), ("ls_batch", ctypes.c_int32),
                ("max_epochs", ctypes.c_int64), ("prec", ctypes.c_int), ("warm_start", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("refresh", ctypes.c_int32), ("spin_limit", ctypes.c_uint32),
                ("shrink", ctypes.c_int32), ("epoch0", ctypes.c_int64), ("kkt_ref", ctypes.c_double),
                ("layout", ctypes.c_int32)]


class pcdn_stats(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int64), ("bundles", ctypes.c_int64), ("coord_updates", ctypes.c_int64),
                ("ls_steps", ctypes.c_int64), ("ls_cap_hits", ctypes.c_int64), ("ls_passes", ctypes.c_int64),
                ("nnz_visited", ctypes.c_int64), ("rows_touched", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("F_final", ctypes.c_double), ("kkt_rel", ctypes.c_double),
                ("kkt0", ctypes.c_double), ("wall_s", ctypes.c_double), ("walk_s", ctypes.c_double),
                ("bytes_model", ctypes.c_double), ("converged", ctypes.c_int32), ("walk_grid", ctypes.c_int32)]


class pcdn_trace(ctypes.Structure):
    _fields_ = [("bundle_cap", ctypes.c_int64), ("q", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("Delta", ctypes.c_void_p), ("dF", ctypes.c_void_p), ("epoch_cap", ctypes.c_int64),
                ("epoch_kkt", ctypes.c_void_p), ("epoch_features", ctypes.c_void_p)]


class pcdn_batch_job(ctypes.Structure):
    _fields_ = [("prob", ctypes.c_void_p), ("P", ctypes.c_int32), ("eps", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_C", ctypes.c_int32), ("C_path", ctypes.c_void_p), ("w_out", ctypes.c_void_p),
                ("stats", ctypes.c_void_p), ("status", ctypes.c_int32), ("P_used", ctypes.c_int32),
                ("layout_used", ctypes.c_int32)]


class pcdn_batch_opts(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("threads", ctypes.c_int32), ("probe_eps", ctypes.c_double),
                ("probe_epochs", ctypes.c_int32), ("n_candidates", ctypes.c_int32), ("candidates", ctypes.c_void_p),
                ("no_graphs", ctypes.c_int32), ("tune_layout", ctypes.c_int32)]


class pcdn_batch_stats(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("solves", ctypes.c_int64), ("probe_solves", ctypes.c_int64),
                ("epochs", ctypes.c_int64), ("coord_updates", ctypes.c_int64), ("bytes_model", ctypes.c_double),
                ("graph_solves", ctypes.c_int64), ("retries", ctypes.c_int64)]


class pcdn_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("hbm_budget", ctypes.c_int64), ("solve", pcdn_opts)]


class pcdn_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("bytes", ctypes.c_int64),
                ("stats", pcdn_stats), ("P_used", ctypes.c_int32), ("retries", ctypes.c_int32)]


_lib = None


def load() -> ctypes.CDLL:
    """Load ``libpcdn.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"` "
                          "or `python paper_1306_4080_gb300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    lib.pcdn_default_opts.argtypes = [P(pcdn_opts)]
    lib.pcdn_default_opts.restype = None
    lib.pcdn_create.argtypes = [P(pcdn_csc), vp, d, ctypes.c_int, P(vp)]
    lib.pcdn_create.restype = ctypes.c_int
    lib.pcdn_create_device.argtypes = [P(pcdn_csc), vp, d, ctypes.c_int, vp, P(vp)]
    lib.pcdn_create_device.restype = ctypes.c_int
    lib.pcdn_solve.argtypes = [vp, i32, d, ctypes.c_uint64, P(pcdn_opts), vp, P(pcdn_stats), P(pcdn_trace)]
    lib.pcdn_solve.restype = ctypes.c_int
    lib.pcdn_bundle_step.argtypes = [vp, vp, vp, i32, P(pcdn_opts), vp, vp, vp, P(d), P(i32), P(d), P(d)]
    lib.pcdn_bundle_step.restype = ctypes.c_int
    lib.pcdn_set_w.argtypes = [vp, vp]
    lib.pcdn_set_w.restype = ctypes.c_int
    lib.pcdn_get_w.argtypes = [vp, vp]
    lib.pcdn_get_w.restype = ctypes.c_int
    lib.pcdn_objective.argtypes = [vp, P(d)]
    lib.pcdn_objective.restype = ctypes.c_int
    lib.pcdn_kkt.argtypes = [vp, P(d)]
    lib.pcdn_kkt.restype = ctypes.c_int
    lib.pcdn_permutation.argtypes = [vp, ctypes.c_uint64, i64, vp]
    lib.pcdn_permutation.restype = ctypes.c_int
    lib.pcdn_memory.argtypes = [vp, P(i64)]
    lib.pcdn_memory.restype = ctypes.c_int
    lib.pcdn_destroy.argtypes = [vp]
    lib.pcdn_destroy.restype = None
    lib.pcdn_last_error.argtypes = []
    lib.pcdn_last_error.restype = ctypes.c_char_p
    lib.pcdn_objective_noalloc.argtypes = [P(pcdn_csc), vp, d, ctypes.c_int, vp, vp, vp]
    lib.pcdn_objective_noalloc.restype = ctypes.c_int
    lib.pcdn_set_C.argtypes = [vp, d]
    lib.pcdn_set_C.restype = ctypes.c_int
    lib.pcdn_set_penalty.argtypes = [vp, d, d]
    lib.pcdn_set_penalty.restype = ctypes.c_int
    lib.pcdn_default_batch_opts.argtypes = [P(pcdn_batch_opts)]
    lib.pcdn_default_batch_opts.restype = None
    lib.pcdn_solve_batch.argtypes = [vp, i32, P(pcdn_opts), P(pcdn_batch_opts), P(pcdn_batch_stats)]
    lib.pcdn_solve_batch.restype = ctypes.c_int
    lib.pcdn_autotune.argtypes = [vp, vp, i32, d, i32, ctypes.c_uint64, P(pcdn_opts), P(i32), vp]
    lib.pcdn_autotune.restype = ctypes.c_int
    lib.pcdn_default_server_opts.argtypes = [P(pcdn_server_opts)]
    lib.pcdn_default_server_opts.restype = None
    lib.pcdn_server_create.argtypes = [P(pcdn_server_opts), P(vp)]
    lib.pcdn_server_create.restype = ctypes.c_int
    lib.pcdn_server_submit.argtypes = [vp, P(pcdn_csc), vp, d, ctypes.c_int, i32, d, ctypes.c_uint64, P(i64)]
    lib.pcdn_server_submit.restype = ctypes.c_int
    lib.pcdn_server_submit_borrowed.argtypes = lib.pcdn_server_submit.argtypes
    lib.pcdn_server_submit_borrowed.restype = ctypes.c_int
    lib.pcdn_server_wait.argtypes = [vp, i64, d, vp, P(pcdn_request_info)]
    lib.pcdn_server_wait.restype = ctypes.c_int
    lib.pcdn_server_stats.argtypes = [vp, P(i64), P(i64), P(i32), P(i64)]
    lib.pcdn_server_stats.restype = ctypes.c_int
    lib.pcdn_server_destroy.argtypes = [vp]
    lib.pcdn_server_destroy.restype = None
    _lib = lib
    return lib


def pcdn_last_error() -> str:
    return load().pcdn_last_error().decode()


def _check(rc: int, ok=(PCDN_OK,)) -> int:
    if rc not in ok:
        raise PcdnError(rc, pcdn_last_error())
    return rc


def pcdn_default_opts(**overrides) -> pcdn_opts:
    o = pcdn_opts()
    load().pcdn_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "prec" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "layout" and isinstance(v, str):
            v = LAYOUTS[v]
        setattr(o, k, v)
    return o


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def pcdn_create(col_ptr, row_idx, val, y, C: float, loss: str = "logistic") -> int:
    """Copy host CSC X and labels y to the device; returns an opaque problem handle."""
    lib = load()
    cp, ri, vv, yy = _host(col_ptr, np.int64), _host(row_idx, np.int32), _host(val, np.float32), _host(y, np.int8)
    X = pcdn_csc(int(yy.shape[0]), int(cp.shape[0] - 1), int(ri.shape[0]), cp.ctypes.data, ri.ctypes.data,
                 vv.ctypes.data)
    h = ctypes.c_void_p()
    _check(lib.pcdn_create(ctypes.byref(X), yy.ctypes.data, float(C), LOSSES[loss], ctypes.byref(h)))
    return h.value


def pcdn_create_device(col_ptr, row_idx, val, y, C: float, loss: str = "logistic", stream=None) -> int:
    """Device-resident inputs (PyTorch CUDA tensors: int64, int32, float32, int8); the caller keeps
    them alive until pcdn_destroy.  ``stream`` is a torch.cuda.Stream or raw handle (None: own)."""
    lib = load()
    n, m, nnz = int(y.shape[0]), int(col_ptr.shape[0] - 1), int(row_idx.shape[0])
    for t, dt in ((col_ptr, "torch.int64"), (row_idx, "torch.int32"), (val, "torch.float32"), (y, "torch.int8")):
        if str(t.dtype) != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA tensor of {dt}, got {t.dtype} on {t.device}")
    X = pcdn_csc(n, m, nnz, col_ptr.data_ptr(), row_idx.data_ptr(), val.data_ptr())
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    h = ctypes.c_void_p()
    _check(lib.pcdn_create_device(ctypes.byref(X), y.data_ptr(), float(C), LOSSES[loss], s, ctypes.byref(h)))
    return h.value


def pcdn_destroy(h: int) -> None:
    if h:
        load().pcdn_destroy(h)


def pcdn_solve(h: int, P: int, eps: float = 1e-3, seed: int = 0, opts: pcdn_opts | None = None,
               n_features: int | None = None, want_w: bool = True, trace_bundles: int = 0, trace_epochs: int = 0):
    """Algorithm 3 to relative KKT ``eps``.  Returns (status, w or None, stats dict, trace dict)."""
    lib = load()
    o = opts if opts is not None else pcdn_default_opts()
    w = None
    if want_w:
        if n_features is None:
            raise ValueError("n_features is needed to receive w")
        w = np.empty(int(n_features), dtype=np.float64)
    st = pcdn_stats()
    tr = None
    arrs = {}
    if trace_bundles or trace_epochs:
        arrs = dict(q=np.zeros(trace_bundles, np.int32), alpha=np.zeros(trace_bundles), Delta=np.zeros(trace_bundles),
                    dF=np.zeros(trace_bundles), epoch_kkt=np.zeros(trace_epochs),
                    epoch_features=np.zeros(trace_epochs, np.int64))
        tr = pcdn_trace(trace_bundles, arrs["q"].ctypes.data, arrs["alpha"].ctypes.data, arrs["Delta"].ctypes.data,
                        arrs["dF"].ctypes.data, trace_epochs, arrs["epoch_kkt"].ctypes.data,
                        arrs["epoch_features"].ctypes.data)
    rc = lib.pcdn_solve(h, int(P), float(eps), int(seed) & (2**64 - 1), ctypes.byref(o),
                        w.ctypes.data if w is not None else None, ctypes.byref(st),
                        ctypes.byref(tr) if tr is not None else None)
    _check(rc, ok=(PCDN_OK, PCDN_ENOTCONVERGED))
    stats = {f: getattr(st, f) for f, _ in pcdn_stats._fields_}
    stats["status"] = rc
    if arrs:
        nb = min(int(stats["bundles"]), trace_bundles)
        ne = min(int(stats["epochs"]), trace_epochs)
        arrs = {k: (v[:ne] if k.startswith("epoch_") else v[:nb]) for k, v in arrs.items()}
    return rc, w, stats, arrs


def pcdn_bundle_step(h: int, w_in, bundle, opts: pcdn_opts | None = None):
    """One inner iteration on ``bundle``; returns a dict of g, h, d, Delta, q, alpha, dF."""
    lib = load()
    o = opts if opts is not None else pcdn_default_opts()
    B = _host(bundle, np.int32)
    P = int(B.shape[0])
    wp = None
    if w_in is not None:
        wv = _host(w_in, np.float64)
        wp = wv.ctypes.data
    g, hh, d = np.empty(P), np.empty(P), np.empty(P)
    Delta, alpha, dF = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    q = ctypes.c_int32()
    _check(lib.pcdn_bundle_step(h, wp, B.ctypes.data, P, ctypes.byref(o), g.ctypes.data, hh.ctypes.data, d.ctypes.data,
                                ctypes.byref(Delta), ctypes.byref(q), ctypes.byref(alpha), ctypes.byref(dF)))
    return dict(g=g, h=hh, d=d, Delta=Delta.value, q=q.value, alpha=alpha.value, dF=dF.value)


def pcdn_set_w(h: int, w) -> None:
    wv = _host(w, np.float64)
    _check(load().pcdn_set_w(h, wv.ctypes.data))


def pcdn_get_w(h: int, n_features: int) -> np.ndarray:
    w = np.empty(int(n_features), dtype=np.float64)
    _check(load().pcdn_get_w(h, w.ctypes.data))
    return w


def pcdn_objective(h: int) -> float:
    F = ctypes.c_double()
    _check(load().pcdn_objective(h, ctypes.byref(F)))
    return F.value


def pcdn_kkt(h: int) -> float:
    k = ctypes.c_double()
    _check(load().pcdn_kkt(h, ctypes.byref(k)))
    return k.value


def pcdn_permutation(h: int, seed: int, epoch: int, n_features: int) -> np.ndarray:
    perm = np.empty(int(n_features), dtype=np.int32)
    _check(load().pcdn_permutation(h, int(seed) & (2**64 - 1), int(epoch), perm.ctypes.data))
    return perm


def pcdn_objective_noalloc(col_ptr, row_idx, val, y, C: float, loss: str, w, F, stream=None) -> None:
    """F(w) into the one-element device tensor F from device tensors, allocating nothing on the
    device (see include/pcdn.h).  Enqueues on ``stream`` (torch.cuda.Stream, raw handle or None)."""
    lib = load()
    for t, dt, name in ((col_ptr, "torch.int64", "col_ptr"), (row_idx, "torch.int32", "row_idx"),
                        (val, "torch.float32", "val"), (y, "torch.int8", "y"), (w, "torch.float64", "w"),
                        (F, "torch.float64", "F")):
        # the C side receives raw device pointers and cannot check them: every tensor is checked here
        if not (getattr(t, "is_cuda", False) and str(t.dtype) == dt and t.is_contiguous()):
            raise PcdnError(PCDN_EINVAL, f"{name} must be a contiguous CUDA tensor of {dt}")
    if int(w.numel()) != int(col_ptr.numel()) - 1 or int(F.numel()) < 1 or int(row_idx.numel()) != int(val.numel()):
        raise PcdnError(PCDN_EINVAL, "w must hold n_features = col_ptr.numel() - 1 values, F at least one, "
                                     "row_idx and val the same count")
    X = pcdn_csc(int(y.shape[0]), int(col_ptr.shape[0] - 1), int(row_idx.shape[0]), col_ptr.data_ptr(),
                 row_idx.data_ptr(), val.data_ptr())
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.pcdn_objective_noalloc(ctypes.byref(X), y.data_ptr(), float(C), LOSSES[loss], w.data_ptr(),
                                      F.data_ptr(), s))


def pcdn_set_C(h: int, C: float) -> None:
    _check(load().pcdn_set_C(h, float(C)))


def pcdn_set_penalty(h: int, l1: float = 1.0, l2: float = 0.0) -> None:
    """Penalty l1 ||w||_1 + (l2/2) ||w||^2 (the paper's problem: l1 = 1, l2 = 0)."""
    _check(load().pcdn_set_penalty(h, float(l1), float(l2)))


def pcdn_default_batch_opts(**overrides) -> pcdn_batch_opts:
    o = pcdn_batch_opts()
    load().pcdn_default_batch_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _stats_dict(st: pcdn_stats) -> dict:
    return {f: getattr(st, f) for f, _ in pcdn_stats._fields_}


def pcdn_solve_batch(handles, n_features, C_paths, P, eps=1e-3, seed=0, opts: pcdn_opts | None = None,
                     bopts: pcdn_batch_opts | None = None, want_w: bool = True):
    """Solve many problems concurrently, each along its C path (warm-started).  ``P`` is one bundle
    size for all jobs or a list (0 = autotuned).  Returns (status, per-job list of dicts with
    status, P_used, w [n_C, n_features] or None, stats list) and the batch statistics."""
    lib = load()
    J = len(handles)
    Ps = list(P) if hasattr(P, "__len__") else [int(P)] * J
    seeds = list(seed) if hasattr(seed, "__len__") else [int(seed)] * J
    jobs = (pcdn_batch_job * max(J, 1))()
    keep = []
    outs = []
    for k in range(J):
        cp = _host(C_paths[k], np.float64)
        nC = int(cp.shape[0])
        w = np.empty((nC, int(n_features[k])), dtype=np.float64) if want_w else None
        st = (pcdn_stats * nC)()
        keep += [cp, w, st]
        jobs[k] = pcdn_batch_job(handles[k], int(Ps[k]), float(eps), int(seeds[k]) & (2**64 - 1), nC, cp.ctypes.data,
                                 w.ctypes.data if w is not None else None, ctypes.cast(st, ctypes.c_void_p), 0, 0)
        outs.append((w, st, nC))
    o = opts if opts is not None else pcdn_default_opts()
    bo = bopts if bopts is not None else pcdn_default_batch_opts()
    bs = pcdn_batch_stats()
    rc = lib.pcdn_solve_batch(jobs, J, ctypes.byref(o), ctypes.byref(bo), ctypes.byref(bs))
    _check(rc, ok=(PCDN_OK, PCDN_ENOTCONVERGED))
    res = []
    for k in range(J):
        w, st, nC = outs[k]
        res.append(dict(status=jobs[k].status, P_used=jobs[k].P_used, layout_used=LAYOUT_NAMES[jobs[k].layout_used],
                        w=w, stats=[_stats_dict(st[i]) for i in range(nC)]))
    return rc, res, {f: getattr(bs, f) for f, _ in pcdn_batch_stats._fields_}


def pcdn_autotune(h: int, candidates=None, probe_eps: float = 0.1, probe_epochs: int = 3, seed: int = 0,
                    opts: pcdn_opts | None = None):
    """The bundle-size autotuner on one problem; returns (P_best, list of (P, score))."""
    lib = load()
    cand = None if candidates is None else _host(candidates, np.int32)
    n = 0 if cand is None else int(cand.shape[0])
    scores = np.zeros(max(n, 16))
    Pb = ctypes.c_int32()
    o = opts if opts is not None else pcdn_default_opts()
    _check(lib.pcdn_autotune(h, cand.ctypes.data if cand is not None else None, n, float(probe_eps), int(probe_epochs),
                               int(seed) & (2**64 - 1), ctypes.byref(o), ctypes.byref(Pb), scores.ctypes.data))
    return Pb.value, scores


class Server:
    """Request server (continuous batching on one GPU); see include/pcdn.h."""

    def __init__(self, slots: int = 0, hbm_budget: int = 0, opts: pcdn_opts | None = None):
        lib = load()
        so = pcdn_server_opts()
        lib.pcdn_default_server_opts(ctypes.byref(so))
        so.slots = int(slots)
        if hbm_budget:
            so.hbm_budget = int(hbm_budget)
        if opts is not None:
            so.solve = opts
        h = ctypes.c_void_p()
        _check(lib.pcdn_server_create(ctypes.byref(so), ctypes.byref(h)))
        self.handle = h.value
        self._nf = {}
        self._keep = {}

    def submit(self, col_ptr, row_idx, val, y, C: float, loss: str, P: int, eps: float = 1e-3, seed: int = 0,
               borrow: bool = False) -> int:
        """Queue a solve; with ``borrow`` the arrays are not copied and are kept referenced here
        until the result is collected."""
        cp, ri, vv, yy = _host(col_ptr, np.int64), _host(row_idx, np.int32), _host(val, np.float32), _host(y, np.int8)
        X = pcdn_csc(int(yy.shape[0]), int(cp.shape[0] - 1), int(ri.shape[0]), cp.ctypes.data, ri.ctypes.data,
                     vv.ctypes.data)
        t = ctypes.c_int64()
        fn = load().pcdn_server_submit_borrowed if borrow else load().pcdn_server_submit
        _check(fn(self.handle, ctypes.byref(X), yy.ctypes.data, float(C), LOSSES[loss], int(P), float(eps),
                  int(seed) & (2**64 - 1), ctypes.byref(t)))
        self._nf[t.value] = int(cp.shape[0] - 1)
        if borrow:
            self._keep[t.value] = (cp, ri, vv, yy)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 0.0):
        """Returns (status, w, info dict)."""
        nf = self._nf[ticket]
        w = np.empty(nf, dtype=np.float64)
        info = pcdn_request_info()
        info.status = _NOT_FINISHED  # written by the library only for a finished request
        rc = load().pcdn_server_wait(self.handle, int(ticket), float(timeout_s), w.ctypes.data, ctypes.byref(info))
        if rc == PCDN_ETIMEOUT and info.status == _NOT_FINISHED:  # the wait timed out (not the solve)
            raise PcdnError(rc, pcdn_last_error())
        msg = pcdn_last_error() if rc < 0 else ""
        del self._nf[ticket]
        self._keep.pop(ticket, None)
        d = dict(status=info.status, t_submit=info.t_submit, t_admit=info.t_admit, t_start=info.t_start,
                 t_done=info.t_done,
                 bytes=info.bytes, stats=_stats_dict(info.stats), P_used=info.P_used, retries=info.retries,
                 message=msg)
        return rc, w, d

    def stats(self):
        a, b, c, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().pcdn_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(e)))
        return dict(submitted=a.value, finished=b.value, in_flight=c.value, bytes_in_use=e.value)

    def close(self):
        if self.handle:
            load().pcdn_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcdn_memory(h: int) -> int:
    b = ctypes.c_int64()
    _check(load().pcdn_memory(h, ctypes.byref(b)))
    return b.value


@dataclass
class Problem:
    """Owning wrapper of a problem handle (destroyed with the object)."""
    handle: int
    n_samples: int
    n_features: int

    @classmethod
    def from_csc(cls, col_ptr, row_idx, val, y, C: float, loss: str = "logistic") -> "Problem":
        return cls(pcdn_create(col_ptr, row_idx, val, y, C, loss), int(len(y)), int(len(col_ptr) - 1))

    @classmethod
    def from_device(cls, col_ptr, row_idx, val, y, C: float, loss: str = "logistic", stream=None) -> "Problem":
        return cls(pcdn_create_device(col_ptr, row_idx, val, y, C, loss, stream), int(y.shape[0]),
                   int(col_ptr.shape[0] - 1))

    def solve(self, P, eps=1e-3, seed=0, opts=None, **kw):
        return pcdn_solve(self.handle, P, eps, seed, opts, self.n_features, **kw)

    def bundle_step(self, w_in, bundle, opts=None):
        return pcdn_bundle_step(self.handle, w_in, bundle, opts)

    def set_penalty(self, l1=1.0, l2=0.0):
        pcdn_set_penalty(self.handle, l1, l2)

    def set_w(self, w):
        pcdn_set_w(self.handle, w)

    def get_w(self):
        return pcdn_get_w(self.handle, self.n_features)

    def objective(self):
        return pcdn_objective(self.handle)

    def kkt(self):
        return pcdn_kkt(self.handle)

    def permutation(self, seed, epoch):
        return pcdn_permutation(self.handle, seed, epoch, self.n_features)

    def memory(self):
        return pcdn_memory(self.handle)

    def close(self):
        if self.handle:
            pcdn_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
