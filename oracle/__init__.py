"""PCDN CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 C restatement of the paper's method (``pcdn_oracle.c``) behind a
ctypes binding.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
(``paper_1306_4080_gb300``) neither imports it nor shares code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcdn_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_libs: dict = {}

LOSSES = {"logistic": 0, "l2svm": 1}


_OMP_SRC = os.path.join(_HERE, "pcdn_omp.c")
_OMP_LIB = os.path.join(_HERE, "_liboracle_omp.so")


def compile_source(src: str, out: str, openmp: bool = False) -> str:
    """gcc, FP64, no floating-point contraction, no fast-math."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           *(["-fopenmp"] if openmp else []), "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (and its OpenMP CPU-baseline variant) next to the sources."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_OMP_SRC))
    if force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < newest:
        compile_source(_OMP_SRC, _OMP_LIB, openmp=True)
    return _LIB


_omp_lib = None


def _load_omp():
    """The OpenMP variant (the paper's shared-memory parallel scheme, all host cores): CPU baseline."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            build()
            lib = ctypes.CDLL(_OMP_LIB)
            P = ctypes.POINTER
            lib.or_solve_omp.argtypes = [P(_Problem), P(_Armijo), ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, P(_Stats)]
            lib.or_solve_omp.restype = ctypes.c_int
            lib.or_omp_threads.restype = ctypes.c_int
            _omp_lib = lib
    return _omp_lib


def omp_threads() -> int:
    return int(_load_omp().or_omp_threads())


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("c", ctypes.c_double), ("loss", ctypes.c_int),
                ("l1", ctypes.c_double), ("l2", ctypes.c_double)]


class _Armijo(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("nu", ctypes.c_double), ("q_max", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int64), ("bundles", ctypes.c_int64), ("coord_updates", ctypes.c_int64),
                ("ls_steps", ctypes.c_int64), ("ls_cap_hits", ctypes.c_int64),
                ("F_final", ctypes.c_double), ("kkt_rel", ctypes.c_double), ("kkt0", ctypes.c_double),
                ("converged", ctypes.c_int)]


def _load(path: str | None = None):
    key = path or "default"
    with _lock:
        if key not in _libs:
            lib = ctypes.CDLL(path if path else build())
            vp, i64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            P = ctypes.POINTER
            lib.or_splitmix64_output.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.or_splitmix64_output.restype = ctypes.c_uint64
            lib.or_perm_key.argtypes = [ctypes.c_uint64, i64, i64]
            lib.or_perm_key.restype = ctypes.c_uint64
            lib.or_permutation.argtypes = [ctypes.c_uint64, i64, i64, vp]
            lib.or_permutation.restype = i32
            lib.or_objective.argtypes = [P(_Problem), vp]
            lib.or_objective.restype = d
            lib.or_refresh.argtypes = [P(_Problem), vp, vp]
            lib.or_refresh.restype = i32
            lib.or_grad_hess.argtypes = [P(_Problem), vp, i64, d, P(d), P(d)]
            lib.or_grad_hess.restype = None
            lib.or_direction.argtypes = [d, d, d]
            lib.or_direction.restype = d
            lib.or_direction_l1.argtypes = [d, d, d, d]
            lib.or_direction_l1.restype = d
            lib.or_kkt_l1.argtypes = [P(_Problem), vp, vp, d]
            lib.or_kkt_l1.restype = d
            lib.or_bundle_step.argtypes = [P(_Problem), P(_Armijo), vp, vp, vp, i64, i32,
                                           vp, vp, vp, P(d), P(ctypes.c_int32), P(d), P(d)]
            lib.or_bundle_step.restype = i32
            lib.or_solve.argtypes = [P(_Problem), P(_Armijo), i64, d, ctypes.c_uint64, i64, i32, i64, vp,
                                     P(_Stats), i64, vp, vp, vp, vp, i64, vp, vp, i32, vp]
            lib.or_active_set.argtypes = [P(_Problem), vp, vp, d, vp, P(d)]
            lib.or_active_set.restype = i64
            lib.or_solve.restype = i32
            lib.or_loss_change.argtypes = [P(_Problem), d, i32, d]
            lib.or_loss_change.restype = d
            lib.or_cdn_epoch.argtypes = [P(_Problem), P(_Armijo), ctypes.c_uint64, i64, vp, vp]
            lib.or_cdn_epoch.restype = i32
            _libs[key] = lib
    return _libs[key]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Armijo:
    """Armijo parameters; defaults are the paper's (Section 5.1): sigma=0.01, gamma=0, beta=0.5;
    nu=1e-12 from Appendix A (proof of Lemma 1(b)); q_max caps the backtracking."""
    sigma: float = 0.01
    beta: float = 0.5
    gamma: float = 0.0
    nu: float = 1e-12
    q_max: int = 30

    def _c(self) -> _Armijo:
        return _Armijo(self.sigma, self.beta, self.gamma, self.nu, self.q_max)


class Oracle:
    """FP64 oracle bound to one problem (X in CSC, labels y, weight c, loss; penalty
    l1 ||w||_1 + (l2/2) ||w||^2, the paper's l1 = 1, l2 = 0 by default)."""

    def __init__(self, col_ptr, row_idx, val, y, c: float, loss: str, lib_path: str | None = None,
                 l1: float = 1.0, l2: float = 0.0):
        self.lib = _load(lib_path)
        self.col_ptr = np.ascontiguousarray(col_ptr, dtype=np.int64)
        self.row_idx = np.ascontiguousarray(row_idx, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float32)
        self.y = np.ascontiguousarray(y, dtype=np.int8)
        self.n = int(self.y.shape[0])
        self.m = int(self.col_ptr.shape[0] - 1)
        self.c = float(c)
        self.loss = loss
        self.l1, self.l2 = float(l1), float(l2)
        self._p = _Problem(self.n, self.m, _ptr(self.col_ptr), _ptr(self.row_idx), _ptr(self.val), _ptr(self.y),
                           self.c, LOSSES[loss], self.l1, self.l2)

    @classmethod
    def from_problem(cls, prob, c: float, loss: str, lib_path: str | None = None, l1: float = 1.0,
                     l2: float = 0.0) -> "Oracle":
        return cls(prob.col_ptr, prob.row_idx, prob.val, prob.y, c, loss, lib_path, l1=l1, l2=l2)

    # -- pieces -------------------------------------------------------------------------
    def objective(self, w) -> float:
        w = np.ascontiguousarray(w, dtype=np.float64)
        return float(self.lib.or_objective(ctypes.byref(self._p), _ptr(w)))

    def maintained(self, w) -> np.ndarray:
        """e^{w^T x_i} (logistic) or b_i = 1 - y_i w^T x_i (L2-SVM)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        mq = np.empty(self.n, dtype=np.float64)
        rc = self.lib.or_refresh(ctypes.byref(self._p), _ptr(w), _ptr(mq))
        if rc:
            raise RuntimeError(f"or_refresh failed: {rc}")
        return mq

    def grad_hess(self, mq, j: int, nu: float = 1e-12):
        mq = np.ascontiguousarray(mq, dtype=np.float64)
        g, h = ctypes.c_double(), ctypes.c_double()
        self.lib.or_grad_hess(ctypes.byref(self._p), _ptr(mq), int(j), float(nu), ctypes.byref(g), ctypes.byref(h))
        return g.value, h.value

    def row_loss_change(self, mq_i: float, y_i: int, u: float) -> float:
        """Loss change of one sample with maintained quantity mq_i when w^T x_i moves by u."""
        return float(self.lib.or_loss_change(ctypes.byref(self._p), float(mq_i), int(y_i), float(u)))

    def kkt_l1(self, w, mq=None, nu: float = 1e-12) -> float:
        w = np.ascontiguousarray(w, dtype=np.float64)
        if mq is None:
            mq = self.maintained(w)
        mq = np.ascontiguousarray(mq, dtype=np.float64)
        return float(self.lib.or_kkt_l1(ctypes.byref(self._p), _ptr(w), _ptr(mq), float(nu)))

    def bundle_step(self, w, mq, bundle, armijo: Armijo = Armijo(), direct: bool = False):
        """One bundle step; returns (w_new, mq_new, dict of g, h, d, Delta, q, alpha, dF, status)."""
        w = np.array(w, dtype=np.float64, copy=True)
        mq = np.array(mq, dtype=np.float64, copy=True)
        B = np.ascontiguousarray(bundle, dtype=np.int32)
        P = int(B.shape[0])
        g = np.empty(P); h = np.empty(P); d = np.empty(P)
        Delta, alpha, dF = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        q = ctypes.c_int32()
        rc = self.lib.or_bundle_step(ctypes.byref(self._p), ctypes.byref(armijo._c()), _ptr(w), _ptr(mq), _ptr(B), P,
                                     int(direct), _ptr(g), _ptr(h), _ptr(d), ctypes.byref(Delta), ctypes.byref(q),
                                     ctypes.byref(alpha), ctypes.byref(dF))
        if rc < 0:
            raise RuntimeError(f"or_bundle_step failed: {rc}")
        return w, mq, dict(g=g, h=h, d=d, Delta=Delta.value, q=q.value, alpha=alpha.value, dF=dF.value, status=rc)

    def solve(self, P: int, eps: float = 1e-3, seed: int = 0, max_epochs: int = 1000, armijo: Armijo = Armijo(),
              direct: bool = False, bundle_limit: int = -1, w0=None, trace: bool = False, shrink: bool = False):
        """Algorithm 3 to the relative KKT tolerance eps; returns (w, stats dict).  With shrink, outer
        iterations after the first visit only the active features (stats 'epoch_active': features
        visited per outer iteration)."""
        w = np.zeros(self.m) if w0 is None else np.array(w0, dtype=np.float64, copy=True)
        st = _Stats()
        cap = 0
        tq = ta = tD = tF = None
        ecap = max_epochs if (trace or shrink) else 0
        ek = eF = None
        ea = np.zeros(max(ecap, 1), dtype=np.int64)
        if trace:
            nb = (self.m + P - 1) // P
            cap = nb * max_epochs if bundle_limit < 0 else bundle_limit
            tq = np.zeros(cap, dtype=np.int32); ta = np.zeros(cap); tD = np.zeros(cap); tF = np.zeros(cap)
            ek = np.zeros(ecap); eF = np.zeros(ecap)
        nul = None
        rc = self.lib.or_solve(ctypes.byref(self._p), ctypes.byref(armijo._c()), int(P), float(eps), int(seed) & (2**64 - 1),
                               int(max_epochs), int(direct), int(bundle_limit), _ptr(w), ctypes.byref(st),
                               cap, _ptr(tq) if trace else nul, _ptr(ta) if trace else nul,
                               _ptr(tD) if trace else nul, _ptr(tF) if trace else nul,
                               ecap, _ptr(ek) if trace else nul, _ptr(eF) if trace else nul, int(bool(shrink)),
                               _ptr(ea))
        if rc < 0:
            raise RuntimeError(f"or_solve failed: {rc}")
        out = dict(epochs=st.epochs, bundles=st.bundles, coord_updates=st.coord_updates, ls_steps=st.ls_steps,
                   ls_cap_hits=st.ls_cap_hits, F_final=st.F_final, kkt_rel=st.kkt_rel, kkt0=st.kkt0,
                   converged=bool(st.converged), status=rc)
        if trace or shrink:
            out["epoch_active"] = ea[:st.epochs].copy()
        if trace:
            nbt = int(st.bundles)
            out.update(q=tq[:nbt], alpha=ta[:nbt], Delta=tD[:nbt], dF=tF[:nbt],
                       epoch_kkt=ek[:st.epochs], epoch_F=eF[:st.epochs])
        return w, out

    def solve_omp(self, P: int, eps: float = 1e-3, seed: int = 0, max_epochs: int = 1000, armijo: Armijo = Armijo(),
                  bundle_limit: int = -1, w0=None):
        """Algorithm 3 with the paper's shared-memory parallel scheme on all host cores (OpenMP);
        the CPU baseline.  Same partitions and stop rule as solve(); sums in another order."""
        lib = _load_omp()
        w = np.zeros(self.m) if w0 is None else np.array(w0, dtype=np.float64, copy=True)
        st = _Stats()
        rc = lib.or_solve_omp(ctypes.byref(self._p), ctypes.byref(armijo._c()), int(P), float(eps),
                              int(seed) & (2**64 - 1), int(max_epochs), int(bundle_limit), _ptr(w), ctypes.byref(st))
        if rc < 0:
            raise RuntimeError(f"or_solve_omp failed: {rc}")
        return w, dict(epochs=st.epochs, bundles=st.bundles, coord_updates=st.coord_updates, ls_steps=st.ls_steps,
                       ls_cap_hits=st.ls_cap_hits, F_final=st.F_final, kkt_rel=st.kkt_rel, kkt0=st.kkt0,
                       converged=bool(st.converged), status=rc)

    def active_set(self, w, nu: float = 1e-12):
        """Shrinking's active set at w (maintained quantities recomputed from w): (mask, M)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        mq = self.maintained(w)
        act = np.zeros(self.m, dtype=np.uint8)
        M = ctypes.c_double()
        cnt = self.lib.or_active_set(ctypes.byref(self._p), _ptr(w), _ptr(mq), float(nu), _ptr(act), ctypes.byref(M))
        if cnt < 0:
            raise RuntimeError("or_active_set failed")
        return act.astype(bool), M.value

    def cdn_epoch(self, w, mq, seed: int, epoch: int, armijo: Armijo = Armijo()):
        w = np.array(w, dtype=np.float64, copy=True)
        mq = np.array(mq, dtype=np.float64, copy=True)
        rc = self.lib.or_cdn_epoch(ctypes.byref(self._p), ctypes.byref(armijo._c()), int(seed) & (2**64 - 1),
                                   int(epoch), _ptr(w), _ptr(mq))
        if rc:
            raise RuntimeError(f"or_cdn_epoch failed: {rc}")
        return w, mq


def permutation(seed: int, epoch: int, m: int, lib_path: str | None = None) -> np.ndarray:
    lib = _load(lib_path)
    perm = np.empty(m, dtype=np.int32)
    rc = lib.or_permutation(int(seed) & (2**64 - 1), int(epoch), int(m), _ptr(perm))
    if rc:
        raise RuntimeError(f"or_permutation failed: {rc}")
    return perm


def perm_key(seed: int, epoch: int, j: int) -> int:
    return int(_load().or_perm_key(int(seed) & (2**64 - 1), int(epoch), int(j)))


def splitmix64_output(s0: int, k: int) -> int:
    return int(_load().or_splitmix64_output(int(s0) & (2**64 - 1), int(k)))


def direction(g: float, h: float, w: float, lib_path: str | None = None, l1: float | None = None) -> float:
    """argmin_d g d + h d^2/2 + l1 |w + d| (Eq. 5; l1 = 1 unless given)."""
    if l1 is None:
        return float(_load(lib_path).or_direction(float(g), float(h), float(w)))
    return float(_load(lib_path).or_direction_l1(float(g), float(h), float(w), float(l1)))
