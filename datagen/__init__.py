"""Seeded synthetic inputs for the PCDN solver (inputs only, no solver arithmetic).

The generator itself is C (``gen.c``, compiled on first use with gcc); this
module marshals its output into numpy arrays.  Both the CPU oracle tests and the
CUDA path take their inputs from here, and from nowhere else.

Workload presets follow the sparse text-classification shapes of the paper's
experiments (Section 5, Table 2): uniform-density |N(0,1)| rows and Zipf-column
tf-idf rows, all rows L2-normalised, labels from a sparse planted w* with a
fixed fraction of flips.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_libgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into ``_libgen.so`` (gcc, OpenMP, no fp contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Spec(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("kind", ctypes.c_int),
                ("density", ctypes.c_double), ("row_mean", ctypes.c_double), ("zipf_s", ctypes.c_double),
                ("value_kind", ctypes.c_int), ("wstar_nnz", ctypes.c_int64), ("flip_frac", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class _Out(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int64)), ("col_idx", ctypes.POINTER(ctypes.c_int32)),
                ("rval", ctypes.POINTER(ctypes.c_float)),
                ("col_ptr", ctypes.POINTER(ctypes.c_int64)), ("row_idx", ctypes.POINTER(ctypes.c_int32)),
                ("cval", ctypes.POINTER(ctypes.c_float)),
                ("y", ctypes.POINTER(ctypes.c_int8)),
                ("wstar_idx", ctypes.POINTER(ctypes.c_int32)), ("wstar_val", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.gen_generate.argtypes = [ctypes.POINTER(_Spec), ctypes.POINTER(_Out)]
            lib.gen_generate.restype = ctypes.c_int
            lib.gen_free.argtypes = [ctypes.POINTER(_Out)]
            lib.gen_free.restype = ctypes.c_int
            lib.gen_nthreads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Spec:
    """Shape and distribution of one synthetic problem.

    kind "uniform": every entry present with probability ``density``; values |N(0,1)|.
    kind "zipf": row length max(1, Poisson(row_mean)); column of each entry drawn
    without replacement with probability proportional to rank**-zipf_s over a
    random ranking of the columns; values log(1+c), c ~ Poisson(2) given c >= 1,
    times idf_j = log(1 + n/df_j).  Rows are L2-normalised in both kinds.
    """
    n_samples: int
    n_features: int
    kind: str = "uniform"
    density: float = 0.005
    row_mean: float = 100.0
    zipf_s: float = 1.1
    values: str = "halfnormal"
    wstar_nnz: int = 50
    flip_frac: float = 0.05
    seed: int = 0


@dataclass
class Problem:
    """One generated problem: CSC (solver layout), CSR mirror, labels, planted w*."""
    spec: Spec
    col_ptr: np.ndarray   # int64 [m+1]
    row_idx: np.ndarray   # int32 [nnz]
    val: np.ndarray       # float32 [nnz]
    y: np.ndarray         # int8 [n], entries in {-1, +1}
    row_ptr: np.ndarray | None = None   # int64 [n+1]
    col_idx: np.ndarray | None = None   # int32 [nnz]
    rval: np.ndarray | None = None      # float32 [nnz]
    wstar_idx: np.ndarray | None = None
    wstar_val: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_samples(self) -> int:
        return int(self.spec.n_samples)

    @property
    def n_features(self) -> int:
        return int(self.spec.n_features)

    @property
    def nnz(self) -> int:
        return int(self.col_ptr[-1])

    def dense(self) -> np.ndarray:
        """Dense float64 copy of X (small problems only)."""
        X = np.zeros((self.n_samples, self.n_features), dtype=np.float64)
        for j in range(self.n_features):
            a, b = self.col_ptr[j], self.col_ptr[j + 1]
            X[self.row_idx[a:b], j] = self.val[a:b]
        return X


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def generate(spec: Spec, with_csr: bool = True) -> Problem:
    """Generate one problem; deterministic in ``spec`` (thread count does not matter)."""
    lib = _load()
    kinds = {"uniform": 0, "zipf": 1}
    vals = {"halfnormal": 0, "tfidf": 1}
    cs = _Spec(n=spec.n_samples, m=spec.n_features, kind=kinds[spec.kind], density=spec.density,
               row_mean=spec.row_mean, zipf_s=spec.zipf_s, value_kind=vals[spec.values],
               wstar_nnz=spec.wstar_nnz, flip_frac=spec.flip_frac, seed=spec.seed)
    out = _Out()
    rc = lib.gen_generate(ctypes.byref(cs), ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"datagen: generation failed (code {rc}) for {spec}")
    try:
        n, m, nnz = spec.n_samples, spec.n_features, int(out.nnz)
        p = Problem(spec=spec,
                    col_ptr=_arr(out.col_ptr, m + 1, np.int64),
                    row_idx=_arr(out.row_idx, nnz, np.int32),
                    val=_arr(out.cval, nnz, np.float32),
                    y=_arr(out.y, n, np.int8),
                    wstar_idx=_arr(out.wstar_idx, spec.wstar_nnz, np.int32),
                    wstar_val=_arr(out.wstar_val, spec.wstar_nnz, np.float64))
        if with_csr:
            p.row_ptr = _arr(out.row_ptr, n + 1, np.int64)
            p.col_idx = _arr(out.col_idx, nnz, np.int32)
            p.rval = _arr(out.rval, nnz, np.float32)
    finally:
        lib.gen_free(ctypes.byref(out))
    p.meta = {"generator_threads": int(lib.gen_nthreads())}
    return p


# ---- workload presets (the solver settings travel with them) -------------------------------

@dataclass
class Workload:
    name: str
    spec: Spec
    loss: str          # "logistic" or "l2svm"
    C: float
    P: int
    eps: float = 1e-3
    solver_seed: int = 0

    def describe(self) -> dict:
        d = asdict(self)
        d["spec"] = asdict(self.spec)
        return d


WORKLOADS = {
    # 2,000 x 10,000, density 0.5 %, |N(0,1)| values, 50-sparse w*, 5 % flips, logistic, C=1, P=64
    "lr_2k_10k": Workload("lr_2k_10k", Spec(2000, 10000, "uniform", density=0.005, values="halfnormal",
                                           wstar_nnz=50, flip_frac=0.05, seed=0), "logistic", 1.0, 64),
    # 20,000 x 100,000, ~100 nnz/row, Zipf 1.1 columns, tf-idf values, 200-sparse w*, 3 % flips, L2-SVM, C=0.5
    "svm_20k_100k": Workload("svm_20k_100k", Spec(20000, 100000, "zipf", row_mean=100.0, zipf_s=1.1,
                                                 values="tfidf", wstar_nnz=200, flip_frac=0.03, seed=0),
                             "l2svm", 0.5, 256),
    # 2,000,000 x 3,000,000, ~150 nnz/row (~300M nnz), Zipf 1.05, tf-idf, 5000-sparse w*, 5 % flips,
    # logistic, C=1, P=4096
    "lr_2m_3m": Workload("lr_2m_3m", Spec(2000000, 3000000, "zipf", row_mean=150.0, zipf_s=1.05,
                                         values="tfidf", wstar_nnz=5000, flip_frac=0.05, seed=0),
                         "logistic", 1.0, 4096),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def scaled(name: str, factor: float, seed: int | None = None) -> Workload:
    """The same recipe with n, m (and so nnz) scaled by ``factor``; P scaled alike (>= 1)."""
    w = WORKLOADS[name]
    s = Spec(**asdict(w.spec))
    s.n_samples = max(8, int(round(s.n_samples * factor)))
    s.n_features = max(8, int(round(s.n_features * factor)))
    if s.kind == "zipf":
        s.row_mean = min(s.row_mean, 0.25 * s.n_features)
    s.wstar_nnz = max(1, min(s.n_features, int(round(s.wstar_nnz * factor))))
    if seed is not None:
        s.seed = seed
    return Workload(f"{name}@{factor:g}", s, w.loss, w.C, max(1, int(round(w.P * factor))), w.eps, w.solver_seed)


# ---- batched workload: many independent problems, each along a regularisation path ---------------

@dataclass
class PathJob:
    """One problem of the batched workload and the C values it is solved at (in order, each
    warm-started from the previous solution)."""
    name: str
    spec: Spec
    loss: str
    C_path: list
    eps: float = 1e-3
    solver_seed: int = 0


def batch_jobs(count: int = 64, seed: int = 0, scale: float = 1.0, n_C: int = 16,
               C_range: tuple = (1e-2, 1e1)) -> list:
    """``count`` problems of uneven sizes in the shape of the paper's sparse text workloads:
    n_samples log-uniform in [1k, 50k], n_features log-uniform in [5k, 200k] (both times ``scale``),
    density uniform in [0.1 %, 1 %] (row length = density * n_features), Zipf 1.1 columns, tf-idf
    values, rows L2-normalised, planted w* with max(10, n_features/500) nonzeros; losses alternate
    logistic (5 % label flips) / L2-SVM (3 %); each solved along ``n_C`` values of C log-spaced over
    ``C_range``.  Problem k's generator seed is k + 1000 * seed."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5CD, int(seed)]))
    out = []
    C_path = list(np.logspace(np.log10(C_range[0]), np.log10(C_range[1]), n_C))
    for k in range(count):
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(5e4))) * scale))
        m = int(round(np.exp(rng.uniform(np.log(5e3), np.log(2e5))) * scale))
        dens = float(rng.uniform(1e-3, 1e-2))
        n, m = max(16, n), max(32, m)
        row_mean = max(2.0, dens * m)
        loss = "logistic" if k % 2 == 0 else "l2svm"
        spec = Spec(n, m, "zipf", row_mean=row_mean, zipf_s=1.1, values="tfidf",
                    wstar_nnz=max(10, min(m, m // 500)), flip_frac=0.05 if loss == "logistic" else 0.03,
                    seed=k + 1000 * int(seed))
        out.append(PathJob(f"batch{k}", spec, loss, C_path))
    return out
