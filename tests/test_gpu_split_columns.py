"""Columns longer than one chunk (512 nonzeros): the GPU path cuts them into chunks whose sums
are combined across thread blocks.  Checked against the FP64 oracle through the C ABI on a matrix
built for the purpose (seeded): one column of 300,000 nonzeros (586 chunks, combined by a whole
block), many columns of 1,025 to 6,000 nonzeros (3 to 12 chunks, several per block), and short
columns of 1 to 900 nonzeros (one or two chunks); with one block (more split chunks than a block
lists: the one-at-a-time path) and with every block of the GPU (listed chunks, one warp per column).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4080_gb300 import build
    build.build()
    import paper_1306_4080_gb300 as m
    m.load()
    return m


def split_matrix(seed=5):
    """CSC (n = 300,000 samples, m = 160 features): column 0 dense, columns 1..99 of 1,025..6,000
    nonzeros, columns 100..159 of 1..900 nonzeros; values |N(0, 1)| / 4, labels +-1."""
    rng = np.random.default_rng(seed)
    n = 300_000
    lens = [n] + list(rng.integers(1025, 6001, 99)) + list(rng.integers(1, 901, 60))
    rows = [np.arange(n, dtype=np.int32)] + [np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
                                             for k in lens[1:]]
    col_ptr = np.zeros(len(lens) + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum([len(r) for r in rows])
    row_idx = np.concatenate(rows)
    val = (np.abs(rng.standard_normal(len(row_idx))) / 4).astype(np.float32)
    y = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    return col_ptr, row_idx, val, y


@pytest.mark.parametrize("loss,C", [("logistic", 1.0), ("l2svm", 0.5)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", [1, 100000])
def test_split_column_paths(pk, loss, C, prec, grid):
    col_ptr, row_idx, val, y = split_matrix()
    m = len(col_ptr) - 1
    orc = oracle.Oracle(col_ptr, row_idx, val, y, C, loss)
    P = pk.Problem.from_csc(col_ptr, row_idx, val, y, C, loss)
    opts = pk.pcdn_default_opts(prec=prec, grid_ctas=grid)
    tol = 1e-9 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(3)
    try:
        w1 = np.where(rng.random(m) < 0.3, rng.normal(0, 0.05, m), 0.0)
        for w in (np.zeros(m), w1):
            mq = orc.maintained(w)
            for B in (rng.permutation(m).astype(np.int32), np.arange(m, dtype=np.int32)[::-1].copy()):
                r = P.bundle_step(w, B, opts)
                _, _, ro = orc.bundle_step(w, mq, B)
                gs = np.abs(ro["g"]).max()
                assert np.abs(r["g"] - ro["g"]).max() <= tol * gs
                assert np.abs(r["h"] - ro["h"]).max() <= tol * np.abs(ro["h"]).max()
                dscale = np.abs(ro["g"]) / ro["h"] + np.abs(ro["d"])
                assert np.all(np.abs(r["d"] - ro["d"]) <= tol * dscale + 1e-300)
                assert abs(r["Delta"] - ro["Delta"]) <= tol * abs(ro["Delta"])
                assert r["q"] == ro["q"] and r["alpha"] == ro["alpha"]
                assert abs(r["dF"] - ro["dF"]) <= (1e-7 if prec == "fp64" else 1e-4) * abs(ro["dF"]) + 1e-12 * abs(ro["Delta"])
    finally:
        P.close()
