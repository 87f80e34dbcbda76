"""Margins beyond FP64's e^{w^T x} range (logistic loss).

Algorithm 4 maintains E_i = e^{w^T x_i}; in FP64 that holds |w^T x_i| up to about 709, and the
library stops with PCDN_ENUMERIC a little before (about 699).  Mixed precision keeps the margin
w^T x_i itself (a double-float pair) and forms every coefficient with e^{-|z|}, so it has no such
limit.  The problem below drives one sample's margin to several thousand at the optimum: the
mixed solve must converge there, to a w whose objective (the oracle's, evaluated from z = Xw
without overflow) matches the reported one and whose L1 KKT measure, recomputed here with a
stable logistic function, meets the tolerance; the FP64 solve must stop with the documented
status and message.
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


def big_margin_problem(seed=11):
    """n = 2000 samples, m = 200 features: 199 sparse N(0, 1) features (density 5%) under random
    labels, and feature 0, set to 1 on 300 samples labelled +1 and to 1000 on one more sample
    labelled +1 that has no other entry.  The 300 samples push w_0 to about log(300 C), so that
    last sample's margin 1000 w_0 ends in the thousands."""
    rng = np.random.default_rng(seed)
    n, m = 2000, 200
    y = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    big = n - 1
    pos = np.flatnonzero(y[:big] > 0)
    f0 = np.sort(rng.choice(pos, size=300, replace=False))
    y[big] = 1
    cols_r, cols_v = [np.append(f0, big).astype(np.int32)], [np.append(np.ones(300), 1000.0).astype(np.float32)]
    for j in range(1, m):
        rows = np.flatnonzero(rng.random(big) < 0.05).astype(np.int32)  # the big sample stays out
        cols_r.append(rows)
        cols_v.append(rng.normal(0.0, 1.0, rows.size).astype(np.float32))
    col_ptr = np.zeros(m + 1, np.int64)
    col_ptr[1:] = np.cumsum([c.size for c in cols_r])
    return col_ptr, np.concatenate(cols_r), np.concatenate(cols_v), y


def l1_kkt(col_ptr, row_idx, val, y, C, w):
    """Sum over features of |minimum-norm subgradient| of F at w (the solver's stopping measure),
    with the logistic derivative 1 - sigma(y z) = 1 / (1 + e^{y z}) formed without overflow."""
    n = y.shape[0]
    z = np.zeros(n)
    for j in range(w.shape[0]):
        a, b = col_ptr[j], col_ptr[j + 1]
        z[row_idx[a:b]] += val[a:b].astype(np.float64) * w[j]
    yz = y.astype(np.float64) * z
    t = np.where(yz > 0, np.exp(-np.abs(yz)) / (1.0 + np.exp(-np.abs(yz))), 1.0 / (1.0 + np.exp(-np.abs(yz))))
    coef = -y.astype(np.float64) * t  # d loss_i / d z_i
    s = 0.0
    for j in range(w.shape[0]):
        a, b = col_ptr[j], col_ptr[j + 1]
        g = C * float(np.dot(val[a:b].astype(np.float64), coef[row_idx[a:b]]))
        if w[j] > 0:
            v = g + 1.0
        elif w[j] < 0:
            v = g - 1.0
        else:
            v = max(abs(g) - 1.0, 0.0)
        s += abs(v)
    return s, z


def test_mixed_solve_past_the_fp64_margin_range(pk):
    col_ptr, row_idx, val, y = big_margin_problem()
    C, eps = 1.0, 1e-4
    orc = oracle.Oracle(col_ptr, row_idx, val, y, C, "logistic")
    P = pk.Problem.from_csc(col_ptr, row_idx, val, y, C, "logistic")
    try:
        rc, w, st, _ = P.solve(16, eps, 0, pk.pcdn_default_opts(prec="mixed", max_epochs=2000))
        assert rc == pk.PCDN_OK and st["converged"]
        kkt, z = l1_kkt(col_ptr, row_idx, val, y, C, w)
        kkt0, _ = l1_kkt(col_ptr, row_idx, val, y, C, np.zeros_like(w))
        assert np.max(np.abs(z)) > 2000.0, np.max(np.abs(z))  # far past e^z's FP64 range
        assert kkt / kkt0 <= eps * 1.05, (kkt / kkt0, st["kkt_rel"])
        F = orc.objective(w)
        assert np.isfinite(F) and st["F_final"] == pytest.approx(F, rel=1e-9)
        # the same problem in FP64 stops with the documented status once a margin passes e^z's range
        with pytest.raises(pk.PcdnError) as ei:
            P.solve(16, eps, 0, pk.pcdn_default_opts(prec="fp64", max_epochs=2000))
        assert ei.value.code == pk.PCDN_ENUMERIC
        assert "699" in pk.pcdn_last_error()
    finally:
        P.close()
