"""GPU path vs the FP64 oracle, through the C ABI, on identical seeded inputs and partitions.

Tolerances (the bar: per-bundle d and step size within 1e-5 relative, final objective
within 1e-6 relative):
  FP64 mode   g, h, d, Delta within 1e-9 of the bundle's largest magnitude; q and alpha equal;
              dF within 1e-7 relative (different reduction order over up to 10^5 rows).
  mixed mode  g, h within 1e-5 of the bundle's largest magnitude; d within 1e-5 on the scale of
              the Newton step, |d_j - d*_j| <= 1e-5 (|g_j| / h_j + |d*_j|) (how FP32 errors in g and h
              reach d = -(g +/- 1)/h); q and alpha equal unless the oracle's Armijo margin is within
              1e-5 of the compared quantities.
"""
import numpy as np
import pytest

import datagen
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


_CACHE = {}


def problem(name):
    if name in _CACHE:
        return _CACHE[name]
    if name == "ragged_lr":
        wl = datagen.Workload("ragged_lr", datagen.Spec(333, 1001, "uniform", density=0.02, values="halfnormal",
                                                        wstar_nnz=20, flip_frac=0.05, seed=7), "logistic", 2.0, 100)
    elif name == "ragged_svm":
        wl = datagen.Workload("ragged_svm", datagen.Spec(4000, 3001, "zipf", row_mean=30.0, zipf_s=1.1,
                                                         values="tfidf", wstar_nnz=40, flip_frac=0.05, seed=8),
                              "l2svm", 1.0, 97)
    else:
        wl = datagen.workload(name)
    p = datagen.generate(wl.spec)
    _CACHE[name] = (wl, p)
    return wl, p


def rel_err(a, b):
    scale = max(float(np.max(np.abs(b))) if np.size(b) else 0.0, 1e-300)
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / scale if np.size(b) else 0.0


def armijo_margin(orc, p, w, mq, B, d, Delta, q_lo, q_hi, armijo):
    """The smallest relative Armijo margin |dF(a) - sigma a Delta| / scale over q in [q_lo, q_hi],
    dF(a) in the oracle's maintained form (Eq. 10 per sample plus the penalty change), scale =
    c sum_i |change_i| + sum_j |penalty change_j| + |sigma a Delta|: the size of the rounding that
    any order of summation leaves."""
    dx = np.zeros(p.n_samples)
    for k, j in enumerate(B):
        a, b = p.col_ptr[j], p.col_ptr[j + 1]
        dx[p.row_idx[a:b]] += p.val[a:b].astype(np.float64) * d[k]
    rows = np.flatnonzero(dx)
    best = np.inf
    for q in range(q_lo, q_hi + 1):
        a = armijo.beta ** q
        ch = np.array([orc.row_loss_change(mq[i], int(p.y[i]), a * dx[i]) for i in rows])
        pen = np.abs(w[B] + a * d) - np.abs(w[B])
        dF = orc.c * ch.sum() + pen.sum()
        thr = armijo.sigma * a * Delta
        best = min(best, abs(dF - thr) / (orc.c * np.abs(ch).sum() + np.abs(pen).sum() + abs(thr)))
    return best


def oracle_state_at(orc, m, Pb, seed, t):
    """The oracle's w after t bundles of its solve (Algorithm 3 from w = 0, no shrinking) and the
    bundle it takes next."""
    nb = (m + Pb - 1) // Pb
    w, _ = orc.solve(Pb, eps=1e-300, seed=seed, max_epochs=t // nb + 1, bundle_limit=t)
    k, i = divmod(t, nb)
    perm = oracle.permutation(seed, k, m)
    return w, perm[i * Pb:(i + 1) * Pb].astype(np.int32)


def margin_small(orc, w, ro, bundle, q_gpu, q_or, armijo, tol):
    """True when, at every step size between the two accepted ones, the oracle's objective change
    F(w + a d) - F(w) is within tol of the Armijo threshold sigma a Delta (Eq. 6)."""
    F0 = orc.objective(w)
    for q in range(min(q_gpu, q_or), max(q_gpu, q_or) + 1):
        a = armijo.beta ** q
        wt = w.copy()
        wt[bundle] += a * ro["d"]
        dF = orc.objective(wt) - F0
        thr = armijo.sigma * a * ro["Delta"]
        if abs(dF - thr) <= tol * (abs(dF) + abs(thr)):
            return True
    return False


@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k", "ragged_lr", "ragged_svm"])
def test_permutation_bitwise(pk, name):
    wl, p = problem(name)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        for seed, epoch in [(0, 0), (0, 1), (wl.solver_seed + 99, 5), (2**64 - 1, 2)]:
            np.testing.assert_array_equal(P.permutation(seed, epoch), oracle.permutation(seed, epoch, p.n_features))
    finally:
        P.close()


CASES = [("lr_2k_10k", 64), ("svm_20k_100k", 1024), ("svm_20k_100k", 8), ("ragged_lr", 100), ("ragged_svm", 97)]


@pytest.mark.parametrize("layout", ["scatter", "rows"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", [1, 0])
@pytest.mark.parametrize("name,Pb", CASES)
def test_bundle_step_parity(pk, name, Pb, grid, prec, layout):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    opts = pk.pcdn_default_opts(prec=prec, grid_ctas=(grid if grid else 100000), layout=layout)
    armijo = oracle.Armijo()
    tol = 1e-9 if prec == "fp64" else 1e-5
    try:
        # states: w = 0, and w after part of an outer iteration of the oracle
        w1, _ = orc.solve(Pb, eps=1e-12, seed=3, max_epochs=2, bundle_limit=max(1, (p.n_features // Pb) // 2))
        rng = np.random.default_rng(11)
        for w in (np.zeros(p.n_features), w1):
            mq = orc.maintained(w)
            for trial in range(3):
                B = rng.choice(p.n_features, size=Pb, replace=False).astype(np.int32)
                r = P.bundle_step(w, B, opts)
                _, _, ro = orc.bundle_step(w, mq, B, armijo=armijo)
                assert rel_err(r["g"], ro["g"]) <= tol, ("g", rel_err(r["g"], ro["g"]))
                assert rel_err(r["h"], ro["h"]) <= tol, ("h", rel_err(r["h"], ro["h"]))
                if prec == "fp64":
                    assert rel_err(r["d"], ro["d"]) <= tol, ("d", rel_err(r["d"], ro["d"]))
                dscale = np.abs(ro["g"]) / ro["h"] + np.abs(ro["d"])
                assert np.all(np.abs(r["d"] - ro["d"]) <= tol * dscale + 1e-300), ("d (Newton scale)",)
                assert abs(r["Delta"] - ro["Delta"]) <= tol * max(abs(ro["Delta"]), 1e-300) + 1e-300
                if r["q"] != ro["q"]:
                    assert prec == "mixed" and margin_small(orc, w, ro, B, r["q"], ro["q"], armijo, 1e-5), \
                        (r["q"], ro["q"], r["dF"], ro["dF"])
                    continue
                assert r["alpha"] == ro["alpha"]
                if ro["dF"] != 0.0:
                    dtol = 1e-7 if prec == "fp64" else 1e-4
                    assert abs(r["dF"] - ro["dF"]) <= dtol * abs(ro["dF"]) + 1e-12 * abs(ro["Delta"]), (r["dF"], ro["dF"])
                else:
                    assert r["dF"] == 0.0
    finally:
        P.close()


@pytest.mark.parametrize("layout", ["scatter", "rows"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,Pb,grid", [("lr_2k_10k", 64, 0), ("lr_2k_10k", 64, 100000), ("svm_20k_100k", 256, 0),
                                          ("svm_20k_100k", 1024, 0), ("ragged_svm", 97, 100000)])
def test_solve_parity(pk, name, Pb, grid, prec, layout):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    wo, so = orc.solve(Pb, eps=wl.eps, seed=wl.solver_seed, trace=True, max_epochs=200)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        opts = pk.pcdn_default_opts(prec=prec, grid_ctas=grid, max_epochs=200, layout=layout)
        nb = so["bundles"] + 8
        rc, w, st, tr = P.solve(Pb, wl.eps, wl.solver_seed, opts, trace_bundles=int(nb), trace_epochs=200)
        assert st["converged"] and so["converged"]
        assert abs(st["F_final"] - so["F_final"]) <= 1e-6 * abs(so["F_final"]), (st["F_final"], so["F_final"])
        if prec == "fp64":
            # same trajectory: same epochs, same accepted steps, same relative KKT per epoch
            assert st["epochs"] == so["epochs"]
            n = min(len(tr["q"]), len(so["q"]))
            assert n == so["bundles"]
            # a differing accepted step is a near-tie: at the oracle's state there, the Armijo test
            # (Eq. 6) is within 1e-10 of equality at some step size between the two choices
            mism = np.flatnonzero(tr["q"][:n] != so["q"][:n])
            assert mism.size <= max(2, n // 500), (mism.size, n)
            armijo = oracle.Armijo()
            for t in mism:
                wt, B = oracle_state_at(orc, p.n_features, Pb, wl.solver_seed, int(t))
                mq = orc.maintained(wt)
                _, _, ro = orc.bundle_step(wt, mq, B, armijo=armijo)
                mg = armijo_margin(orc, p, wt, mq, B, ro["d"], ro["Delta"], int(min(tr["q"][t], ro["q"])),
                                   int(max(tr["q"][t], ro["q"])), armijo)
                assert mg <= 1e-10, (int(t), int(tr["q"][t]), int(so["q"][t]), mg)
            np.testing.assert_allclose(tr["epoch_kkt"], so["epoch_kkt"], rtol=1e-6)
            np.testing.assert_allclose(w, wo, rtol=0, atol=1e-7 * max(1.0, np.abs(wo).max()))
        else:
            # mixed precision stops at the oracle's outer iteration: its stopping test is FP64-grade
            assert st["epochs"] == so["epochs"], (st["epochs"], so["epochs"], st["kkt_rel"], so["kkt_rel"])
        assert st["bundles"] == so["bundles"]
        # F is non-increasing bundle by bundle (Lemma 1(c)) on the GPU as well
        assert np.all(tr["dF"] <= 1e-9 * abs(so["F_final"]))
        assert st["kernel_launches"] > 0
    finally:
        P.close()


@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k"])
def test_objective_and_kkt(pk, name):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        rng = np.random.default_rng(2)
        for _ in range(3):
            w = rng.normal(0, 0.5, p.n_features) * (rng.random(p.n_features) < 0.05)
            P.set_w(w)
            np.testing.assert_array_equal(P.get_w(), w)
            assert P.objective() == pytest.approx(orc.objective(w), rel=1e-12)
            assert P.kkt() == pytest.approx(orc.kkt_l1(w), rel=1e-10)
    finally:
        P.close()


@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k", "ragged_svm"])
def test_mixed_mode_refresh(pk, name):
    """After a mixed-precision solve the problem refreshes z = Xw in double-float arithmetic on the
    FP32 pipe: the objective from it stays within 1e-12 of the oracle's FP64 one, also at large
    margins; the KKT norm (per-sample FP64 coefficients split into FP32 pairs, double-float column
    sums) within 1e-9."""
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        P.solve(min(wl.P, p.n_features), 1e-1, 0, pk.pcdn_default_opts(prec="mixed", max_epochs=1), want_w=False)
        rng = np.random.default_rng(5)
        for scale in (0.5, 20.0):
            w = rng.normal(0, scale, p.n_features) * (rng.random(p.n_features) < 0.05)
            P.set_w(w)
            assert P.objective() == pytest.approx(orc.objective(w), rel=1e-12)
            assert P.kkt() == pytest.approx(orc.kkt_l1(w), rel=1e-9)
    finally:
        P.close()


@pytest.mark.parametrize("name,Pb", [("svm_20k_100k", 1024), ("lr_2k_10k", 64), ("ragged_svm", 97)])
def test_fp64_rows_layout_repeats_bit_for_bit(pk, name, Pb):
    """FP64 with the row-sorted layout on the largest walker grid: every sum of the path is formed in
    a fixed order or exactly (integer limbs), so two solves give the same w, bit for bit, and the
    same trajectory."""
    wl, p = problem(name)
    runs = []
    for _ in range(2):
        P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
        try:
            opts = pk.pcdn_default_opts(prec="fp64", grid_ctas=100000, layout="rows", max_epochs=200)
            rc, w, st, tr = P.solve(Pb, wl.eps, wl.solver_seed, opts, trace_bundles=100000, trace_epochs=200)
            assert st["walk_grid"] > 1
            runs.append((w, st, tr))
        finally:
            P.close()
    (w1, s1, t1), (w2, s2, t2) = runs
    assert np.array_equal(w1.view(np.uint64), w2.view(np.uint64))
    assert s1["epochs"] == s2["epochs"] and s1["bundles"] == s2["bundles"] and s1["F_final"] == s2["F_final"]
    for k in ("q", "alpha", "Delta", "dF"):
        assert np.array_equal(t1[k], t2[k]), k


@pytest.mark.parametrize("long_row", [False, True])
def test_row_mirror_paths(pk, long_row):
    """z = Xw runs on a row-major copy of X built at creation: by a scatter into rows and a sort of
    each row when every row has at most 1024 entries, else by a stable sort of all entries by row.
    Both give each row's entries in column order, the oracle's summation order: the FP64 objective
    (refresh) matches the oracle to 1e-13 and an FP64 solve follows the oracle's trajectory."""
    rng = np.random.default_rng(9)
    n, m = 3000, 4000
    cols = [np.sort(rng.choice(n, size=int(k), replace=False)) for k in rng.integers(1, 12, m)]
    if long_row:  # row 7 present in 1,500 columns
        for j in rng.choice(m, size=1500, replace=False):
            cols[j] = np.unique(np.append(cols[j], 7))
    col_ptr = np.zeros(m + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum([len(c) for c in cols])
    row_idx = np.concatenate(cols).astype(np.int32)
    val = (np.abs(rng.standard_normal(len(row_idx))) / 3).astype(np.float32)
    y = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    assert (np.bincount(row_idx, minlength=n).max() > 1024) == long_row
    orc = oracle.Oracle(col_ptr, row_idx, val, y, 1.0, "logistic")
    P = pk.Problem.from_csc(col_ptr, row_idx, val, y, 1.0, "logistic")
    try:
        for _ in range(3):
            w = rng.normal(0, 1.0, m) * (rng.random(m) < 0.2)
            P.set_w(w)
            assert P.objective() == pytest.approx(orc.objective(w), rel=1e-13)
        _, w1, st, _ = P.solve(64, 1e-3, 0, pk.pcdn_default_opts(max_epochs=300))
        _, so = orc.solve(64, eps=1e-3, seed=0, max_epochs=300)
        assert st["epochs"] == so["epochs"]
        assert st["F_final"] == pytest.approx(so["F_final"], rel=1e-9)
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_and_resume(pk, prec):
    """A solve stopped after k outer iterations (its checkpoint: w and k) and resumed on a fresh
    problem with warm_start = 1, epoch0 = k and kkt_ref = the first part's start-point KKT draws the
    same partitions (Eq. 8) and stops at the same outer iteration as the uninterrupted solve."""
    wl, p = problem("lr_2k_10k")
    Pb, eps = 64, 1e-4
    A = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    B = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        opts = pk.pcdn_default_opts(prec=prec, max_epochs=500)
        _, w_full, st_full, _ = A.solve(Pb, eps, 3, opts)
        assert st_full["converged"] and st_full["epochs"] >= 4
        k = st_full["epochs"] // 2
        _, w_k, st1, _ = A.solve(Pb, eps, 3, pk.pcdn_default_opts(prec=prec, max_epochs=k))
        assert st1["epochs"] == k and not st1["converged"]
        B.set_w(w_k)
        _, w_end, st2, _ = B.solve(Pb, eps, 3, pk.pcdn_default_opts(prec=prec, max_epochs=500, warm_start=1, epoch0=k,
                                                                   kkt_ref=st1["kkt0"]))
        assert st2["converged"]
        if prec == "fp64":  # the same trajectory (up to the order of the atomic adds of d^T x_i)
            assert st1["epochs"] + st2["epochs"] == st_full["epochs"]
            assert st2["kkt_rel"] == pytest.approx(st_full["kkt_rel"], rel=1e-6)
            assert st2["F_final"] == pytest.approx(st_full["F_final"], rel=1e-12)
            np.testing.assert_allclose(w_end, w_full, rtol=0, atol=1e-8 * max(1.0, np.abs(w_full).max()))
        else:  # FP32 atomic sums: trajectories equal to rounding
            assert abs(st1["epochs"] + st2["epochs"] - st_full["epochs"]) <= 1
            assert st2["F_final"] == pytest.approx(st_full["F_final"], rel=1e-6)
        # a resumed solve that is already converged ends at once
        _, _, st3, _ = B.solve(Pb, eps, 3, pk.pcdn_default_opts(prec=prec, warm_start=1, epoch0=st_full["epochs"],
                                                                kkt_ref=st1["kkt0"]))
        assert st3["converged"] and st3["epochs"] == 0
        with pytest.raises(pk.PcdnError) as ei:
            B.solve(Pb, eps, 3, pk.pcdn_default_opts(epoch0=-1))
        assert ei.value.code == pk.PCDN_EINVAL
    finally:
        A.close()
        B.close()


def test_device_pointer_create_matches_host_create(pk):
    import torch
    wl, p = problem("svm_20k_100k")
    dev = torch.device("cuda:0")
    t = [torch.from_numpy(a).to(dev) for a in (p.col_ptr, p.row_idx, p.val, p.y)]
    s = torch.cuda.Stream()
    Pd = pk.Problem.from_device(*t, wl.C, wl.loss, stream=s)
    Ph = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        _, wd, sd, _ = Pd.solve(wl.P, wl.eps, 0)
        _, wh, sh, _ = Ph.solve(wl.P, wl.eps, 0)
        assert sd["epochs"] == sh["epochs"]
        assert sd["F_final"] == pytest.approx(sh["F_final"], rel=1e-12)
        np.testing.assert_allclose(wd, wh, atol=1e-9)
    finally:
        Pd.close()
        Ph.close()


@pytest.mark.parametrize("case", ["rows_not_ascending", "row_out_of_range", "nan_value", "bad_label",
                                  "col_ptr_decreasing"])
def test_device_create_rejects_bad_input(pk, case):
    """Validation on the device (pcdn_create_device), with the fault placed inside the longest
    (Zipf head) column, which the entry-parallel order check spreads over many threads."""
    import torch
    wl, p = problem("svm_20k_100k")
    cp, ri, vv, yy = p.col_ptr.copy(), p.row_idx.copy(), p.val.copy(), p.y.copy()
    j = int(np.argmax(np.diff(cp)))
    a = int(cp[j] + (cp[j + 1] - cp[j]) // 2)
    if case == "rows_not_ascending":
        ri[a], ri[a + 1] = ri[a + 1], ri[a]
    elif case == "row_out_of_range":
        ri[a] = p.n_samples
    elif case == "nan_value":
        vv[a] = np.nan
    elif case == "bad_label":
        yy[3] = 0
    elif case == "col_ptr_decreasing":
        cp[j + 1] = cp[j] - 1
    dev = torch.device("cuda:0")
    t = [torch.from_numpy(x).to(dev) for x in (cp, ri, vv, yy)]
    with pytest.raises(pk.PcdnError) as ei:
        pk.Problem.from_device(*t, wl.C, wl.loss)
    assert ei.value.code == pk.PCDN_EINVAL
    # the context is intact: the unmodified problem creates and solves
    t = [torch.from_numpy(x).to(dev) for x in (p.col_ptr, p.row_idx, p.val, p.y)]
    q = pk.Problem.from_device(*t, wl.C, wl.loss)
    try:
        assert q.solve(wl.P, 1e-1, 0)[2]["converged"]
    finally:
        q.close()


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_p1_and_pm(pk, loss):
    # P = 1 (CDN, Algorithm 1) and P = m (one bundle per outer iteration)
    wl, p = problem("ragged_lr")
    orc = oracle.Oracle.from_problem(p, wl.C, loss)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, loss)
    try:
        for Pb in (1, p.n_features):
            wo, so = orc.solve(Pb, eps=1e-4, seed=5, max_epochs=500)
            _, w, st, _ = P.solve(Pb, 1e-4, 5, pk.pcdn_default_opts(max_epochs=500))
            assert st["epochs"] == so["epochs"]
            assert st["F_final"] == pytest.approx(so["F_final"], rel=1e-9)
    finally:
        P.close()


def test_zero_direction_bundle(pk):
    # at w = 0 a feature with |g_j| <= 1 keeps d_j = 0; a bundle of only such features changes nothing
    wl, p = problem("lr_2k_10k")
    orc = oracle.Oracle.from_problem(p, 1e-3, wl.loss)  # tiny c: every |g_j| < 1
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, 1e-3, wl.loss)
    try:
        B = np.arange(64, dtype=np.int32)
        r = P.bundle_step(np.zeros(p.n_features), B)
        assert np.all(r["d"] == 0) and r["q"] == 0 and r["alpha"] == 1.0 and r["dF"] == 0.0 and r["Delta"] == 0.0
        np.testing.assert_array_equal(P.get_w(), 0.0)
        _, _, ro = orc.bundle_step(np.zeros(p.n_features), orc.maintained(np.zeros(p.n_features)), B)
        assert np.all(ro["d"] == 0)
    finally:
        P.close()


def test_errors_and_bounded_wait(pk):
    wl, p = problem("svm_20k_100k")
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        with pytest.raises(pk.PcdnError) as ei:
            P.bundle_step(None, np.array([1, 2, 1], dtype=np.int32))
        assert ei.value.code == pk.PCDN_EINVAL
        with pytest.raises(pk.PcdnError) as ei:
            P.solve(0, 1e-3, 0)
        assert ei.value.code == pk.PCDN_EINVAL
        # a wait between blocks that gives up at once: the launch ends with PCDN_ETIMEOUT and the
        # context stays usable
        opts = pk.pcdn_default_opts(grid_ctas=100000, spin_limit=1, max_epochs=1)
        with pytest.raises(pk.PcdnError) as ei:
            P.solve(1024, 1e-3, 0, opts)
        assert ei.value.code == pk.PCDN_ETIMEOUT
        rc, w, st, _ = P.solve(wl.P, wl.eps, 0)
        assert st["converged"]
    finally:
        P.close()
