"""Shrinking between outer iterations (pcdn_opts.shrink) on the GPU vs the oracle's shrinking, through
the C ABI, on identical seeded inputs and partitions.

Both sides decide the active set of outer iteration k from the gradient of the stopping test after
iteration k - 1 (feature j kept when w_j != 0 or |g_j| >= 1 - M/s).  A feature whose |g_j| lies
within rounding of the bound may go either way: in mixed mode through the FP32 column sums, in FP64
mode through the order of the floating-point atomic adds of d^T x_i, which varies run to run.  Where
the two sides took the same decisions (equal active-set sizes in every outer iteration), the FP64
trajectories must agree as the plain ones do: same outer iterations and accepted steps, final
objective within 1e-6 relative.  Where a decision went the other way the trajectories part; both
stop at a relative KKT of eps, where F is still well above F* (0.65 % on the 20k x 100k SVM), so
the result is held to the oracle's own accuracy instead: F - F* at most twice the oracle's F - F*
plus 1e-6 |F*| (F* from the oracle at a relative KKT of 1e-6), or, along warm-started batch paths,
a relative KKT within 1.5 eps by the oracle's FP64 measure at the GPU's w.
"""
import numpy as np
import pytest

import datagen
import oracle
from tests.test_gpu_parity import problem

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


_FSTAR = {}


def f_star(name, Pb):
    """The oracle's objective at a relative KKT of 1e-6 (within 1e-7 relative of F* on these workloads)."""
    if (name, Pb) not in _FSTAR:
        wl, p = problem(name)
        orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
        _, st = orc.solve(Pb, eps=1e-6, seed=wl.solver_seed, max_epochs=5000, shrink=True)
        assert st["converged"]
        _FSTAR[(name, Pb)] = st["F_final"]
    return _FSTAR[(name, Pb)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,Pb,grid", [("lr_2k_10k", 64, 0), ("svm_20k_100k", 256, 0), ("ragged_svm", 97, 100000),
                                          ("ragged_lr", 100, 1)])
def test_shrink_solve_parity(pk, name, Pb, grid, prec):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss)
    wo, so = orc.solve(Pb, eps=wl.eps, seed=wl.solver_seed, trace=True, max_epochs=300, shrink=True)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        opts = pk.pcdn_default_opts(prec=prec, grid_ctas=grid, max_epochs=300, shrink=1)
        rc, w, st, tr = P.solve(Pb, wl.eps, wl.solver_seed, opts, trace_bundles=int(so["bundles"]) + 64,
                                trace_epochs=300)
        assert st["converged"] and so["converged"]
        fa, oa = tr["epoch_features"], so["epoch_active"]
        same = np.array_equal(fa, oa)
        if prec == "fp64" and same:
            assert abs(st["F_final"] - so["F_final"]) <= 1e-6 * abs(so["F_final"]), (st["F_final"], so["F_final"])
        else:
            Fs = f_star(name, Pb)
            gap_or = so["F_final"] - Fs
            assert gap_or >= -1e-6 * abs(Fs)
            assert -1e-6 * abs(Fs) <= st["F_final"] - Fs <= 2 * max(gap_or, 0.0) + 1e-6 * abs(Fs), \
                (st["F_final"], so["F_final"], Fs)
        assert fa[0] == p.n_features and oa[0] == p.n_features
        assert so["epochs"] == 1 or np.all(oa[1:] < p.n_features)
        # the walker visited exactly the features the host planned
        assert st["coord_updates"] == int(fa.sum())
        if st["epochs"] > 1:
            assert st["nnz_visited"] < st["epochs"] * p.nnz
        n_ep = min(len(fa), len(oa))
        if prec == "fp64" and same:
            assert st["epochs"] == so["epochs"]
            n = min(len(tr["q"]), len(so["q"]))
            assert n == so["bundles"]
            assert np.mean(tr["q"][:n] == so["q"][:n]) >= 0.999
            np.testing.assert_allclose(tr["epoch_kkt"], so["epoch_kkt"], rtol=1e-6)
        elif prec == "fp64":
            # the first decision that went the other way moved at most a couple of features
            first = int(np.argmax(fa[:n_ep] != oa[:n_ep])) if np.any(fa[:n_ep] != oa[:n_ep]) else n_ep
            if first < n_ep:
                assert abs(int(fa[first]) - int(oa[first])) <= 2, (fa, oa)
        else:
            assert np.all(np.abs(fa[:n_ep] - oa[:n_ep]) <= 0.02 * p.n_features)
        # F is non-increasing bundle by bundle (Lemma 1(c))
        assert np.all(tr["dF"] <= 1e-9 * abs(so["F_final"]))
    finally:
        P.close()


def test_shrink_first_outer_iteration_is_plain(pk):
    wl, p = problem("svm_20k_100k")
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        nb = (p.n_features + 255) // 256
        out = []
        for shrink in (0, 1):
            opts = pk.pcdn_default_opts(prec="fp64", max_epochs=1, shrink=shrink)
            rc, w, st, tr = P.solve(256, 1e-9, 3, opts, trace_bundles=nb, trace_epochs=1)
            out.append((w, st, tr))
        (w0, s0, t0), (w1, s1, t1) = out
        assert s0["bundles"] == s1["bundles"] == nb
        assert np.mean(t0["q"] == t1["q"]) >= 0.999
        assert t1["epoch_features"][0] == p.n_features
        assert s1["F_final"] == pytest.approx(s0["F_final"], rel=1e-12)
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shrink_batch_path_matches_oracle(pk, prec):
    """Shrinking solves issued by the batch solver (tasks, not captured as graphs) along warm-started
    C paths, against the oracle's shrinking solves along the same path: the oracle's answer where the
    decisions coincided (FP64), else a valid eps-solution by the oracle's measure (module docstring)."""
    jobs = datagen.batch_jobs(4, seed=5, scale=0.05, n_C=3, C_range=(0.05, 5.0))
    items = [(j, datagen.generate(j.spec, with_csr=False)) for j in jobs]
    probs = [pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, j.C_path[0], j.loss) for j, p in items]
    try:
        Ps = [min(64, p.n_features) for _, p in items]
        opts = pk.pcdn_default_opts(prec=prec, max_epochs=400, shrink=1)
        rc, res, bs = pk.pcdn_solve_batch([q.handle for q in probs], [q.n_features for q in probs],
                                          [j.C_path for j, _ in items], Ps, eps=1e-3, seed=9, opts=opts)
        assert rc == pk.PCDN_OK
        assert bs["graph_solves"] == 0
        for k, (job, p) in enumerate(items):
            w = ws = None
            for ci, C in enumerate(job.C_path):
                orc = oracle.Oracle.from_problem(p, C, job.loss)
                w, so = orc.solve(Ps[k], eps=1e-3, seed=9, w0=w, max_epochs=400, shrink=True)
                st = res[k]["stats"][ci]
                assert st["converged"] and so["converged"]
                if prec == "fp64" and st["epochs"] == so["epochs"] and \
                        abs(st["F_final"] - so["F_final"]) <= 1e-6 * abs(so["F_final"]):
                    pass  # the same decisions: the same answer as the oracle
                else:
                    # a valid answer by the oracle's FP64 measure: the relative KKT at the GPU's w, against
                    # the GPU's start point (the previous C's solution), within 1.5 eps; and F not below F*
                    w_prev = res[k]["w"][ci - 1] if ci else np.zeros(p.n_features)
                    k0, k1 = orc.kkt_l1(w_prev), orc.kkt_l1(res[k]["w"][ci])
                    ws, ss = orc.solve(Ps[k], eps=1e-6, seed=9, w0=ws, max_epochs=5000, shrink=True)
                    Fs = ss["F_final"]
                    diag = (k, ci, k1 / k0, st["kkt_rel"], st["kkt0"], k0, st["F_final"], so["F_final"], Fs,
                            st["epochs"], so["epochs"])
                    assert k1 <= 1.5e-3 * k0, diag
                    assert st["F_final"] >= Fs - 1e-6 * abs(Fs), diag
                assert st["nnz_visited"] <= st["epochs"] * p.nnz
    finally:
        for q in probs:
            q.close()


def test_shrink_option_is_validated(pk):
    wl, p = problem("lr_2k_10k")
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        with pytest.raises(pk.PcdnError) as e:
            P.solve(64, 1e-3, 0, pk.pcdn_default_opts(shrink=2))
        assert "shrink" in str(e.value)
    finally:
        P.close()
