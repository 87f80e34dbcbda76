"""The separable penalty l1 ||w||_1 + (l2/2) ||w||^2 (pcdn_set_penalty: L1, ridge, elastic net) on the
GPU vs the oracle with the same penalty, through the C ABI, on identical seeded inputs and bundles.

Tolerances as for the paper's penalty (test_gpu_parity.py): FP64 mode g, h, d, Delta within 1e-9
of the bundle's largest magnitude, q and alpha equal, whole solves on the same trajectory with the
final objective within 1e-6 relative; mixed mode g, h within 1e-5, d within 1e-5 of
max|g| / h_j + |d_j| (the FP32 sums' error is on the bundle's |g| scale, and a ridge direction
-g/h has no threshold to absorb it), q and alpha equal unless the oracle's Armijo margin is within
1e-5, final objective within 1e-6 relative.  Objective and KKT at random points within 1e-12 / 1e-10.
"""
import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import margin_small, problem, rel_err

pytestmark = pytest.mark.gpu

PENALTIES = [(1.0, 0.5), (0.3, 2.0), (0.0, 1.0)]


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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("l1,l2", PENALTIES)
@pytest.mark.parametrize("name,Pb,grid", [("lr_2k_10k", 64, 0), ("svm_20k_100k", 1024, 0), ("ragged_lr", 100, 1)])
def test_penalised_bundle_step_parity(pk, name, Pb, grid, l1, l2, prec):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss, l1=l1, l2=l2)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    P.set_penalty(l1, l2)
    opts = pk.pcdn_default_opts(prec=prec, grid_ctas=(grid if grid else 100000))
    armijo = oracle.Armijo()
    tol = 1e-9 if prec == "fp64" else 1e-5
    try:
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
                # the FP32 column sums' error is on the bundle's |g| scale (the g check above); without an
                # L1 threshold (ridge) every d = -g/h carries it, so d is held to that scale over h
                dscale = np.max(np.abs(ro["g"])) / ro["h"] + np.abs(ro["d"])
                assert np.all(np.abs(r["d"] - ro["d"]) <= tol * dscale + 1e-300), ("d (Newton scale)",)
                assert abs(r["Delta"] - ro["Delta"]) <= tol * max(abs(ro["Delta"]), 1e-300) + 1e-300
                if r["q"] != ro["q"]:
                    assert prec == "mixed" and margin_small(orc, w, ro, B, r["q"], ro["q"], armijo, 1e-5), \
                        (r["q"], ro["q"], r["dF"], ro["dF"])
                    continue
                assert r["alpha"] == ro["alpha"]
                if ro["dF"] != 0.0:
                    dtol = 1e-7 if prec == "fp64" else 1e-4
                    assert abs(r["dF"] - ro["dF"]) <= dtol * abs(ro["dF"]) + 1e-12 * abs(ro["Delta"]), \
                        (r["dF"], ro["dF"])
    finally:
        P.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("l1,l2", PENALTIES)
@pytest.mark.parametrize("name,Pb", [("lr_2k_10k", 64), ("svm_20k_100k", 256)])
def test_penalised_solve_parity(pk, name, Pb, l1, l2, prec):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss, l1=l1, l2=l2)
    wo, so = orc.solve(Pb, eps=wl.eps, seed=wl.solver_seed, trace=True, max_epochs=300)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    P.set_penalty(l1, l2)
    try:
        opts = pk.pcdn_default_opts(prec=prec, max_epochs=300)
        rc, w, st, tr = P.solve(Pb, wl.eps, wl.solver_seed, opts, trace_bundles=int(so["bundles"]) + 8,
                                trace_epochs=300)
        assert st["converged"] and so["converged"]
        assert abs(st["F_final"] - so["F_final"]) <= 1e-6 * abs(so["F_final"]), (st["F_final"], so["F_final"])
        if prec == "fp64":
            assert st["epochs"] == so["epochs"]
            n = min(len(tr["q"]), len(so["q"]))
            assert n == so["bundles"]
            assert np.mean(tr["q"][:n] == so["q"][:n]) >= 0.999
            np.testing.assert_allclose(tr["epoch_kkt"], so["epoch_kkt"], rtol=1e-6)
            np.testing.assert_allclose(w, wo, rtol=0, atol=1e-7 * max(1.0, np.abs(wo).max()))
        else:
            assert abs(st["epochs"] - so["epochs"]) <= 1
        assert np.all(tr["dF"] <= 1e-9 * abs(so["F_final"]))
        if l1 == 0.0:
            assert np.count_nonzero(w) > 0.5 * p.n_features or np.count_nonzero(wo) <= 0.5 * p.n_features
    finally:
        P.close()


@pytest.mark.parametrize("l1,l2", PENALTIES)
@pytest.mark.parametrize("name", ["lr_2k_10k", "svm_20k_100k"])
def test_penalised_objective_and_kkt(pk, name, l1, l2):
    wl, p = problem(name)
    orc = oracle.Oracle.from_problem(p, wl.C, wl.loss, l1=l1, l2=l2)
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    P.set_penalty(l1, l2)
    try:
        rng = np.random.default_rng(2)
        for _ in range(3):
            w = rng.normal(0, 0.5, p.n_features) * (rng.random(p.n_features) < 0.05)
            P.set_w(w)
            assert P.objective() == pytest.approx(orc.objective(w), rel=1e-12)
            assert P.kkt() == pytest.approx(orc.kkt_l1(w), rel=1e-10)
    finally:
        P.close()


def test_penalty_is_validated(pk):
    wl, p = problem("lr_2k_10k")
    P = pk.Problem.from_csc(p.col_ptr, p.row_idx, p.val, p.y, wl.C, wl.loss)
    try:
        for l1, l2 in [(-1.0, 0.0), (0.0, 0.0), (1.0, float("nan")), (float("inf"), 1.0), (1.0, -0.5)]:
            with pytest.raises(pk.PcdnError):
                P.set_penalty(l1, l2)
        P.set_penalty(1.0, 0.0)
    finally:
        P.close()
