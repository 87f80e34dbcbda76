"""Pins of the oracle's separable penalty (no GPU).

The concluding remarks state that PCDN extends to a convex twice-differentiable loss plus a
separable penalty, covering L1, L2 and their mixture; the oracle minimises
F(w) = c sum_i phi + l1 ||w||_1 + (l2/2) ||w||^2.  The pins take derivatives of the smooth part by
finite differences, directions from a brute-force 1-D minimisation of the penalised model, optima
from FISTA with the same penalty and, for ridge (l1 = 0), from L-BFGS on the smooth objective.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import datagen
import oracle
from tests import np_defs as D
from tests.test_oracle import rand_w, tiny

PENALTIES = [(1.0, 0.5), (0.3, 2.0), (0.0, 1.0)]


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
@pytest.mark.parametrize("l1,l2", PENALTIES)
def test_full_bundle_step_is_the_penalised_proximal_newton_step(loss, l1, l2):
    """P = m: the direction minimises g t + h t^2/2 + (l2/2)(w + t)^2 + l1 |w + t| per feature (g by
    finite differences of the loss, h pinned elsewhere), Delta is Eq. 7 for the smooth part
    c L + (l2/2)||w||^2, and the accepted step is the first one that passes the Armijo test on the
    penalised objective."""
    p, X, y = tiny(loss, n=40, m=10, seed=3, density=0.5)
    c = 0.8
    o = oracle.Oracle.from_problem(p, c, loss, l1=l1, l2=l2)
    rng = np.random.default_rng(4)
    ar = oracle.Armijo()
    for _ in range(4):
        w = rand_w(p.n_features, rng, scale=0.5)
        mq = o.maintained(w)
        B = np.arange(p.n_features)
        w1, _, r = o.bundle_step(w, mq, B, armijo=ar)
        g = np.array([D.fd_grad(X, y, w, c, loss, j) for j in B])
        h = np.array([o.grad_hess(mq, j)[1] for j in B])
        d = np.array([D.ternary_min(lambda t, j=j: g[j] * t + 0.5 * h[j] * t * t + 0.5 * l2 * (w[j] + t) ** 2
                                    + l1 * abs(w[j] + t), -50, 50) for j in B])
        np.testing.assert_allclose(r["d"], d, rtol=1e-5, atol=1e-7)
        gs = np.array([D.fd_grad_smooth(X, y, w, c, loss, j, l2) for j in B])
        Delta = float(gs @ d + l1 * (np.abs(w + d).sum() - np.abs(w).sum()))
        assert r["Delta"] == pytest.approx(Delta, rel=1e-5, abs=1e-7)
        F0 = D.F_pen(X, y, w, c, loss, l1, l2)
        a = 1.0
        for q in range(ar.q_max):
            if D.F_pen(X, y, w + a * d, c, loss, l1, l2) - F0 <= ar.sigma * a * Delta:
                break
            a *= ar.beta
        assert r["alpha"] == a
        assert o.objective(w1) == pytest.approx(D.F_pen(X, y, w1, c, loss, l1, l2), rel=1e-12)


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
@pytest.mark.parametrize("l1,l2", PENALTIES)
def test_penalised_line_search_equals_direct(loss, l1, l2):
    p, X, y = tiny(loss, n=60, m=20, seed=7, density=0.3)
    o = oracle.Oracle.from_problem(p, 1.3, loss, l1=l1, l2=l2)
    rng = np.random.default_rng(8)
    for _ in range(5):
        w = rand_w(p.n_features, rng)
        mq = o.maintained(w)
        B = rng.permutation(p.n_features)[:7].astype(np.int32)
        _, _, a = o.bundle_step(w, mq, B)
        _, _, b = o.bundle_step(w, mq, B, direct=True)
        assert a["q"] == b["q"] and a["alpha"] == b["alpha"]
        assert a["dF"] == pytest.approx(b["dF"], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
@pytest.mark.parametrize("l1,l2", PENALTIES)
def test_kkt_is_the_penalised_min_norm_subgradient(loss, l1, l2):
    p, X, y = tiny(loss, seed=5)
    c = 1.1
    o = oracle.Oracle.from_problem(p, c, loss, l1=l1, l2=l2)
    rng = np.random.default_rng(15)
    for _ in range(5):
        w = rand_w(p.n_features, rng)
        g = np.array([D.fd_grad_smooth(X, y, w, c, loss, j, l2) for j in range(p.n_features)])
        v = D.min_norm_subgradient(g, w, l1)
        assert o.kkt_l1(w) == pytest.approx(np.abs(v).sum(), rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("loss,c,P", [("logistic", 1.0, 3), ("l2svm", 0.5, 4)])
@pytest.mark.parametrize("l1,l2", PENALTIES)
def test_penalised_solve_reaches_the_fista_optimum(loss, c, P, l1, l2):
    p, X, y = tiny(loss, n=30, m=12, seed=21, density=0.45)
    o = oracle.Oracle.from_problem(p, c, loss, l1=l1, l2=l2)
    w, st = o.solve(P, eps=1e-10, seed=2, max_epochs=20000)
    assert st["converged"]
    wf = D.fista(X, y, c, loss, l1=l1, l2=l2)
    assert st["F_final"] == pytest.approx(D.F_pen(X, y, wf, c, loss, l1, l2), rel=1e-9)
    # l2 > 0 makes the objective strongly convex: the minimiser is unique
    np.testing.assert_allclose(w, wf, atol=1e-5)


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_ridge_solution_matches_lbfgs(loss):
    """l1 = 0: a smooth, strongly convex problem; L-BFGS (scipy) on F finds the same minimiser."""
    spec = datagen.Spec(300, 80, "zipf", row_mean=20.0, zipf_s=1.1, values="tfidf", wstar_nnz=10, flip_frac=0.05,
                        seed=12)
    p = datagen.generate(spec, with_csr=False)
    X = sp.csc_matrix((p.val.astype(np.float64), p.row_idx, p.col_ptr), shape=(p.n_samples, p.n_features))
    y = p.y.astype(np.float64)
    c, l2 = 1.0, 0.7
    o = oracle.Oracle.from_problem(p, c, loss, l1=0.0, l2=l2)
    w, st = o.solve(16, eps=1e-11, seed=3, max_epochs=20000)
    assert st["converged"]

    def fun(v):
        return D.F_pen(X, y, v, c, loss, 0.0, l2), D.grad(X, y, v, c, loss) + l2 * v

    r = so.minimize(fun, np.zeros(p.n_features), jac=True, method="L-BFGS-B",
                    options=dict(maxiter=20000, gtol=1e-12, ftol=1e-15))
    assert st["F_final"] == pytest.approx(r.fun, rel=1e-10)
    np.testing.assert_allclose(w, r.x, atol=1e-6)


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_p1_is_cdn_with_a_penalty(loss):
    p, X, y = tiny(loss, n=200, m=60, seed=2, density=0.2)
    o = oracle.Oracle.from_problem(p, 1.0, loss, l1=0.4, l2=1.5)
    w0 = np.zeros(p.n_features)
    w_pcdn, st = o.solve(1, eps=1e-12, seed=17, max_epochs=5, bundle_limit=p.n_features)
    w_cdn, _ = o.cdn_epoch(w0, o.maintained(w0), seed=17, epoch=0)
    np.testing.assert_array_equal(w_pcdn, w_cdn)


@pytest.mark.parametrize("l1,l2", [(1.0, 0.5), (0.3, 2.0)])
def test_shrinking_with_a_penalty(l1, l2):
    """The active set keeps w_j != 0 or |g_j| >= l1 - M/s, g the smooth part's gradient (matrix form)
    and M the largest |v_j| of the penalised minimum-norm subgradient."""
    spec = datagen.Spec(800, 2000, "zipf", row_mean=30.0, zipf_s=1.1, values="tfidf", wstar_nnz=20, flip_frac=0.05,
                        seed=11)
    p = datagen.generate(spec, with_csr=False)
    X = sp.csc_matrix((p.val.astype(np.float64), p.row_idx, p.col_ptr), shape=(p.n_samples, p.n_features))
    y = p.y.astype(np.float64)
    o = oracle.Oracle.from_problem(p, 1.0, "logistic", l1=l1, l2=l2)
    rng = np.random.default_rng(3)
    for _ in range(3):
        w = np.where(rng.random(p.n_features) < 0.02, rng.normal(0, 1.5, p.n_features), 0.0)
        g = D.grad(X, y, w, 1.0, "logistic") + l2 * w
        v = D.min_norm_subgradient(g, w, l1)
        M = float(np.abs(v).max())
        active = (w != 0) | (np.abs(g) >= l1 - M / p.n_samples)
        mask, Mo = o.active_set(w)
        np.testing.assert_array_equal(mask, active)
        assert Mo == pytest.approx(M, rel=1e-9)
    w, st = o.solve(16, eps=1e-3, seed=6, shrink=True)
    assert st["converged"]
