"""Pins of the oracle's optional shrinking between outer iterations (no GPU).

Section 5.1 reports that the comparison's shrinking had to move out of the parallel loop; the
oracle's reading: outer iteration k >= 1 visits, in its random order (Eq. 8), only the features
with w_j != 0 or |g_j| >= 1 - M/s at w^k (M the largest |v_j| of the minimum-norm subgradient, s
the number of samples).  The pins state the active set from an independently written gradient
(Eq. 2 / Eq. 3 differentiated in matrix form) and a ternary-search minimum-norm subgradient, replay
a shrunk outer iteration with the (separately pinned) bundle step over the restricted partition,
and check that shrinking ends at the same optimum.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import datagen
import oracle
from tests import np_defs as D
from tests.test_oracle import tiny

CASES = [("logistic", 1.0, 16), ("l2svm", 0.5, 64)]


def medium(seed=11):
    spec = datagen.Spec(800, 2000, "zipf", row_mean=30.0, zipf_s=1.1, values="tfidf", wstar_nnz=20, flip_frac=0.05,
                        seed=seed)
    p = datagen.generate(spec, with_csr=False)
    X = sp.csc_matrix((p.val.astype(np.float64), p.row_idx, p.col_ptr), shape=(p.n_samples, p.n_features))
    return p, X, p.y.astype(np.float64)


def active_from_definition(X, y, w, c, loss):
    g = D.grad(X, y, w, c, loss)
    v = D.min_norm_subgradient(g, w)
    M = float(np.abs(v).max())
    return (w != 0) | (np.abs(g) >= 1.0 - M / X.shape[0]), v, M


@pytest.mark.parametrize("loss,c,P", CASES)
def test_first_outer_iteration_visits_every_feature(loss, c, P):
    p, _, _ = medium()
    o = oracle.Oracle.from_problem(p, c, loss)
    _, a = o.solve(P, eps=1e-3, seed=6, max_epochs=1, trace=True)
    _, b = o.solve(P, eps=1e-3, seed=6, max_epochs=1, trace=True, shrink=True)
    for k in ("q", "alpha", "Delta", "dF"):
        np.testing.assert_array_equal(a[k], b[k])
    assert b["epoch_active"][0] == p.n_features


@pytest.mark.parametrize("loss,c,P", CASES)
def test_active_set_from_an_independent_gradient(loss, c, P):
    p, X, y = medium()
    o = oracle.Oracle.from_problem(p, c, loss)
    for k in (1, 2):
        wk, _ = o.solve(P, eps=1e-12, seed=6, max_epochs=k, shrink=True)
        _, st = o.solve(P, eps=1e-12, seed=6, max_epochs=k + 1, shrink=True)
        active, v, M = active_from_definition(X, y, wk, c, loss)
        assert 0 < active.sum() < p.n_features
        assert st["epoch_active"][k] == active.sum()
        # a feature that violates the optimality conditions is never skipped
        assert np.all(active[np.abs(v) > 1e-9])
        mask, Mo = o.active_set(wk)
        np.testing.assert_array_equal(mask, active)
        assert Mo == pytest.approx(M, rel=1e-9)


@pytest.mark.parametrize("loss,c,P", CASES)
def test_active_set_at_random_points(loss, c, P):
    """The rule at points far from the optimum, where the margin M/s is wide enough that features
    with w_j = 0 fall on both sides of 1 - M/s and of 1."""
    p, X, y = medium()
    o = oracle.Oracle.from_problem(p, c, loss)
    rng = np.random.default_rng(3)
    in_band = 0
    for _ in range(4):
        w = np.where(rng.random(p.n_features) < 0.02, rng.normal(0, 1.5, p.n_features), 0.0)
        active, _, M = active_from_definition(X, y, w, c, loss)
        g = D.grad(X, y, w, c, loss)
        zero = w == 0
        in_band += int(np.sum(zero & (np.abs(g) >= 1.0 - M / p.n_samples) & (np.abs(g) < 1.0)))
        assert np.any(zero & ~active) and np.any(zero & active)
        mask, Mo = o.active_set(w)
        np.testing.assert_array_equal(mask, active)
        assert Mo == pytest.approx(M, rel=1e-9)
    assert in_band > 0  # the margin decided some features


@pytest.mark.parametrize("loss,c,P", CASES)
def test_shrunk_outer_iteration_is_the_restricted_partition(loss, c, P):
    """Outer iteration 1 of a shrinking solve = bundle steps over the partition of iteration 1
    restricted to the active set, in partition order, from w^1."""
    p, X, y = medium()
    o = oracle.Oracle.from_problem(p, c, loss)
    w1, s1 = o.solve(P, eps=1e-12, seed=6, max_epochs=1, shrink=True, trace=True)
    w2, s2 = o.solve(P, eps=1e-12, seed=6, max_epochs=2, shrink=True, trace=True)
    active, _, _ = active_from_definition(X, y, w1, c, loss)
    order = oracle.permutation(6, 1, p.n_features)
    order = order[active[order]]
    w = w1.copy()
    mq = o.maintained(w)
    nb1 = len(s1["q"])
    qs, alphas = [], []
    for t in range(0, len(order), P):
        w, mq, r = o.bundle_step(w, mq, order[t:t + P])
        qs.append(r["q"])
        alphas.append(r["alpha"])
    np.testing.assert_array_equal(s2["q"][nb1:], qs)
    np.testing.assert_array_equal(s2["alpha"][nb1:], alphas)
    np.testing.assert_array_equal(w2, w)


@pytest.mark.parametrize("loss,c,P", [("logistic", 1.0, 3), ("l2svm", 0.5, 4)])
def test_shrinking_reaches_the_optimum(loss, c, P):
    p, X, y = tiny(loss, n=30, m=12, seed=21, density=0.45)
    o = oracle.Oracle.from_problem(p, c, loss)
    w, st = o.solve(P, eps=1e-10, seed=2, max_epochs=20000, shrink=True)
    assert st["converged"]
    assert st["F_final"] == pytest.approx(D.F(X, y, D.fista(X, y, c, loss), c, loss), rel=1e-9)


@pytest.mark.parametrize("loss,c,P", CASES)
def test_shrinking_descends_to_the_plain_optimum(loss, c, P):
    p, _, _ = medium()
    o = oracle.Oracle.from_problem(p, c, loss)
    w, st = o.solve(P, eps=1e-3, seed=6, shrink=True, trace=True)
    assert st["converged"]
    assert np.all(np.diff(st["epoch_F"]) <= 1e-10 * abs(st["epoch_F"][0]))
    assert np.all(st["epoch_active"][1:] < p.n_features)
    assert st["coord_updates"] == st["epoch_active"].sum()
    _, a = o.solve(P, eps=1e-9, seed=6, max_epochs=5000)
    _, b = o.solve(P, eps=1e-9, seed=6, max_epochs=5000, shrink=True)
    assert a["converged"] and b["converged"]
    assert b["F_final"] == pytest.approx(a["F_final"], rel=1e-8)
