"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it checks.  None of them re-types the oracle's own
formula for the quantity it pins: derivatives come from finite differences of
the objective's definition (Eq. 1-3), directions from a brute-force 1-D
minimisation, line-search values from direct objective differences, optima
from FISTA, bundle statistics from the closed form of Lemma 1(a).
"""
import math

import numpy as np
import pytest

import datagen
import oracle
from tests import np_defs as D


def tiny(loss="logistic", n=30, m=12, seed=1, kind="uniform", density=0.35, flip=0.1, wstar=4):
    if kind == "uniform":
        spec = datagen.Spec(n, m, "uniform", density=density, values="halfnormal", wstar_nnz=wstar,
                            flip_frac=flip, seed=seed)
    else:
        spec = datagen.Spec(n, m, "zipf", row_mean=max(1.0, m / 4), zipf_s=1.1, values="tfidf", wstar_nnz=wstar,
                            flip_frac=flip, seed=seed)
    p = datagen.generate(spec)
    return p, p.dense(), p.y.astype(np.float64)


def rand_w(m, rng, frac=0.6, scale=0.7):
    w = rng.normal(0, scale, m)
    w[rng.random(m) > frac] = 0.0
    return w


# ---------------------------------------------------------------- splitmix64 / partition (Eq. 8)

def test_splitmix64_published_first_output():
    # Reference splitmix64 started at state 0: first output 0xE220A8397B1DCDAF (Steele, Lea, Flood 2014)
    assert oracle.splitmix64_output(0, 1) == 0xE220A8397B1DCDAF
    assert D.splitmix64_outputs(0, 1)[0] == 0xE220A8397B1DCDAF


def test_splitmix64_matches_independent_python():
    rng = np.random.default_rng(5)
    for _ in range(50):
        s0 = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        outs = D.splitmix64_outputs(s0, 7)
        for k in range(1, 8):
            assert oracle.splitmix64_output(s0, k) == outs[k - 1]


@pytest.mark.parametrize("m", [1, 2, 7, 64, 1000])
def test_partition_is_sorted_key_order(m):
    # Algorithm 3 / Eq. 8: a random disjoint partition, drawn (the paper leaves the draw open) as the order of
    # per-feature splitmix64 keys (ties broken by feature index).
    for seed, epoch in [(0, 0), (0, 1), (12345, 7), (2**64 - 1, 3)]:
        perm = oracle.permutation(seed, epoch, m)
        assert sorted(perm.tolist()) == list(range(m))
        s_epoch = D.splitmix64_outputs(seed ^ ((epoch * 0xD1B54A32D192ED03) & D.MASK64), 1)[0]
        keys = D.splitmix64_outputs(s_epoch, m)
        expect = sorted(range(m), key=lambda j: (keys[j], j))
        assert perm.tolist() == expect


def test_partition_changes_between_epochs():
    a = oracle.permutation(0, 0, 500)
    b = oracle.permutation(0, 1, 500)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, oracle.permutation(0, 0, 500))


def test_expected_lambda_bar_closed_form():
    # Lemma 1(a), closed form of E[lambda_bar(B)] (Appendix A): a bundle of the random partition is a
    # uniformly random P-subset, so the Monte Carlo mean of max_{j in B} (X^T X)_jj must match it.
    rng = np.random.default_rng(3)
    m, P = 40, 5
    lam = rng.gamma(2.0, 1.0, m)
    samples = []
    for epoch in range(3000):
        perm = oracle.permutation(99, epoch, m)
        for t in range(m // P):
            samples.append(lam[perm[t * P:(t + 1) * P]].max())
    samples = np.array(samples)
    expect = D.expected_lambda_bar(lam, P)
    se = samples.std() / math.sqrt(samples.size)
    assert abs(samples.mean() - expect) < 4 * se, (samples.mean(), expect, se)
    # Lemma 1(a): E[lambda_bar]/P decreases and E[lambda_bar] increases with P
    vals = [D.expected_lambda_bar(lam, p) for p in range(1, m + 1)]
    assert all(vals[i] <= vals[i + 1] + 1e-12 for i in range(m - 1))
    assert all(vals[i] / (i + 1) > vals[i + 1] / (i + 2) for i in range(m - 1))


# ---------------------------------------------------------------- direction (Eq. 4, Eq. 5)

@pytest.mark.parametrize("g,h,w,expect", [
    (-3.0, 2.0, 0.0, 1.0),      # g + 1 <= h w   -> -(g+1)/h
    (3.0, 2.0, 0.0, -1.0),      # g - 1 >= h w   -> -(g-1)/h
    (0.5, 1.0, 0.0, 0.0),       # |g| < 1 at w = 0 -> stays at 0
    (0.5, 1.0, 2.0, -1.5),      # g + 1 <= h w with w > 0
    (-0.5, 1.0, -2.0, 1.5),     # g - 1 >= h w with w < 0
    (0.2, 4.0, 0.1, -0.1),      # interior: d = -w
    (1.0, 2.0, 1.0, -1.0),      # g + 1 == h w: both branches give -w
    (-1.0, 2.0, -1.0, 1.0),     # g - 1 == h w
])
def test_direction_hand_cases(g, h, w, expect):
    assert oracle.direction(g, h, w) == pytest.approx(expect, abs=1e-15)


def test_direction_is_brute_force_argmin():
    # Eq. 4: d = argmin g d + h d^2 / 2 + |w + d|, checked by ternary search on the convex model.
    rng = np.random.default_rng(7)
    for _ in range(400):
        g = rng.normal(0, 2)
        h = 10 ** rng.uniform(-3, 2)
        w = rng.normal(0, 1) if rng.random() < 0.7 else 0.0
        f = lambda d: g * d + 0.5 * h * d * d + abs(w + d)
        span = 10 + (abs(g) + 1) / h + abs(w)
        dref = D.ternary_min(f, -span, span)
        d = oracle.direction(g, h, w)
        # a comparison search resolves the minimiser only to where f is flat within rounding
        res = 10 * math.sqrt(4e-16 * max(1.0, abs(f(dref))) / h) + 1e-9 * span
        assert abs(d - dref) <= res, (g, h, w, d, dref)
        assert f(d) <= f(dref) + 1e-12 * max(1.0, abs(f(dref)))


# ---------------------------------------------------------------- gradient / Hessian (Eq. 11, Lemma 1(b))

@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_gradient_matches_finite_differences(loss):
    p, X, y = tiny(loss)
    o = oracle.Oracle.from_problem(p, 0.7, loss)
    rng = np.random.default_rng(11)
    for _ in range(5):
        w = rand_w(p.n_features, rng)
        mq = o.maintained(w)
        for j in range(p.n_features):
            g, h = o.grad_hess(mq, j)
            gfd = D.fd_grad(X, y, w, 0.7, loss, j)
            assert g == pytest.approx(gfd, rel=1e-6, abs=1e-8)


def test_logistic_hessian_matches_second_differences():
    p, X, y = tiny("logistic")
    o = oracle.Oracle.from_problem(p, 1.3, "logistic")
    rng = np.random.default_rng(12)
    for _ in range(5):
        w = rand_w(p.n_features, rng)
        mq = o.maintained(w)
        for j in range(p.n_features):
            g, h = o.grad_hess(mq, j)
            if h <= 1e-12:
                continue
            assert h == pytest.approx(D.fd_hess(X, y, w, 1.3, "logistic", j), rel=2e-5, abs=1e-7)


def test_svm_generalised_hessian_matches_second_differences():
    # Appendix A, proof of Lemma 1(b): the generalised Hessian 2c sum_{i in I(w)} x_ij^2; along e_j the
    # loss is piecewise quadratic, so the second difference is exact when no margin crosses 1.
    p, X, y = tiny("l2svm", seed=4)
    c = 0.9
    o = oracle.Oracle.from_problem(p, c, "l2svm")
    rng = np.random.default_rng(13)
    checked = 0
    eps = 1e-2  # exact for a quadratic piece; large enough that rounding stays far below the tolerance
    for _ in range(30):
        w = rand_w(p.n_features, rng)
        mq = o.maintained(w)
        for j in range(p.n_features):
            b0 = 1 - y * (X @ w)
            bp, bm = b0 - eps * y * X[:, j], b0 + eps * y * X[:, j]
            if np.any(np.sign(bp) != np.sign(b0)) or np.any(np.sign(bm) != np.sign(b0)):
                continue
            g, h = o.grad_hess(mq, j)
            if not np.any((b0 > 0) & (X[:, j] != 0)):
                assert h == 1e-12  # nu replaces h <= 0
                continue
            assert h == pytest.approx(D.fd_hess(X, y, w, c, "l2svm", j, eps), rel=1e-8)
            checked += 1
    assert checked > 20


def test_nu_replaces_zero_hessian():
    # Appendix A, proof of Lemma 1(b): nu = 1e-12 stands in for a (generalised) Hessian diagonal <= 0.
    # L2-SVM with every margin met (y_i w^T x_i >= 1): I(w) is empty, so g_j = 0 and h_j = nu.
    X = np.array([[1.0, 0.5, 0.0], [0.5, 1.0, 0.0], [1.0, 1.0, 0.0]])
    y = np.array([1, 1, 1], dtype=np.int8)
    cp, ri, vv = D.dense_to_csc(X)
    w = np.array([5.0, 5.0, 0.0])  # every margin y_i w^T x_i >= 7.5
    for loss in ("l2svm", "logistic"):
        o = oracle.Oracle(cp, ri, vv, y, 1.0, loss)
        mq = o.maintained(w)
        g2, h2 = o.grad_hess(mq, 2)  # empty column: both losses
        assert g2 == 0.0 and h2 == 1e-12
        if loss == "l2svm":
            for j in (0, 1):
                g, h = o.grad_hess(mq, j)
                assert g == 0.0 and h == 1e-12


@pytest.mark.parametrize("loss,theta", [("logistic", 0.25), ("l2svm", 2.0)])
def test_hessian_upper_bound(loss, theta):
    # Lemma 1(b), Eq. 12: h_j <= theta c (X^T X)_jj
    p, X, y = tiny(loss, n=60, m=20, seed=6)
    c = 2.0
    o = oracle.Oracle.from_problem(p, c, loss)
    rng = np.random.default_rng(14)
    diag = (X * X).sum(0)
    for _ in range(10):
        w = rand_w(p.n_features, rng, scale=3.0)
        mq = o.maintained(w)
        for j in range(p.n_features):
            g, h = o.grad_hess(mq, j)
            assert h <= theta * c * diag[j] * (1 + 1e-12) + 1e-12


# ---------------------------------------------------------------- line search (Eq. 6, Eq. 7, Eq. 10)

def _state_after(o, P, epochs_frac=0.5, seed=0):
    """A non-trivial (w, maintained) pair: PCDN run for part of an epoch from w = 0."""
    nb = (o.m + P - 1) // P
    w, _ = o.solve(P, eps=1e-12, seed=seed, max_epochs=3, bundle_limit=max(1, int(nb * epochs_frac)))
    return w, o.maintained(w)


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_maintained_line_search_equals_direct(loss):
    # Section 3.1: the test of Eq. 10 through maintained quantities is equivalent to Eq. 6.
    p, X, y = tiny(loss, n=80, m=30, seed=8)
    c = 1.5
    o = oracle.Oracle.from_problem(p, c, loss)
    w, mq = _state_after(o, 6)
    rng = np.random.default_rng(9)
    for _ in range(30):
        B = rng.choice(p.n_features, size=int(rng.integers(1, p.n_features + 1)), replace=False)
        w1, mq1, r1 = o.bundle_step(w, mq, B, direct=False)
        w2, mq2, r2 = o.bundle_step(w, mq, B, direct=True)
        assert r1["q"] == r2["q"] and r1["alpha"] == r2["alpha"]
        assert r1["dF"] == pytest.approx(r2["dF"], rel=1e-9, abs=1e-11)
        # and against the objective's definition evaluated on the dense matrix
        if r1["status"] == 0:
            dF_def = D.F(X, y, w1, c, loss) - D.F(X, y, w, c, loss)
            assert r1["dF"] == pytest.approx(dF_def, rel=1e-9, abs=1e-11)
            # maintained quantities after the update equal a recomputation from w (Algorithm 4)
            np.testing.assert_allclose(mq1, o.maintained(w1), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("scale", [30.0, 80.0, 400.0])
def test_maintained_line_search_exact_at_extreme_margins(scale):
    # Section 3.1: Eq. 10 is the objective change of Eq. 6.  With |w^T x_i| in the tens or hundreds
    # (saturated samples), the maintained value must still equal the objective difference from the
    # definition, and no ascent step may be accepted (Lemma 1(c)).
    p, X, y = tiny("logistic", n=60, m=16, seed=31, density=0.5)
    o = oracle.Oracle.from_problem(p, 1.0, "logistic")
    rng = np.random.default_rng(int(scale))
    accepted = 0
    for trial in range(12):
        w = rand_w(p.n_features, rng, frac=0.8, scale=scale / 4)
        z = X @ w
        if np.abs(z).max() > 700:
            continue
        mq = o.maintained(w)
        B = rng.choice(p.n_features, size=8, replace=False)
        w1, _, r = o.bundle_step(w, mq, B)
        if r["status"] != 0:
            continue
        F0 = D.F(X, y, w, 1.0, "logistic")
        dF_def = D.F(X, y, w1, 1.0, "logistic") - F0
        assert r["dF"] == pytest.approx(dF_def, rel=1e-9, abs=1e-9 * max(1.0, abs(F0)))
        assert dF_def <= 1e-9 * max(1.0, abs(F0))
        accepted += 1
    assert accepted >= 4


def test_row_loss_change_against_the_definition():
    # one sample: the line search's loss change against phi(z0 + u) - phi(z0) from Eq. 2 evaluated
    # with log-sum-exp, for margins up to |z0| = 600 and steps of either sign up to 900
    X = np.array([[1.0]])
    cp, ri, vv = D.dense_to_csc(X)
    for ysign in (1, -1):
        o = oracle.Oracle(cp, ri, vv, np.array([ysign], dtype=np.int8), 1.0, "logistic")
        for z0 in (-600.0, -60.0, -1.0, 0.0, 3.0, 60.0, 600.0):
            for u in (-900.0, -50.0, -1.0, -1e-6, 1e-6, 1.0, 50.0, 900.0):
                ref = float(np.logaddexp(0, -ysign * (z0 + u)) - np.logaddexp(0, -ysign * z0))
                got = o.row_loss_change(np.exp(z0), ysign, u)
                assert got == pytest.approx(ref, rel=1e-11, abs=1e-12 * max(1.0, abs(z0))), (ysign, z0, u, got, ref)


@pytest.mark.parametrize("loss,theta", [("logistic", 0.25), ("l2svm", 2.0)])
def test_delta_bound_descent_and_step_lower_bound(loss, theta):
    # Lemma 1(c), Eq. 14-15: Delta <= (gamma - 1) d^T H d <= 0 and F(w + a d) - F(w) <= sigma a Delta <= 0.
    # Theorem 1 (Appendix A): the accepted step is bounded below; with backtracking by beta the bound
    # reads a >= min(1, beta 2 h_min (1 - sigma + sigma gamma) / (theta c sqrt(P) lambda_bar(B))).
    rng = np.random.default_rng(21)
    base = rng.normal(0, 1, (120, 10))
    X = np.repeat(base, 4, axis=1) * rng.uniform(0.5, 1.5, 40)  # strongly correlated feature groups
    X = X.astype(np.float32).astype(np.float64)
    y = np.where(base[:, 0] + 0.3 * rng.normal(size=120) >= 0, 1, -1).astype(np.int8)
    cp, ri, vv = D.dense_to_csc(X)
    c = 1.0
    ar = oracle.Armijo()
    o = oracle.Oracle(cp, ri, vv, y, c, loss)
    w = np.zeros(40)
    mq = o.maintained(w)
    diag = (X * X).sum(0)
    seen_backtrack = False
    for epoch in range(6):
        perm = oracle.permutation(5, epoch, 40)
        for P in (40, 13):
            for t in range(0, 40, P):
                B = perm[t:t + P]
                F0 = D.F(X, y.astype(float), w, c, loss)
                w1, mq1, r = o.bundle_step(w, mq, B, armijo=ar)
                d, h = r["d"], r["h"]
                dHd = float((h * d * d).sum())
                assert r["Delta"] <= (ar.gamma - 1) * dHd + 1e-12 * max(1, abs(dHd))
                assert r["Delta"] <= 1e-15
                if r["status"] == 0:
                    assert r["dF"] <= ar.sigma * r["alpha"] * r["Delta"] + 1e-12
                    assert D.F(X, y.astype(float), w1, c, loss) <= F0 + 1e-10
                    bound = min(1.0, ar.beta * 2 * h.min() * (1 - ar.sigma + ar.sigma * ar.gamma)
                                / (theta * c * math.sqrt(len(B)) * diag[B].max()))
                    assert r["alpha"] >= bound * (1 - 1e-12)
                    seen_backtrack |= r["q"] > 0
                w, mq = w1, mq1
    assert seen_backtrack


# ---------------------------------------------------------------- special cases of Algorithm 3

@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_p1_is_cdn(loss):
    # Algorithm 3 with P = 1 is Algorithm 1 (CDN) visiting the features in the same order.
    p, X, y = tiny(loss, n=200, m=60, seed=2, density=0.2)
    o = oracle.Oracle.from_problem(p, 1.0, loss)
    w0 = np.zeros(p.n_features)
    w_pcdn, st = o.solve(1, eps=1e-12, seed=17, max_epochs=5, bundle_limit=p.n_features)
    w_cdn, _ = o.cdn_epoch(w0, o.maintained(w0), seed=17, epoch=0)
    assert st["bundles"] == p.n_features
    np.testing.assert_array_equal(w_pcdn, w_cdn)


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_p_equals_m_is_diagonal_proximal_newton(loss):
    # P = m: one bundle holds every feature, so one step is the diagonal-Hessian proximal Newton step
    # (Eq. 9) with the Armijo rule (Eq. 6).  Checked here with finite-difference derivatives, a
    # brute-force 1-D argmin per feature and direct objective differences.
    p, X, y = tiny(loss, n=40, m=10, seed=3, density=0.5)
    c = 0.8
    o = oracle.Oracle.from_problem(p, c, loss)
    rng = np.random.default_rng(4)
    ar = oracle.Armijo()
    for _ in range(4):
        w = rand_w(p.n_features, rng, scale=0.5)
        mq = o.maintained(w)
        B = np.arange(p.n_features)
        w1, _, r = o.bundle_step(w, mq, B, armijo=ar)
        g = np.array([D.fd_grad(X, y, w, c, loss, j) for j in B])
        h = np.array([o.grad_hess(mq, j)[1] for j in B])  # h pinned separately above
        d = np.array([D.ternary_min(lambda t, j=j: g[j] * t + 0.5 * h[j] * t * t + abs(w[j] + t), -50, 50) for j in B])
        np.testing.assert_allclose(r["d"], d, rtol=1e-5, atol=1e-7)
        Delta = float(g @ d + np.abs(w + d).sum() - np.abs(w).sum())
        assert r["Delta"] == pytest.approx(Delta, rel=1e-5, abs=1e-7)
        F0 = D.F(X, y, w, c, loss)
        a = 1.0
        for q in range(ar.q_max):
            if D.F(X, y, w + a * d, c, loss) - F0 <= ar.sigma * a * Delta:
                break
            a *= ar.beta
        assert r["alpha"] == a


@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_objective_monotone_over_a_solve(loss):
    # Lemma 1(c): F(w^t) is non-increasing along Algorithm 3.
    wl = datagen.scaled("lr_2k_10k", 0.1, seed=3)
    p = datagen.generate(wl.spec)
    o = oracle.Oracle.from_problem(p, 1.0, loss)
    w, st = o.solve(8, eps=1e-6, seed=1, max_epochs=30, trace=True)
    assert np.all(st["dF"] <= 1e-12)
    assert np.all(np.diff(st["epoch_F"]) <= 1e-10 * abs(st["epoch_F"][0]))
    # the backtracking cap may only trigger where the predicted decrease is at rounding level
    capped = st["q"] >= oracle.Armijo().q_max
    assert np.all(np.abs(st["Delta"][capped]) <= 1e-10 * abs(st["epoch_F"][0]))


# ---------------------------------------------------------------- optimality (KKT, FISTA)

@pytest.mark.parametrize("loss", ["logistic", "l2svm"])
def test_kkt_is_min_norm_subgradient(loss):
    p, X, y = tiny(loss, seed=5)
    c = 1.1
    o = oracle.Oracle.from_problem(p, c, loss)
    rng = np.random.default_rng(15)
    for _ in range(5):
        w = rand_w(p.n_features, rng)
        g = np.array([D.fd_grad(X, y, w, c, loss, j) for j in range(p.n_features)])
        v = D.min_norm_subgradient(g, w)
        assert o.kkt_l1(w) == pytest.approx(np.abs(v).sum(), rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("loss,c,P", [("logistic", 1.0, 3), ("logistic", 5.0, 12), ("l2svm", 0.5, 4), ("l2svm", 3.0, 1)])
def test_converged_objective_matches_fista(loss, c, P):
    p, X, y = tiny(loss, n=30, m=12, seed=21, density=0.45)
    o = oracle.Oracle.from_problem(p, c, loss)
    w, st = o.solve(P, eps=1e-10, seed=2, max_epochs=20000)
    assert st["converged"]
    wf = D.fista(X, y, c, loss)
    Ff = D.F(X, y, wf, c, loss)
    assert st["F_final"] == pytest.approx(Ff, rel=1e-9)
    assert st["F_final"] == pytest.approx(D.F(X, y, w, c, loss), rel=1e-12)
    # n > m and X of full column rank: logistic loss is strictly convex, so w* is unique
    if loss == "logistic" and np.linalg.matrix_rank(X) == p.n_features:
        np.testing.assert_allclose(w, wf, atol=1e-5)
    g = np.array([D.fd_grad(X, y, w, c, loss, j) for j in range(p.n_features)])
    assert np.abs(D.min_norm_subgradient(g, w)).sum() <= 1e-6


def test_objective_is_the_definition():
    # sanity of the shared objective (not a pin: Eq. 1-3 written twice)
    p, X, y = tiny("logistic")
    rng = np.random.default_rng(0)
    for loss in ("logistic", "l2svm"):
        o = oracle.Oracle.from_problem(p, 0.3, loss)
        for _ in range(5):
            w = rand_w(p.n_features, rng, scale=2)
            assert o.objective(w) == pytest.approx(D.F(X, y, w, 0.3, loss), rel=1e-12)


@pytest.mark.parametrize("loss,P", [("logistic", 4), ("l2svm", 3)])
def test_warm_started_path_reaches_each_optimum(loss, P):
    """A regularisation path (reading 14): each C solved from the previous C's solution, with the
    relative KKT measured against the start point.  Every step ends at that C's optimum (FISTA,
    Beck and Teboulle), and a warm start at the optimum itself needs no outer iteration."""
    p, X, y = tiny(loss, n=30, m=12, seed=23, density=0.45)
    w = None
    for c in (0.05, 0.3, 1.5, 6.0):
        o = oracle.Oracle.from_problem(p, c, loss)
        w, st = o.solve(P, eps=1e-9, seed=4, max_epochs=20000, w0=w)
        assert st["converged"]
        Ff = D.F(X, y, D.fista(X, y, c, loss), c, loss)
        assert st["F_final"] == pytest.approx(Ff, rel=1e-8)
        g = np.array([D.fd_grad(X, y, w, c, loss, j) for j in range(p.n_features)])
        assert np.abs(D.min_norm_subgradient(g, w)).sum() <= 1e-5
    # w = 0 is optimal when every |g_j(0)| <= 1: the start point's KKT is 0 and the solve ends at once
    c0 = 1e-3
    o = oracle.Oracle.from_problem(p, c0, loss)
    g0 = np.array([D.fd_grad(X, y, np.zeros(p.n_features), c0, loss, j) for j in range(p.n_features)])
    assert np.abs(g0).max() <= 1.0
    w0, st = o.solve(P, eps=1e-3, seed=4, w0=np.zeros(p.n_features))
    assert st["converged"] and st["epochs"] == 0 and st["kkt0"] == 0.0 and not np.any(w0)


@pytest.mark.parametrize("loss,P", [("logistic", 16), ("l2svm", 64)])
def test_openmp_baseline_solves_the_same_problem(loss, P):
    """The OpenMP CPU baseline (the paper's shared-memory parallel scheme) runs Algorithm 3 with the
    oracle's partitions and stop rule: same number of outer iterations and bundles, objective equal
    to rounding (its sums are atomic and parallel)."""
    spec = datagen.Spec(1500, 4000, "zipf", row_mean=40.0, zipf_s=1.1, values="tfidf", wstar_nnz=30, flip_frac=0.05,
                        seed=11)
    p = datagen.generate(spec, with_csr=False)
    o = oracle.Oracle.from_problem(p, 0.7, loss)
    w1, s1 = o.solve(P, eps=1e-3, seed=6, max_epochs=300)
    w2, s2 = o.solve_omp(P, eps=1e-3, seed=6, max_epochs=300)
    assert s1["converged"] and s2["converged"]
    assert abs(s1["epochs"] - s2["epochs"]) <= 1
    assert s2["F_final"] == pytest.approx(s1["F_final"], rel=1e-7)
    assert s2["F_final"] == pytest.approx(o.objective(w2), rel=1e-12)
    assert oracle.omp_threads() >= 1
