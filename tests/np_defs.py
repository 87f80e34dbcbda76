"""Independent numpy statements of the problem's definitions, used to pin the oracle.

Nothing here restates the oracle's algorithm: the objective is Eq. 1 with the
losses of Eq. 2 / Eq. 3 written on a dense matrix, derivatives come from finite
differences of that objective, 1-D minimisers from ternary search, and the
reference optimum from FISTA (Beck and Teboulle 2009), a different algorithm.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64_outputs(seed: int, count: int) -> list[int]:
    """First ``count`` outputs of splitmix64 started at ``seed`` (Steele, Lea, Flood 2014)."""
    out = []
    s = seed & MASK64
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        out.append(z ^ (z >> 31))
    return out


def loss_vector(X: np.ndarray, y: np.ndarray, w: np.ndarray, loss: str) -> np.ndarray:
    """phi(w; x_i, y_i) for every sample (Eq. 2 logistic, Eq. 3 squared hinge)."""
    yz = y.astype(np.float64) * (X @ w)
    if loss == "logistic":
        return np.logaddexp(0.0, -yz)
    return np.maximum(0.0, 1.0 - yz) ** 2


def L(X, y, w, c, loss) -> float:
    return float(c * loss_vector(X, y, w, loss).sum())


def F(X, y, w, c, loss) -> float:
    """Eq. 1: c * sum_i phi + ||w||_1."""
    return L(X, y, w, c, loss) + float(np.abs(w).sum())


def F_pen(X, y, w, c, loss, l1=1.0, l2=0.0) -> float:
    """c * sum_i phi + l1 ||w||_1 + (l2/2) ||w||_2^2 (a separable penalty: L1, L2 or both)."""
    return L(X, y, w, c, loss) + l1 * float(np.abs(w).sum()) + 0.5 * l2 * float(w @ w)


def fd_grad_smooth(X, y, w, c, loss, j, l2, eps=1e-5) -> float:
    """Central difference of the smooth part c L(w) + (l2/2) ||w||^2 along e_j."""
    e = np.zeros_like(w)
    e[j] = eps

    def S(v):
        return L(X, y, v, c, loss) + 0.5 * l2 * float(v @ v)

    return (S(w + e) - S(w - e)) / (2 * eps)


def fd_grad(X, y, w, c, loss, j, eps=1e-5) -> float:
    e = np.zeros_like(w)
    e[j] = eps
    return (L(X, y, w + e, c, loss) - L(X, y, w - e, c, loss)) / (2 * eps)


def fd_hess(X, y, w, c, loss, j, eps=1e-4) -> float:
    e = np.zeros_like(w)
    e[j] = eps
    return (L(X, y, w + e, c, loss) - 2 * L(X, y, w, c, loss) + L(X, y, w - e, c, loss)) / (eps * eps)


def ternary_min(f, lo, hi, iters=300) -> float:
    """Minimiser of a convex 1-D function on [lo, hi] by ternary search."""
    for _ in range(iters):
        a = lo + (hi - lo) / 3
        b = hi - (hi - lo) / 3
        if f(a) <= f(b):
            hi = b
        else:
            lo = a
    return 0.5 * (lo + hi)


def grad(X, y, w, c, loss) -> np.ndarray:
    """Gradient of c sum_i phi(w; x_i, y_i) (Eq. 2 / Eq. 3 differentiated in matrix form); X dense
    or scipy-sparse."""
    yf = np.asarray(y, dtype=np.float64)
    z = X @ w
    if loss == "logistic":
        s = -yf / (1.0 + np.exp(yf * z))
    else:
        s = -2.0 * yf * np.maximum(0.0, 1.0 - yf * z)
    return c * np.asarray(X.T @ s).ravel()


def fista(X, y, c, loss, iters=200000, tol=1e-13, l1=1.0, l2=0.0):
    """FISTA with constant step 1/Lip for min L(w) + l1 ||w||_1 + (l2/2) ||w||^2 (Beck and Teboulle
    2009; the L2 term in the smooth part), with the gradient-based adaptive restart of O'Donoghue
    and Candes (2015)."""
    n, m = X.shape
    theta = 0.25 if loss == "logistic" else 2.0
    lip = theta * c * np.linalg.norm(X, 2) ** 2 + l2
    step = 1.0 / lip

    def grad_w(w):
        return grad(X, y, w, c, loss) + l2 * w

    w = np.zeros(m)
    v = w.copy()
    t = 1.0
    for it in range(iters):
        u = v - step * grad_w(v)
        w_new = np.sign(u) * np.maximum(np.abs(u) - step * l1, 0.0)
        if float(np.dot(v - w_new, w_new - w)) > 0:
            t = 1.0
        t_new = 0.5 * (1 + math.sqrt(1 + 4 * t * t))
        v = w_new + ((t - 1) / t_new) * (w_new - w)
        if np.max(np.abs(w_new - w)) < tol:
            w = w_new
            break
        w, t = w_new, t_new
    return w


def min_norm_subgradient(g: np.ndarray, w: np.ndarray, l1: float = 1.0) -> np.ndarray:
    """g_j + s with s minimising |g_j + s| over the subdifferential of l1 |w_j| ({l1 sign w_j}, or
    [-l1, l1] at w_j = 0), the latter by ternary search."""
    out = np.empty_like(g)
    for j in range(g.shape[0]):
        if w[j] > 0:
            out[j] = g[j] + l1
        elif w[j] < 0:
            out[j] = g[j] - l1
        else:
            s = ternary_min(lambda t, gj=g[j]: abs(gj + t), -l1, l1, iters=200) if l1 > 0 else 0.0
            out[j] = g[j] + s
    return out


def dense_to_csc(X: np.ndarray):
    """CSC arrays of a dense matrix (explicit zeros dropped), rows ascending in each column."""
    n, m = X.shape
    col_ptr = [0]
    rows, vals = [], []
    for j in range(m):
        nz = np.nonzero(X[:, j])[0]
        rows.extend(nz.tolist())
        vals.extend(X[nz, j].tolist())
        col_ptr.append(len(rows))
    return (np.array(col_ptr, dtype=np.int64), np.array(rows, dtype=np.int32), np.array(vals, dtype=np.float32))


def expected_lambda_bar(lams: np.ndarray, P: int) -> float:
    """Appendix A, proof of Lemma 1(a): E[max of P of the values] for a uniform P-subset,
    sum_{k=P}^{m} lambda_(k) C(k-1, P-1) / C(m, P) with lambda_(k) the k-th smallest."""
    lam = np.sort(np.asarray(lams, dtype=np.float64))
    m = lam.shape[0]
    denom = math.comb(m, P)
    tot = 0.0
    for k in range(P, m + 1):
        tot += float(lam[k - 1]) * (math.comb(k - 1, P - 1) / denom)
    return tot
