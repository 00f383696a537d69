"""Independent eigenvalue pins (TEST INFRASTRUCTURE: only tests/, ``__graft_entry__``
and bench.py's CPU arms may import this module).

* ``sturm_count``  number of eigenvalues of T below x, from the signs of the
  pivots of the LDL^T factorisation of T - x I (Sylvester's law of inertia).
* ``bisection_eigvals``  every eigenvalue of T by bisection on the Sturm count,
  to an absolute accuracy of a few eps ||T||.
* ``charpoly_roots``  for n <= 8: the characteristic polynomial built by the
  three-term recurrence p_k = (a_k - x) p_{k-1} - b_{k-1}^2 p_{k-2} with exact
  polynomial arithmetic on coefficients, then all real roots located by sign
  changes on a fine grid and refined by bisection on the polynomial value.
* ``closed_form_121``  lambda_k = 2 - 2 cos(k pi / (n+1)), q_k(j) = sqrt(2/(n+1))
  sin(j k pi / (n+1)) for tridiag(1, 2, 1) (textbook).
"""
from __future__ import annotations

import numpy as np

EPS = 2.0 ** -53


def tnorm(d, e) -> float:
    """||T||_1 = max_i |b_{i-1}| + |a_i| + |b_i| (equal to the infinity norm)."""
    d = np.abs(np.asarray(d, dtype=np.float64))
    e = np.abs(np.asarray(e, dtype=np.float64))
    r = d.copy()
    if e.size:
        r[:-1] += e
        r[1:] += e
    return float(r.max()) if r.size else 0.0


def sturm_count(d, e, x) -> np.ndarray:
    """Eigenvalues of tridiag(e, d, e) strictly below each entry of x (vectorised over x)."""
    d = np.asarray(d, dtype=np.float64)
    e2 = np.asarray(e, dtype=np.float64) ** 2
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    tiny = np.finfo(np.float64).tiny ** 0.5 * max(tnorm(d, np.sqrt(e2)), 1e-300)
    q = d[0] - x
    q = np.where(q == 0.0, -tiny, q)
    count = (q < 0).astype(np.int64)
    for i in range(1, d.shape[0]):
        q = (d[i] - x) - e2[i - 1] / q
        q = np.where(q == 0.0, -tiny, q)
        count += q < 0
    return count


def bisection_eigvals(d, e, idx=None) -> np.ndarray:
    """Eigenvalues number ``idx`` (0-based, ascending; all by default) by Sturm bisection."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n = d.shape[0]
    if idx is None:
        idx = np.arange(n)
    idx = np.asarray(idx, dtype=np.int64)
    nrm = tnorm(d, e)
    lo = np.full(idx.shape[0], -nrm - 1.0)
    hi = np.full(idx.shape[0], nrm + 1.0)
    for _ in range(200):
        mid = lo + (hi - lo) / 2.0
        if np.all((mid <= lo) | (mid >= hi) | (hi - lo <= 2.0 * EPS * nrm)):
            break
        c = sturm_count(d, e, mid)
        below = c <= idx                    # fewer than idx+1 eigenvalues below mid
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return lo + (hi - lo) / 2.0


def charpoly_coeffs(d, e) -> np.ndarray:
    """Coefficients (highest degree first) of det(T - x I) from the three-term recurrence."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    p_prev = np.array([1.0])
    p = np.array([-1.0, d[0]])
    for k in range(1, d.shape[0]):
        nxt = np.polymul(np.array([-1.0, d[k]]), p)
        nxt = np.polysub(nxt, e[k - 1] ** 2 * p_prev)
        p_prev, p = p, nxt
    return p


def charpoly_roots(d, e, grid: int = 200001) -> np.ndarray:
    """All eigenvalues of a small (n <= 8) tridiagonal as roots of its characteristic polynomial."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n = d.shape[0]
    assert n <= 8
    c = charpoly_coeffs(d, e)
    nrm = tnorm(d, e) + 1.0
    xs = np.linspace(-nrm, nrm, grid)
    vals = np.polyval(c, xs)
    roots = []
    for i in range(grid - 1):
        a, b = vals[i], vals[i + 1]
        if a == 0.0:
            roots.append(xs[i])
            continue
        if a * b < 0:
            lo, hi = xs[i], xs[i + 1]
            flo = a
            for _ in range(200):
                mid = lo + (hi - lo) / 2.0
                if mid <= lo or mid >= hi:
                    break
                fm = np.polyval(c, mid)
                if (fm < 0) == (flo < 0):
                    lo, flo = mid, fm
                else:
                    hi = mid
            roots.append(lo + (hi - lo) / 2.0)
    return np.array(sorted(roots))


def closed_form_121(n: int):
    """Eigenpairs of tridiag(1, 2, 1) of order n, ascending, columns sign-normalised."""
    k = np.arange(1, n + 1, dtype=np.float64)
    lam = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    j = np.arange(1, n + 1, dtype=np.float64)
    # eigenvalue 2 - 2cos(k pi/(n+1)) has vector sin(j k pi/(n+1)) (up to the sign pattern
    # (-1)^j, which tridiag(1,2,1) absorbs: its vector for 2 + 2cos is the k-th sine)
    q = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, k) * np.pi / (n + 1))
    q = q * ((-1.0) ** (j - 1))[:, None]
    return lam, q


def clement_eigvals(n: int) -> np.ndarray:
    """Clement matrix of order n (off-diagonal sqrt(i (n - i))): -(n-1), -(n-3), ..., n-1."""
    return np.arange(-(n - 1), n, 2, dtype=np.float64)
