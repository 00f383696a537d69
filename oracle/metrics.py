"""Accuracy measures (TEST INFRASTRUCTURE: only tests/, ``__graft_entry__`` and bench.py's
CPU arms may import this module).

* orthogonality ||I - Q^T Q||_max (the measure of Table 4)
* scaled residual ||T Q - Q Lambda||_F / (n eps ||T||), with eps = DBL_EPSILON
* per-column eigenvector agreement for well-separated eigenvalues
"""
from __future__ import annotations

import numpy as np

DBL_EPSILON = 2.0 ** -52


def tnorm(d, e) -> float:
    d = np.abs(np.asarray(d, dtype=np.float64))
    e = np.abs(np.asarray(e, dtype=np.float64))
    r = d.copy()
    if e.size:
        r[:-1] += e
        r[1:] += e
    return float(r.max()) if r.size else 0.0


def tri_matmul(d, e, q):
    """T @ Q for T = tridiag(e, d, e) without forming T."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    out = d[:, None] * q
    if e.size:
        out[:-1] += e[:, None] * q[1:]
        out[1:] += e[:, None] * q[:-1]
    return out


def orthogonality(q) -> float:
    q = np.asarray(q, dtype=np.float64)
    g = q.T @ q
    g[np.diag_indices_from(g)] -= 1.0
    return float(np.max(np.abs(g))) if g.size else 0.0


def scaled_residual(d, e, lam, q) -> float:
    n = len(d)
    r = tri_matmul(d, e, q) - q * np.asarray(lam)[None, :]
    nrm = tnorm(d, e)
    if n == 0 or nrm == 0.0:
        return 0.0
    return float(np.linalg.norm(r) / (n * DBL_EPSILON * nrm))


def column_agreement(lam_ref, q_ref, q, tnrm, min_relgap=1e-6):
    """max over well-separated columns of || q_i - sign * q_ref_i ||_2, and the mask used."""
    lam_ref = np.asarray(lam_ref)
    n = lam_ref.shape[0]
    gap = np.full(n, np.inf)
    if n > 1:
        dl = np.diff(lam_ref)
        gap[:-1] = np.minimum(gap[:-1], dl)
        gap[1:] = np.minimum(gap[1:], dl)
    mask = gap >= min_relgap * max(tnrm, 1e-300)
    if not mask.any():
        return 0.0, mask
    a = q_ref[:, mask]
    b = q[:, mask]
    sgn = np.sign(np.sum(a * b, axis=0))
    sgn[sgn == 0] = 1.0
    err = np.linalg.norm(b - a * sgn[None, :], axis=0)
    return float(err.max()), mask
