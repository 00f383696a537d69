"""Extended-precision eigenvectors of the rank-one problem (TEST INFRASTRUCTURE: only
tests/, ``__graft_entry__`` and bench.py's CPU arms may import this module).

Section 1 names two ways to keep the eigenvectors (D - lambda_i)^{-1} z of
D + rho z z^T orthogonal: the Loewner-theorem recomputation of z (Remark 1, the
``dc.lowner_z`` path), and Sorensen and Tang's extended precision, where each
eigenvalue is computed to more than working precision so that every difference
d_j - lambda_i, and with it every component, is accurate for the given (d, z).

This module states the second approach with exact arithmetic: the roots of the
secular equation f(tau) = 1 + rho sum_j z_j^2 / ((d_j - d_origin) - tau) are bracketed
and bisected on exact rationals (Python's ``fractions``: every d_j, z_j is a double,
so every sum is exact) until the bracket is narrower than 2^-110 |tau|, far below
the 2^-106 of a double-double; the eigenvector components z_j / (d_j - lambda_i) are
formed from the exact differences and rounded once.  Pure-Python loops: small K only.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

REL_BITS = 110


def _f(shift, z2, rho, tau):
    """f(tau) exactly: shift[j] = d_j - d_origin and z2[j] = z_j^2 as Fractions."""
    s = Fraction(0)
    for sj, zj in zip(shift, z2):
        s += zj / (sj - tau)
    return 1 + rho * s


def exact_roots(dbar, zbar, rho, origin, tau_hint=None):
    """Roots as (tau_hi, tau_lo): tau_hi + tau_lo is within 2^-110 |tau| of the exact
    root tau of the interval given by ``origin`` (the oracle's own choice of the nearer
    pole, as in ``dc.secular_roots``).  Root i lies in (d_i, d_{i+1}) (the last one in
    (d_K, d_K + rho ||z||^2)); with origin o the bracket in tau is (d_i - d_o, d_{i+1} - d_o).
    tau_hint (optional doubles) narrows the first bracket to a few units around it
    when f changes sign there, and is otherwise ignored."""
    kk = len(dbar)
    d = [Fraction(float(x)) for x in dbar]
    z2 = [Fraction(float(x)) ** 2 for x in zbar]
    r = Fraction(float(rho))
    hi_out = np.empty(kk)
    lo_out = np.empty(kk)
    exact = []
    for i in range(kk):
        o = int(origin[i])
        shift = [dj - d[o] for dj in d]
        lo = shift[i]
        hi = shift[i + 1] if i + 1 < kk else r * sum(z2)
        if tau_hint is not None:
            t = Fraction(float(tau_hint[i]))
            u = Fraction(abs(float(np.spacing(abs(float(tau_hint[i])) + 0.0)))) * 8
            a, b = max(lo, t - u), min(hi, t + u)
            if a < b and a != lo and b != hi and _f(shift, z2, r, a) < 0 < _f(shift, z2, r, b):
                lo, hi = a, b
        # f increases from -inf to +inf on the interval
        while True:
            mid = (lo + hi) / 2
            if hi - lo <= abs(mid) * Fraction(1, 2 ** REL_BITS):
                break
            if _f(shift, z2, r, mid) < 0:
                lo = mid
            else:
                hi = mid
        tau = (lo + hi) / 2
        exact.append(tau)
        th = float(tau)
        hi_out[i] = th
        lo_out[i] = float(tau - Fraction(th))
    return hi_out, lo_out, exact


def extended_vectors(dbar, zbar, origin, exact_tau):
    """Normalised eigenvectors of D + rho z z^T with the original z: column i has the
    components z_j / (d_j - lambda_i), each difference (d_j - d_origin) - tau taken
    exactly and the quotient rounded once; then the column is normalised in FP64."""
    kk = len(dbar)
    d = [Fraction(float(x)) for x in dbar]
    u = np.empty((kk, kk))
    for i in range(kk):
        o = int(origin[i])
        for j in range(kk):
            u[j, i] = float(Fraction(float(zbar[j])) / ((d[j] - d[o]) - exact_tau[i]))
    return u / np.sqrt(np.sum(u * u, axis=0))[None, :]


def merge_extended(D, Q, n1, beta):
    """The merge of ``dc.merge`` with the eigenvectors of the non-deflated part taken
    by extended precision instead of the Loewner z: same deflation, same eigenvalues
    (the FP64 roots), Qhat = ``extended_vectors`` of the exact roots, then Q_sel Qhat
    placed at the columns ``dc.merge`` gives them.  Returns (lambda, U, info) with
    info["tau_hi"], info["tau_lo"] (the exact roots split into two doubles) and
    info["qhat_ext"]."""
    from . import dc
    lam, u, info = dc.merge(D, Q, n1, beta)
    kk = info["K"]
    if kk == 0:
        return lam, u, dict(info, tau_hi=np.zeros(0), tau_lo=np.zeros(0), qhat_ext=np.zeros((0, 0)))
    hi, lo, ex = exact_roots(info["dbar"], info["zbar"], info["rho"], info["origin"], info["tau"])
    qhat = extended_vectors(info["dbar"], info["zbar"], info["origin"], ex)
    n = len(D)
    cols = np.asarray(Q, dtype=np.float64)[:, info["order"]].copy()
    for (j, k, c, s) in info["rotations"]:
        cj, ck = cols[:, j].copy(), cols[:, k].copy()
        cols[:, j] = c * cj + s * ck
        cols[:, k] = -s * cj + c * ck
    u_nd = cols[:, info["kept"]] @ qhat
    pos = np.empty(n, dtype=np.int64)
    pos[info["final_order"]] = np.arange(n)
    out = u.copy()
    out[:, pos[:kk]] = u_nd
    return lam, out, dict(info, tau_hi=hi, tau_lo=lo, qhat_ext=qhat)
