"""Dense reference gradient of (lambda, Q) with respect to (d, e) (TEST INFRASTRUCTURE:
only tests/, ``__graft_entry__`` and bench.py's CPU arms may import this module).

For T = Q Lambda Q^T with distinct eigenvalues, first-order perturbation theory
gives d lambda_i = q_i^T dT q_i and d q_i = sum_{j != i} q_j (q_j^T dT q_i) /
(lambda_i - lambda_j).  Hence the adjoint of T is

    Tbar = Q (diag(lambda_bar) + F o (Q^T Qbar)) Q^T,  F_ji = 1/(lambda_i - lambda_j), F_ii = 0,

and, since d_i enters T once and e_i twice, dbar_i = Tbar_ii and
ebar_i = Tbar_{i,i+1} + Tbar_{i+1,i}.  This module forms Tbar densely in FP64.
"""
from __future__ import annotations

import numpy as np


def tbar_dense(lam, q, g_lam=None, g_q=None) -> np.ndarray:
    lam = np.asarray(lam, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = lam.shape[0]
    c = np.zeros((n, n))
    if g_q is not None:
        diff = lam[None, :] - lam[:, None]             # [j, i] = lambda_i - lambda_j
        with np.errstate(divide="ignore"):
            f = np.where(np.eye(n, dtype=bool), 0.0, 1.0 / np.where(diff == 0.0, np.inf, diff))
        c += f * (q.T @ np.asarray(g_q, dtype=np.float64))
    if g_lam is not None:
        c[np.diag_indices(n)] += np.asarray(g_lam, dtype=np.float64)
    return q @ c @ q.T


def band_gradient(lam, q, g_lam=None, g_q=None):
    """(dbar, ebar) from the dense Tbar."""
    tb = tbar_dense(lam, q, g_lam, g_q)
    n = tb.shape[0]
    gd = np.diag(tb).copy()
    ge = np.array([tb[i, i + 1] + tb[i + 1, i] for i in range(n - 1)])
    return gd, ge


def config_loss(lam, q, w, G) -> float:
    """sum_i w_i lambda_i + ||Q[:, :m]^T G||_F^2 with m = G.shape[1]."""
    m = G.shape[1]
    return float(np.dot(w, lam) + np.sum((q[:, :m].T @ G) ** 2))


def config_loss_grads(lam, q, w, G):
    """(lambda_bar, Q_bar) of ``config_loss``: Q_bar[:, :m] = 2 G (G^T Q[:, :m])."""
    m = G.shape[1]
    gq = np.zeros_like(q)
    gq[:, :m] = 2.0 * G @ (G.T @ q[:, :m])
    return np.asarray(w, dtype=np.float64).copy(), gq
