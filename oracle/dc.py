"""Plain FP64 Cuppen divide-and-conquer (TEST INFRASTRUCTURE: only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU arms may import this module).

Each function restates one step of the method, in the paper's order and notation:

* tearing  T = diag(T1, T2) + b_k v v^T                        (Eq. 2)
* merge form T = Q (D + b_k z z^T) Q^T, z = Q^T v              (Eq. 3)
* deflation: negligible z_i, and equal d_i removed by plane
  rotations G, deflated pairs permuted to the back by P       (Eq. 5)
* secular equation f(lambda) = 1 + rho sum_j z_j^2/(d_j - lambda)  (Section 1,
  the formula printed after Eq. 4, read with the sum over j)
* eigenvectors (D - lambda_i)^{-1} z, with z recomputed from all the
  eigenvalues by the Loewner-theorem approach (Section 1, Remark 1)
* eigenvector assembly U = Q (G P) diag(Qhat, I_d)             (Eq. 6)

Readings where the paper is silent (also listed in the design notes):

* v = e_k + sign(b_k) e_{k+1} and rho = |b_k|, so both corner entries of T1 and
  T2 are reduced by |b_k| and rho >= 0.  z is normalised (||z||^2 = 2 before),
  giving rho = 2 |b_k|.
* deflation tolerance tol = 8 eps max(max|d|, max|z|), eps = 2^-53; type 1 if
  rho |z_j| <= tol; type 2 (pair j < k of kept entries, adjacent in sorted
  order) if |(d_k - d_j) c s| <= tol with t = sqrt(z_j^2 + z_k^2),
  c = z_k / t, s = -z_j / t.
* roots are stored as (origin, tau): lambda_i = d_origin + tau, so that every
  difference d_j - lambda_i is formed as (d_j - d_origin) - tau.
* the Loewner formula is Gu and Eisenstat's:  zhat_j^2 = prod_i (lambda_i - d_j)
  / (rho prod_{i != j} (d_i - d_j)), taken as a product of ratios that are each
  in (0, 1); zhat_j carries the sign of z_j.
* leaves (n <= leaf) are solved by cyclic Jacobi on the dense leaf matrix; the
  tree splits a node of size n at n1 = floor(n / 2).
* the output is sorted ascending (stable); ``syev`` additionally makes the
  largest-magnitude entry of every eigenvector positive.
"""
from __future__ import annotations

import numpy as np

EPS = 2.0 ** -53            # unit roundoff (LAPACK's dlamch('E'))
INV_SQRT2 = 0.7071067811865476


# ----------------------------------------------------------------------------
# Leaves: cyclic Jacobi on a small dense symmetric matrix (textbook; the paper
# assumes T1 and T2 are already decomposed and does not name a leaf solver).
# ----------------------------------------------------------------------------
def _round_robin(n: int):
    """Disjoint pairings covering every (p, q), p < q, once per sweep (n even)."""
    players = list(range(n))
    rounds = []
    for _ in range(n - 1):
        rounds.append([(min(players[i], players[n - 1 - i]), max(players[i], players[n - 1 - i]))
                       for i in range(n // 2)])
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_eigh(a: np.ndarray, max_sweeps: int = 60):
    """Eigenvalues (ascending) and orthonormal eigenvectors of a symmetric matrix
    by cyclic Jacobi rotations applied in round-robin order."""
    a = np.array(a, dtype=np.float64, copy=True)
    n = a.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros((0, 0))
    m = n + (n % 2)
    if m != n:                                  # pad to even size with a decoupled entry
        b = np.zeros((m, m))
        b[:n, :n] = a
        a = b
    v = np.eye(m)
    rounds = _round_robin(m)
    fro = np.linalg.norm(a)
    last = np.inf
    for _ in range(max_sweeps):
        off = np.linalg.norm(a - np.diag(np.diag(a)))
        if off <= 1e-2 * EPS * fro or off >= last:
            break
        last = off
        for pairs in rounds:
            p = np.array([x for x, _ in pairs])
            q = np.array([y for _, y in pairs])
            apq = a[p, q]
            act = apq != 0.0
            if not act.any():
                continue
            p, q, apq = p[act], q[act], apq[act]
            theta = (a[q, q] - a[p, p]) / (2.0 * apq)
            t = np.where(theta >= 0, 1.0, -1.0) / (np.abs(theta) + np.sqrt(theta * theta + 1.0))
            c = 1.0 / np.sqrt(t * t + 1.0)
            s = t * c
            j = np.eye(m)
            j[p, p] = c
            j[q, q] = c
            j[p, q] = s
            j[q, p] = -s
            a = j.T @ a @ j
            v = v @ j
    w = np.diag(a)[:n].copy()
    v = v[:n, :n].copy()
    order = np.argsort(w, kind="stable")
    return w[order], v[:, order]


def tridiag_dense(d: np.ndarray, e: np.ndarray) -> np.ndarray:
    """T of Eq. (1) as a dense matrix."""
    t = np.diag(np.asarray(d, dtype=np.float64))
    if len(e):
        t += np.diag(e, 1) + np.diag(e, -1)
    return t


# ----------------------------------------------------------------------------
# Secular equation (Section 1): roots of 1 + rho sum z_j^2 / (d_j - lambda) = 0.
# ----------------------------------------------------------------------------
def secular_f(dbar, zbar, rho, origin, tau):
    """f at lambda = d_origin + tau, differences formed as (d_j - d_origin) - tau."""
    delta = (dbar - dbar[origin]) - tau
    return 1.0 + rho * np.sum(zbar * zbar / delta)


def secular_roots(dbar: np.ndarray, zbar: np.ndarray, rho: float, chunk: int = 512):
    """All K roots by bisection on tau in the shifted variable.

    Root i (0-based) lies in (d_i, d_{i+1}) for i < K-1 and in
    (d_{K-1}, d_{K-1} + rho ||z||^2] for the last one.  The origin is d_i if
    f at the midpoint of the interval is positive (the root is in the left half),
    else d_{i+1}.  Bisection runs until the bracket can no longer be split.
    Returns (origin int array, tau float array)."""
    dbar = np.asarray(dbar, dtype=np.float64)
    zbar = np.asarray(zbar, dtype=np.float64)
    kk = dbar.shape[0]
    z2 = zbar * zbar
    origin = np.empty(kk, dtype=np.int64)
    lo = np.empty(kk)
    hi = np.empty(kk)
    for c0 in range(0, kk, chunk):
        idx = np.arange(c0, min(kk, c0 + chunk))
        last = idx == kk - 1
        inner = idx[~last]
        if inner.size:
            gap = dbar[inner + 1] - dbar[inner]
            half = gap / 2.0
            delta = (dbar[None, :] - dbar[inner][:, None]) - half[:, None]
            fmid = 1.0 + rho * np.sum(z2[None, :] / delta, axis=1)
            left = fmid > 0.0
            origin[inner] = np.where(left, inner, inner + 1)
            lo[inner] = np.where(left, 0.0, -half)
            hi[inner] = np.where(left, half, 0.0)
        if last.any():
            origin[kk - 1] = kk - 1
            lo[kk - 1] = 0.0
            hi[kk - 1] = rho * np.sum(z2)
    tau = np.empty(kk)
    for c0 in range(0, kk, chunk):
        sl = slice(c0, min(kk, c0 + chunk))
        o = origin[sl]
        base = dbar[None, :] - dbar[o][:, None]          # d_j - d_origin
        l, h = lo[sl].copy(), hi[sl].copy()
        done = np.zeros(l.shape[0], dtype=bool)
        mid = l + (h - l) / 2.0
        for _ in range(2200):
            mid = np.where(done, mid, l + (h - l) / 2.0)
            done |= (mid <= l) | (mid >= h)
            if done.all():
                break
            f = 1.0 + rho * np.sum(z2[None, :] / (base - mid[:, None]), axis=1)
            neg = f < 0.0
            l = np.where(~done & neg, mid, l)
            h = np.where(~done & ~neg, mid, h)
        tau[sl] = mid
    return origin, tau


def lambda_from(dbar, origin, tau):
    return dbar[origin] + tau


# ----------------------------------------------------------------------------
# Loewner-theorem recomputation of z (Remark 1; Gu-Eisenstat).
# ----------------------------------------------------------------------------
def lowner_z(dbar, zbar, rho, origin, tau):
    """zhat with D + rho zhat zhat^T having exactly the eigenvalues d_origin + tau.

    zhat_j^2 = (lambda_{K-1} - d_j)/rho * prod_{i<j} (lambda_i - d_j)/(d_i - d_j)
                                        * prod_{j<=i<K-1} (lambda_i - d_j)/(d_{i+1} - d_j)
    with lambda_i - d_j = (d_origin(i) - d_j) + tau_i."""
    kk = dbar.shape[0]
    lam_m_d = (dbar[origin][:, None] - dbar[None, :]) + tau[:, None]   # [i, j] = lambda_i - d_j
    zhat2 = np.empty(kk)
    for j in range(kk):
        num_lo = lam_m_d[:j, j]
        den_lo = dbar[:j] - dbar[j]
        num_hi = lam_m_d[j:kk - 1, j]
        den_hi = dbar[j + 1:kk] - dbar[j]
        r = lam_m_d[kk - 1, j] / rho
        r *= np.prod(num_lo / den_lo)
        r *= np.prod(num_hi / den_hi)
        zhat2[j] = r
    return np.copysign(np.sqrt(zhat2), zbar)


def rank_one_vectors(dbar, zhat, origin, tau):
    """Normalised eigenvectors of D + rho zhat zhat^T: column i = (D - lambda_i)^{-1} zhat."""
    delta = (dbar[:, None] - dbar[origin][None, :]) - tau[None, :]     # [j, i] = d_j - lambda_i
    u = zhat[:, None] / delta
    return u / np.sqrt(np.sum(u * u, axis=0))[None, :]


# ----------------------------------------------------------------------------
# Deflation (Eq. 5) and the full merge (Eqs. 3-6).
# ----------------------------------------------------------------------------
def deflate(d: np.ndarray, z: np.ndarray, rho: float):
    """Deflation on sorted (d, z).  Returns a dict with the kept (non-deflated)
    indices, the deflated indices (ascending), the rotations (j, k, c, s) in the
    order applied, and the updated d, z (copies)."""
    d = np.array(d, dtype=np.float64, copy=True)
    z = np.array(z, dtype=np.float64, copy=True)
    n = d.shape[0]
    tol = 8.0 * EPS * max(float(np.max(np.abs(d))) if n else 0.0,
                          float(np.max(np.abs(z))) if n else 0.0)
    type1 = rho * np.abs(z) <= tol
    kept, deflated, rots = [], [], []
    prev = -1
    for k in range(n):
        if type1[k]:
            deflated.append(k)
            continue
        if prev < 0:
            prev = k
            continue
        j = prev
        zj, zk = float(z[j]), float(z[k])
        t = float(np.sqrt(zj * zj + zk * zk))
        c = zk / t
        s = -zj / t
        dj, dk = float(d[j]), float(d[k])
        if abs(((dk - dj) * c) * s) <= tol:
            z[k] = t
            z[j] = 0.0
            d[j] = dj * c * c + dk * s * s
            d[k] = dj * s * s + dk * c * c
            rots.append((j, k, c, s))
            deflated.append(j)
        else:
            kept.append(j)
        prev = k
    if prev >= 0:
        kept.append(prev)
    return dict(kept=np.array(kept, dtype=np.int64),
                deflated=np.array(sorted(deflated), dtype=np.int64),
                rotations=rots, d=d, z=z, tol=tol, type1=type1)


def merge_z(q: np.ndarray, n1: int, beta: float):
    """z = Q^T v / sqrt(2) with v = e_{n1} + sign(beta) e_{n1+1} (Eq. 3), rho = 2|beta|."""
    sgn = -1.0 if beta < 0 else 1.0
    z = np.concatenate([q[n1 - 1, :n1], sgn * q[n1, n1:]]) * INV_SQRT2
    return z, 2.0 * abs(beta)


def merge(D: np.ndarray, Q: np.ndarray, n1: int, beta: float):
    """One rank-one merge.  D holds the eigenvalues of T1 (first n1, ascending) and
    of T2 (ascending); Q = diag(Q1, Q2).  Returns (lambda ascending, U, info) where
    U = Q (G P) diag(Qhat, I_d) reordered to ascending lambda (Eq. 6)."""
    D = np.asarray(D, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    n = D.shape[0]
    z, rho = merge_z(Q, n1, beta)
    order = np.argsort(D, kind="stable")                 # merge of the two sorted halves
    ds, zs = D[order], z[order]
    cols = Q[:, order].copy()
    half = np.where(order < n1, 1, 2)                      # 1: rows of T1 only, 2: rows of T2 only
    df = deflate(ds, zs, rho)
    for (j, k, c, s) in df["rotations"]:                   # G: plane rotations on columns j, k
        cj, ck = cols[:, j].copy(), cols[:, k].copy()
        cols[:, j] = c * cj + s * ck
        cols[:, k] = -s * cj + c * ck
        half[j] = half[k] = half[j] | half[k]
    kept, defl = df["kept"], df["deflated"]
    dbar, zbar = df["d"][kept], df["z"][kept]
    kk = kept.shape[0]
    if kk:
        origin, tau = secular_roots(dbar, zbar, rho)
        zhat = lowner_z(dbar, zbar, rho, origin, tau)
        qhat = rank_one_vectors(dbar, zhat, origin, tau)
        lam_nd = dbar[origin] + tau
        u_nd = cols[:, kept] @ qhat
    else:
        origin = np.zeros(0, dtype=np.int64)
        tau = np.zeros(0)
        zhat = np.zeros(0)
        qhat = np.zeros((0, 0))
        lam_nd = np.zeros(0)
        u_nd = np.zeros((n, 0))
    lam_all = np.concatenate([lam_nd, df["d"][defl]])
    vec_all = np.concatenate([u_nd, cols[:, defl]], axis=1)
    fin = np.argsort(lam_all, kind="stable")
    info = dict(K=kk, rho=rho, z=z, tol=df["tol"], order=order, kept=kept, deflated=defl,
                rotations=df["rotations"], dbar=dbar, zbar=zbar, origin=origin, tau=tau,
                zhat=zhat, qhat=qhat, lam_nd=lam_nd, half=half, final_order=fin)
    return lam_all[fin], vec_all[:, fin], info


def merge_hss(D: np.ndarray, Q: np.ndarray, n1: int, beta: float, leaf: int, rp: int, tol: float,
              seed: int, grow: int = 0):
    """The merge of ``merge`` with Qhat replaced by its HSS approximation (Section 2.2):
    Qhat, in the order of the sorted non-deflated d, is compressed by Algorithm 1 with
    the Gaussian sampling matrices Omega1 = G(seed, 1), Omega2 = G(seed, 2)
    (``hss.gaussian_matrix``), and Q_sel Qhat is formed by the HSS multiply.  With
    grow > 0 the sample is doubled up to `grow` times while an ID rank reaches it
    (``hss.rand_hss_adaptive``); a compression still saturated after that is not used:
    the merge keeps the exact product (info["hss_dense"] = True)."""
    from . import hss
    lam, u, info = merge(D, Q, n1, beta)
    kk = info["K"]
    if kk == 0:
        return lam, u, info
    n = D.shape[0]
    order = info["order"]
    cols = np.asarray(Q, dtype=np.float64)[:, order].copy()
    for (j, k, c, s) in info["rotations"]:
        cj, ck = cols[:, j].copy(), cols[:, k].copy()
        cols[:, j] = c * cj + s * ck
        cols[:, k] = -s * cj + c * ck
    qsel = cols[:, info["kept"]]
    root, nodes, rp_used, sat = hss.rand_hss_adaptive(info["qhat"], seed, rp, grow, leaf, tol)
    if sat:
        return lam, u, dict(info, hss_ranks=hss.hss_ranks(nodes), hss_rp=rp_used, hss_dense=True)
    u_nd = hss.hss_left_multiply(qsel, root, nodes)
    # place the non-deflated columns where ``merge`` put them
    fin = info["final_order"]
    out = u.copy()
    pos = np.empty(n, dtype=np.int64)
    pos[fin] = np.arange(n)
    out[:, pos[:kk]] = u_nd
    info = dict(info, hss_ranks=hss.hss_ranks(nodes), hss_rp=rp_used, hss_dense=False)
    return lam, out, info


# ----------------------------------------------------------------------------
# The DC tree (PDSTEDC analogue).
# ----------------------------------------------------------------------------
def sign_normalize(q: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of every column positive (first one on ties)."""
    q = np.array(q, copy=True)
    if q.size == 0:
        return q
    idx = np.argmax(np.abs(q), axis=0)
    sgn = np.sign(q[idx, np.arange(q.shape[1])])
    sgn[sgn == 0] = 1.0
    return q * sgn[None, :]


def dc_eig(d: np.ndarray, e: np.ndarray, leaf: int = 32, record=None):
    """Eigenvalues (ascending) and eigenvectors of tridiag(e, d, e) by Cuppen DC.

    If ``record`` is a list, (offset, n1, n2, info) of every merge is appended."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    return _dc(d, e, leaf, 0, record)


def _dc(d, e, leaf, offset, record):
    n = d.shape[0]
    if n <= leaf:
        return jacobi_eigh(tridiag_dense(d, e))
    n1 = n // 2
    beta = float(e[n1 - 1])
    d1 = d[:n1].copy()
    d2 = d[n1:].copy()
    d1[-1] -= abs(beta)                                   # Eq. (2) corner modification
    d2[0] -= abs(beta)
    l1, q1 = _dc(d1, e[:n1 - 1], leaf, offset, record)
    l2, q2 = _dc(d2, e[n1:], leaf, offset + n1, record)
    qb = np.zeros((n, n))
    qb[:n1, :n1] = q1
    qb[n1:, n1:] = q2
    lam, u, info = merge(np.concatenate([l1, l2]), qb, n1, beta)
    if record is not None:
        record.append((offset, n1, n - n1, info))
    return lam, u


def syev(d, e, leaf: int = 32):
    """dc_eig followed by the sign convention of the library's output."""
    lam, q = dc_eig(d, e, leaf)
    return lam, sign_normalize(q)
