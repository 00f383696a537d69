"""HSS construction and multiplication (TEST INFRASTRUCTURE: only tests/,
``__graft_entry__`` and bench.py's CPU arms may import this module).

* ``hss_tree``   binary postordered tree over contiguous index sets t_i
                 (Section 2, the conditions on t_i and Fig. 1).
* ``rand_hss``   Algorithm 1 (RandHSS): random sampling Y = A Omega1,
                 Z = A^T Omega2, then leaves-to-root interpolative
                 decompositions, in the algorithm's order and notation.
* ``interp_decomp``  row ID  Phi ~= U Phi|_I  by column-pivoted QR of Phi^T
                 (the paper does not name the ID method; CPQR is the usual one).
* ``hss_to_dense``   the matrix represented by the generators (Eqs. 7-8).
* ``hss_left_multiply``  X A for A in HSS form by an up-sweep of X U, the
                 sibling couplings B, and a down-sweep through V (the fast
                 multiply of Section 2, O(N r) per row of X).

Generators follow Eq. (7): for a leaf, D_i, U_i, V_i; for every non-root node,
B_i couples it to its sibling: A(t_{i1}, t_{i2}) = Uhat_{i1} B_{i1} Vhat_{i2}^T.
Skeleton index sets (I~_i, J~_i) are global indices into A.
The random matrices Omega1, Omega2 are inputs (drawn by the caller).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

SPLITMIX_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, idx) -> np.ndarray:
    """Output number idx (0-based) of the SplitMix64 sequence seeded with `seed`
    (Steele, Lea and Flood, 2014): z = seed + (idx+1) * gamma, then the two
    xor-shift-multiply rounds and a final xor-shift, all modulo 2^64."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * np.uint64(SPLITMIX_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def gaussian_matrix(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols standard normal matrix (column-major element order) by Box-Muller:
    element (r, c) with q = stream * 2^40 + c * rows + r uses draws 2q and 2q+1,
    u1 = (draw >> 11 + 1) 2^-53 in (0, 1], u2 = (draw >> 11) 2^-53, and
    g = sqrt(-2 ln u1) cos(2 pi u2).  These are the random sampling matrices of
    Algorithm 1 as the library draws them."""
    r = np.arange(rows, dtype=np.uint64)[:, None]
    c = np.arange(cols, dtype=np.uint64)[None, :]
    q = np.uint64(stream) * np.uint64(1 << 40) + c * np.uint64(rows) + r
    z1 = splitmix64(seed, np.uint64(2) * q)
    z2 = splitmix64(seed, np.uint64(2) * q + np.uint64(1))
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


class Node:
    __slots__ = ("idx", "lo", "hi", "left", "right", "parent", "level",
                 "D", "U", "V", "B", "I", "J", "Phi", "Theta", "Yh", "Zh")

    def __init__(self, lo, hi, level):
        self.lo, self.hi, self.level = lo, hi, level
        self.left = self.right = self.parent = None
        self.D = self.U = self.V = self.B = None
        self.I = self.J = None
        self.Phi = self.Theta = self.Yh = self.Zh = None
        self.idx = -1

    @property
    def leaf(self):
        return self.left is None


def hss_tree(n: int, leaf: int):
    """Postordered binary tree: a node of size > leaf splits at floor(size / 2)."""
    nodes = []

    def build(lo, hi, level):
        nd = Node(lo, hi, level)
        if hi - lo > leaf:
            mid = lo + (hi - lo) // 2
            nd.left = build(lo, mid, level + 1)
            nd.right = build(mid, hi, level + 1)
            nd.left.parent = nd
            nd.right.parent = nd
        nd.idx = len(nodes)
        nodes.append(nd)
        return nd

    root = build(0, n, 0)
    return root, nodes


def interp_decomp(phi: np.ndarray, tol: float, max_rank: int | None = None):
    """Row interpolative decomposition: phi ~= U @ phi[I], U[I] = identity.

    Column-pivoted QR of phi^T; the rank is the number of |R_kk| > tol |R_00|."""
    m = phi.shape[0]
    if m == 0 or phi.shape[1] == 0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    _, r, piv = sla.qr(phi.T, mode="economic", pivoting=True)
    diag = np.abs(np.diag(r))
    if diag.size == 0 or diag[0] == 0.0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    k = int(np.sum(diag > tol * diag[0]))
    if max_rank is not None:
        k = min(k, max_rank)
    t = sla.solve_triangular(r[:k, :k], r[:k, k:], lower=False) if k < m else np.zeros((k, 0))
    u = np.zeros((m, k))
    u[piv[:k], :] = np.eye(k)
    u[piv[k:], :] = t.T
    return u, piv[:k].astype(np.int64)


def rand_hss(A, omega1: np.ndarray, omega2: np.ndarray, leaf: int, tol: float,
             entries=None):
    """Algorithm 1.  ``A`` is a dense matrix, or None when ``entries(rows, cols)``
    returns A[rows][:, cols]; in that case the samples Y, Z must be passed as
    ``A = (Y, Z)``.  Returns (root, nodes) carrying the generators."""
    if entries is None:
        a = np.asarray(A, dtype=np.float64)
        n = a.shape[0]
        y = a @ omega1
        z = a.T @ omega2

        def entries(r, c):
            return a[np.ix_(r, c)]
    else:
        y, z = A
        n = y.shape[0]
    root, nodes = hss_tree(n, leaf)
    maxlev = max(nd.level for nd in nodes)
    for lev in range(maxlev, 0, -1):                     # do l = L, ..., 1
        for nd in nodes:
            if nd.level != lev:
                continue
            if nd.leaf:
                t = np.arange(nd.lo, nd.hi)
                nd.D = entries(t, t)                                     # step 1
                nd.Phi = y[t] - nd.D @ omega1[t]                         # step 2
                nd.Theta = z[t] - nd.D.T @ omega2[t]
                nd.U, iloc = interp_decomp(nd.Phi, tol)                  # step 3
                nd.V, jloc = interp_decomp(nd.Theta, tol)
                nd.I, nd.J = t[iloc], t[jloc]
                nd.Phi, nd.Theta = nd.Phi[iloc], nd.Theta[jloc]          # keep Phi|_I, Theta|_J
                nd.Yh = nd.V.T @ omega1[t]                               # step 4
                nd.Zh = nd.U.T @ omega2[t]
            else:
                c1, c2 = nd.left, nd.right
                c1.B = entries(c1.I, c2.J)                               # step 1
                c2.B = entries(c2.I, c1.J)
                phi = np.vstack([c1.Phi - c1.B @ c2.Yh,                  # step 2
                                 c2.Phi - c2.B @ c1.Yh])
                theta = np.vstack([c1.Theta - c2.B.T @ c2.Zh,
                                   c2.Theta - c1.B.T @ c1.Zh])
                nd.U, iloc = interp_decomp(phi, tol)                     # step 3
                nd.V, jloc = interp_decomp(theta, tol)
                ivec = np.concatenate([c1.I, c2.I])
                jvec = np.concatenate([c1.J, c2.J])
                nd.I, nd.J = ivec[iloc], jvec[jloc]
                nd.Phi, nd.Theta = phi[iloc], theta[jloc]
                nd.Yh = nd.V.T @ np.vstack([c1.Yh, c2.Yh])               # step 4
                nd.Zh = nd.U.T @ np.vstack([c1.Zh, c2.Zh])
    if not root.leaf:                                                    # root couplings
        root.left.B = entries(root.left.I, root.right.J)
        root.right.B = entries(root.right.I, root.left.J)
    else:
        t = np.arange(root.lo, root.hi)
        root.D = entries(t, t)
    return root, nodes


def _nested(nd, which):
    """Uhat_i (which='U') or Vhat_i (which='V') as a dense (|t_i| x rank) matrix."""
    g = nd.U if which == "U" else nd.V
    if nd.leaf:
        return g
    a = _nested(nd.left, which)
    b = _nested(nd.right, which)
    blk = np.zeros((a.shape[0] + b.shape[0], a.shape[1] + b.shape[1]))
    blk[:a.shape[0], :a.shape[1]] = a
    blk[a.shape[0]:, a.shape[1]:] = b
    return blk @ g


def hss_to_dense(root) -> np.ndarray:
    """Eq. (7): D_i = [[D_i1, Uhat_i1 B_i1 Vhat_i2^T], [Uhat_i2 B_i2 Vhat_i1^T, D_i2]]."""
    if root.leaf:
        return root.D.copy()
    c1, c2 = root.left, root.right
    a11 = hss_to_dense(c1)
    a22 = hss_to_dense(c2)
    a12 = _nested(c1, "U") @ c1.B @ _nested(c2, "V").T
    a21 = _nested(c2, "U") @ c2.B @ _nested(c1, "V").T
    return np.block([[a11, a12], [a21, a22]])


def hss_left_multiply(x: np.ndarray, root, nodes) -> np.ndarray:
    """X @ A with A given by its HSS generators (X has A's order columns)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((x.shape[0], root.hi - root.lo))
    if root.leaf:
        return x @ root.D
    g = {}
    for nd in nodes:                                  # postorder: children before parents
        if nd is root:
            continue
        if nd.leaf:
            g[nd.idx] = x[:, nd.lo:nd.hi] @ nd.U
        else:
            g[nd.idx] = np.hstack([g[nd.left.idx], g[nd.right.idx]]) @ nd.U
    f = {}
    for nd in reversed(nodes):                        # parents before children
        if nd.leaf:
            continue
        c1, c2 = nd.left, nd.right
        f1 = g[c2.idx] @ c2.B                         # A(t_c2, t_c1) = Uhat_c2 B_c2 Vhat_c1^T
        f2 = g[c1.idx] @ c1.B
        if nd.idx in f:
            e = f[nd.idx] @ nd.V.T
            k1 = c1.V.shape[1]
            f1 = f1 + e[:, :k1]
            f2 = f2 + e[:, k1:]
        f[c1.idx] = f1
        f[c2.idx] = f2
    for nd in nodes:
        if nd.leaf:
            out[:, nd.lo:nd.hi] = x[:, nd.lo:nd.hi] @ nd.D + f[nd.idx] @ nd.V.T
    return out


def hss_ranks(nodes):
    return [nd.U.shape[1] for nd in nodes if nd.U is not None]


def saturated(nodes, rp: int) -> bool:
    """True when some non-root node's row or column ID kept all rp sample columns while
    its sample had more rows than that: the sampled range may then miss part of the
    off-diagonal block, and the compression cannot be trusted at the tolerance."""
    for nd in nodes:
        if nd.parent is None or nd.U is None:
            continue
        if (nd.U.shape[1] >= rp and nd.U.shape[0] > rp) or (nd.V.shape[1] >= rp and nd.V.shape[0] > rp):
            return True
    return False


def rand_hss_adaptive(a, seed: int, rp0: int, grow: int, leaf: int, tol: float):
    """Algorithm 1 with the sample grown as the paper's adaptive sampling does
    (Section 2.1): compress with r + p = rp0 Gaussian sample columns; while a node's ID
    rank reaches the sample count, double it (at most `grow` times) and compress again
    with the larger sample, whose first columns are the previous sample's (column c of
    ``gaussian_matrix`` does not depend on the column count).  Returns
    (root, nodes, rp used, still saturated)."""
    a = np.asarray(a, dtype=np.float64)
    k = a.shape[0]
    rp = rp0
    for g in range(grow + 1):
        om1 = gaussian_matrix(seed, 1, k, rp)
        om2 = gaussian_matrix(seed, 2, k, rp)
        root, nodes = rand_hss(a, om1, om2, leaf, tol)
        if not saturated(nodes, rp):
            return root, nodes, rp, False
        if g < grow:
            rp *= 2
    return root, nodes, rp, True
