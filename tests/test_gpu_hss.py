"""The HSS form of the eigenvector product (Algorithm 1 + HSS multiply) through the
C ABI, against the oracle's HSS merge (same sampling matrices: SplitMix64 Gaussian,
seed 0x5EED + merge id, streams 1 and 2) and against the exact dense merge.

The accuracy contract of the HSS path is the dense contract loosened by the stated
compression tolerance tol (1e-12, relative to each node's largest pivot), through
this bound.  An HSS merge replaces the orthogonal Qhat (||Qhat||_2 = 1) by an
approximation whose error is made level by level: at each of the L levels of the HSS
tree every node's ID drops the directions of its (r + p)-column sample whose pivots
are below tol times the largest, and the dropped part of a sample of r + p columns
of norm <= 1 has norm <= sqrt(r + p) tol.  The errors of the L levels add, and the
row and column sides (U and V bases) each contribute, so

    ||Qhat - Qhat_hss||_2 <= c_L tol,   c_L = 2 L sqrt(r + p).

The merge output Q_sel Qhat_hss then differs from the exact one by at most c_L tol
in 2-norm (Q_sel has orthonormal columns), so orthogonality moves by at most
2 c_L tol and the residual of the merged matrix A by at most 2 ||A|| c_L tol.  A full
solve adds the errors of the HSS merges on each root-to-leaf path, one per tree level
(the FP64 products above and below preserve the error's size)."""
import numpy as np
import pytest

import workloads as W
from oracle import dc, metrics, sturm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52
HSS = 2
AUTO = 3
TOL = 1e-12


def hss_levels(k, leaf):
    """Levels below the root of the HSS tree over k indices (a node of size > leaf
    splits at floor(size / 2), as Algorithm 1's tree is built)."""
    lv = 0
    while k > leaf:
        k = (k + 1) // 2
        lv += 1
    return lv


def merge_bound(k, leaf, rp, tol=TOL):
    """c_L tol of the module docstring for one HSS merge of order k."""
    return 2.0 * hss_levels(k, leaf) * np.sqrt(rp) * tol


def syev_bound(n, leaf, rp, is_hss, tol=TOL):
    """Sum of the HSS merges' bounds on the path through the largest merges of each DC
    level (node sizes n, ceil(n / 2), ... down to the 32-leaves); is_hss(m) says whether
    a merge of order m takes the HSS product."""
    tot, m = 0.0, n
    while m > 32:
        if is_hss(m):
            tot += merge_bound(m, leaf, rp, tol)
        m = (m + 1) // 2
    return tot


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _fortran(q):
    return torch.tensor(q, device="cuda").t().contiguous().t()


@pytest.mark.parametrize("n1,n2,seed,leaf,rp", [(600, 600, 5, 128, 64), (700, 555, 6, 128, 64),
                                                (1024, 1024, 7, 256, 96),
                                                # 512 samples on up to 1024 rows: the row IDs
                                                # do not fit a cluster's shared memory and take
                                                # the one-CTA kernel
                                                (1100, 1100, 9, 1024, 512)])
def test_merge_hss(api, n1, n2, seed, leaf, rp):
    D, Q, beta = W.merge_problem(n1, n2, seed)
    n = n1 + n2
    lam_d, u_d, info = dc.merge(D, Q, n1, beta)
    lam_h, u_h, info_h = dc.merge_hss(D, Q, n1, beta, leaf=leaf, rp=rp, tol=TOL, seed=0x5EED)
    opts = {"path": HSS, "hss_leaf": leaf, "hss_rp": rp, "hss_tol": TOL}
    lam, qo, K = api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta, opts=opts)
    lam = lam.cpu().numpy()
    qo = qo.cpu().numpy()
    assert K == info["K"]
    assert np.max(np.abs(lam - lam_d)) <= 10 * n * EPS * np.abs(D).max()
    b = merge_bound(K, leaf, rp)
    # same samples: the oracle's HSS merge; both are within b of the exact merge
    assert np.linalg.norm(qo - u_h, 2) <= 2 * b + 100 * n * EPS
    assert np.linalg.norm(qo - u_d, 2) <= b + 100 * n * EPS          # the exact merge
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n)
    v[n1 - 1] = 1.0
    v[n1] = np.sign(beta)
    a += abs(beta) * np.outer(v, v)
    na = np.linalg.norm(a, 2)
    assert np.linalg.norm(a @ qo - qo * lam, 2) <= 2 * na * b + 10 * n * EPS * na
    assert np.max(np.abs(qo.T @ qo - np.eye(n))) <= 2 * b + 100 * n * EPS


@pytest.mark.parametrize("gen,n", [("toeplitz", 4096), ("normal", 3000)])
def test_syev_hss(api, gen, n):
    d, e = W.toeplitz_121(n) if gen == "toeplitz" else W.normal_tridiag(n, 8)
    opts = {"path": HSS, "hss_leaf": 256, "hss_rp": 96, "hss_tol": TOL}
    lam_t, q_t = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"), opts=opts)
    lam = lam_t.cpu().numpy()
    q = q_t.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    idx = np.arange(0, n, max(1, n // 64))
    assert np.max(np.abs(lam[idx] - sturm.bisection_eigvals(d, e, idx))) <= 10 * n * EPS * nrm
    b = syev_bound(n, 256, 96, lambda m: m >= 2 * 256)
    assert metrics.orthogonality(q) <= 2 * b + 100 * n * EPS
    r = metrics.tri_matmul(d, e, q) - q * lam[None, :]
    assert np.linalg.norm(r) <= (2 * b * np.sqrt(n) + 10 * n * EPS) * nrm


def _profiled(api, fn):
    import ctypes
    from paper_1612_07526_gb300 import _lib
    lib = _lib.load()
    torch.cuda.synchronize()
    lib.tdc_profile_begin()
    out = fn()
    torch.cuda.synchronize()
    p = _lib.TdcProfile()
    lib.tdc_profile_end(ctypes.byref(p))
    return out, p


def test_hss_saturated_ranks_take_dense_product(api):
    """With r + p = 8 samples and no growth allowed the ID ranks of tridiag(1,2,1)'s
    Cauchy-like Qhat blocks reach the sample count, so every HSS merge (the 15 merges of
    order >= 2 x 128) takes the dense FP64 product instead: the solve equals the FP64
    path bit for bit.  With the default 128 samples no merge falls back."""
    n = 3000
    d, e = W.toeplitz_121(n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    (lam_h, q_h), p = _profiled(api, lambda: api.syev_tridiag(
        dt, et, opts={"path": 2, "hss_rp": 8, "hss_leaf": 128, "tile_cfg": 2, "hss_grow": 0}))
    assert p.hss_fallbacks == 15
    lam_f, q_f = api.syev_tridiag(dt, et, opts={"path": 0, "tile_cfg": 2})
    assert torch.equal(lam_h, lam_f) and torch.equal(q_h, q_f)
    (lam_d, q_d), p = _profiled(api, lambda: api.syev_tridiag(dt, et, opts={"path": 2, "hss_leaf": 128}))
    assert p.hss_fallbacks == 0
    lh, qh = lam_d.cpu().numpy(), q_d.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    b = syev_bound(n, 128, 128, lambda m: m >= 2 * 128)
    r = metrics.tri_matmul(d, e, qh) - qh * lh[None, :]
    assert np.linalg.norm(r) <= (2 * b * np.sqrt(n) + 10 * n * EPS) * nrm
    assert metrics.orthogonality(qh) <= 2 * b + 100 * n * EPS


@pytest.mark.parametrize("gen,n,kt", [("toeplitz", 4096, 4096), ("sht", 4096, 2048)])
def test_syev_auto_dispatch(api, gen, n, kt):
    """The AUTO path (Section 2.2's rule: the HSS product only for merges with large K,
    here of order >= k_threshold; the split product for the other merges of order >=
    1024; FP64 below): eigenvalues against Sturm bisection, eigenvectors against the
    FP64 path where the gaps allow, residual and orthogonality within the HSS bound of
    the merges that took HSS."""
    d, e = W.toeplitz_121(n) if gen == "toeplitz" else W.sht(n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    lam_a, q_a = api.syev_tridiag(dt, et, opts={"path": AUTO, "k_threshold": kt})
    lam_f, q_f = api.syev_tridiag(dt, et, opts={"path": 0})
    lam, q = lam_a.cpu().numpy(), q_a.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    idx = np.arange(0, n, max(1, n // 64))
    assert np.max(np.abs(lam[idx] - sturm.bisection_eigvals(d, e, idx))) <= 10 * n * EPS * nrm
    b = syev_bound(n, 512, 128, lambda m: m >= kt)
    assert b > 0
    assert metrics.orthogonality(q) <= 2 * b + 100 * n * EPS
    r = metrics.tri_matmul(d, e, q) - q * lam[None, :]
    assert np.linalg.norm(r) <= (2 * b * np.sqrt(n) + 10 * n * EPS) * nrm
    # eigenvectors whose gap g to the neighbours is large: sin(angle) <= (error) / g
    lf = lam_f.cpu().numpy()
    gap = np.full(n, np.inf)
    gap[:-1] = np.minimum(gap[:-1], np.diff(lf))
    gap[1:] = np.minimum(gap[1:], np.diff(lf))
    sel = np.nonzero(gap >= 1e-3 * nrm)[0]
    dots = np.abs(np.sum(q[:, sel] * q_f.cpu().numpy()[:, sel], axis=0))
    assert np.all(1.0 - dots <= ((2 * b + 20 * n * EPS) * nrm / gap[sel]) ** 2 + 1e-13)



def test_merge_hss_adaptive_growth(api):
    """Adaptive sampling: from r + p = 8 the sample is doubled while an ID rank reaches
    it (8 -> 16 -> 32 -> 64 here), and the merge equals the oracle's adaptive HSS merge
    (same sampling columns) within the bound of the sample it ended with."""
    n1, n2 = 600, 600
    D, Q, beta = W.merge_problem(n1, n2, 5)
    n = n1 + n2
    lam_h, u_h, info = dc.merge_hss(D, Q, n1, beta, leaf=128, rp=8, tol=TOL, seed=0x5EED, grow=3)
    assert not info["hss_dense"] and info["hss_rp"] == 64
    lam_d, u_d, _ = dc.merge(D, Q, n1, beta)
    opts = {"path": HSS, "hss_leaf": 128, "hss_rp": 8, "hss_tol": TOL, "hss_grow": 3}
    (lam, qo, K), p = _profiled(api, lambda: api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta,
                                                       opts=opts))
    assert p.hss_regrowths == 3 and p.hss_fallbacks == 0
    qo = qo.cpu().numpy()
    b = merge_bound(K, 128, 64)
    assert np.linalg.norm(qo - u_h, 2) <= 2 * b + 100 * n * EPS
    assert np.linalg.norm(qo - u_d, 2) <= b + 100 * n * EPS
    assert np.max(np.abs(qo.T @ qo - np.eye(n))) <= 2 * b + 100 * n * EPS
    # the grown sample extends the 64-column one: the same compression as r + p = 64
    lam64, q64, _ = api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta,
                              opts={"path": HSS, "hss_leaf": 128, "hss_rp": 64, "hss_tol": TOL, "hss_grow": 0})
    assert np.array_equal(q64.cpu().numpy(), qo)


def test_syev_hss_adaptive_growth(api):
    """A full HSS solve that starts every compression at r + p = 8: the samples grow
    until the ranks fit, no merge falls back to the dense product, and the solve meets
    the HSS contract of the largest sample it may reach."""
    n = 3000
    d, e = W.toeplitz_121(n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    (lam_t, q_t), p = _profiled(api, lambda: api.syev_tridiag(
        dt, et, opts={"path": HSS, "hss_rp": 8, "hss_leaf": 128, "hss_grow": 4}))
    assert p.hss_regrowths >= 15 and p.hss_fallbacks == 0
    lam, q = lam_t.cpu().numpy(), q_t.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    lref, _ = sturm.closed_form_121(n)
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * nrm
    b = syev_bound(n, 128, 8 << 4, lambda m: m >= 2 * 128)
    assert metrics.orthogonality(q) <= 2 * b + 100 * n * EPS
    r = metrics.tri_matmul(d, e, q) - q * lam[None, :]
    assert np.linalg.norm(r) <= (2 * b * np.sqrt(n) + 10 * n * EPS) * nrm
