"""The HSS form of the eigenvector product (Algorithm 1 + HSS multiply) through the
C ABI, against the oracle's HSS merge (same sampling matrices: SplitMix64 Gaussian,
seed 0x5EED + merge id, streams 1 and 2) and against the exact dense merge.

The accuracy contract of the HSS path is the dense contract loosened by the stated
compression tolerance (1e-12 relative, per ID): eigenvectors agree with the dense
result, and residual and orthogonality are bounded, to a small multiple of it."""
import numpy as np
import pytest

import workloads as W
from oracle import dc, metrics, sturm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52
HSS = 2
TOL = 1e-12


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _fortran(q):
    return torch.tensor(q, device="cuda").t().contiguous().t()


@pytest.mark.parametrize("n1,n2,seed,leaf,rp", [(600, 600, 5, 128, 64), (700, 555, 6, 128, 64),
                                                (1024, 1024, 7, 256, 96)])
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
    assert np.max(np.abs(qo - u_h)) <= 1e-10          # same samples: the oracle's HSS merge
    assert np.max(np.abs(qo - u_d)) <= 1e-9           # the exact merge, to the tolerance
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n)
    v[n1 - 1] = 1.0
    v[n1] = np.sign(beta)
    a += abs(beta) * np.outer(v, v)
    assert np.linalg.norm(a @ qo - qo * lam) <= 1e-9 * np.linalg.norm(a)
    assert np.max(np.abs(qo.T @ qo - np.eye(n))) <= 1e-9


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
    assert metrics.orthogonality(q) <= 1e-9
    r = metrics.tri_matmul(d, e, q) - q * lam[None, :]
    assert np.linalg.norm(r) <= 1e-9 * nrm * np.sqrt(n)


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
    """With r + p = 8 samples the ID ranks of tridiag(1,2,1)'s Cauchy-like Qhat blocks
    reach the sample count, so every HSS merge (the 15 merges of order >= 2 x 128) takes
    the dense FP64 product instead: the solve equals the FP64 path bit for bit.  With
    the default 128 samples no merge falls back."""
    n = 3000
    d, e = W.toeplitz_121(n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    (lam_h, q_h), p = _profiled(api, lambda: api.syev_tridiag(
        dt, et, opts={"path": 2, "hss_rp": 8, "hss_leaf": 128, "tile_cfg": 2}))
    assert p.hss_fallbacks == 15
    lam_f, q_f = api.syev_tridiag(dt, et, opts={"path": 0, "tile_cfg": 2})
    assert torch.equal(lam_h, lam_f) and torch.equal(q_h, q_f)
    (lam_d, q_d), p = _profiled(api, lambda: api.syev_tridiag(dt, et, opts={"path": 2, "hss_leaf": 128}))
    assert p.hss_fallbacks == 0
    lh, qh = lam_d.cpu().numpy(), q_d.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    r = metrics.tri_matmul(d, e, qh) - qh * lh[None, :]
    assert np.linalg.norm(r) <= 1e-9 * nrm * np.sqrt(n)        # the HSS contract (tolerance 1e-12)
    assert metrics.orthogonality(qh) <= 1e-9
