"""Extended-precision eigenvectors (tdc_opts.eigvec = extended; Section 1's alternative to
the Loewner z, after Sorensen and Tang) through the C ABI, against the oracle's exact
version (oracle/extended.py: roots bisected on exact rationals, differences taken
exactly).

Bounds.  The GPU refines each FP64 root by one Newton step on the secular function
summed in double-double: the sum of K terms carries an error of at most
E2 = (K + 4) eps^2 (1 + rho sum_j z_j^2 / |d_j - lambda|), so the refined root lies
within E2 / f' of the exact one, plus the Newton step's own quadratic remainder
(about (tau_err)^2 / |tau| <= (c eps)^2 |tau| from an FP64 root c ulp off; c <= 512
covers the roots' conditioning seen in the secular tests), plus one rounding of the
pair (eps^2 |tau|).  The eigenvector components are then the oracle's to a few units
of eps each, and the merge output (one FP64 product over K terms) to n eps."""
import numpy as np
import pytest

import workloads as W
from oracle import dc, extended, metrics, sturm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
EXT = 1


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _fortran(q):
    return torch.tensor(np.asfortranarray(q), device="cuda").t().contiguous().t()


def _structured(n1, n2, a, b, seed):
    g = W.rng(seed)
    Q = np.zeros((n1 + n2, n1 + n2))
    Q[:n1, :n1] = np.eye(n1)
    Q[n1 - a:n1, n1 - a:n1] = W.random_orthogonal(a, g)
    Q[n1:, n1:] = np.eye(n2)
    Q[n1:n1 + b, n1:n1 + b] = W.random_orthogonal(b, g)
    D = np.concatenate([np.sort(g.uniform(-1, 1, n1)), np.sort(g.uniform(-1, 1, n2))])
    return D, Q, float(g.uniform(0.1, 1.0))


def _level_merge(n, seed):
    d, e = W.uniform_tridiag(n, seed)
    n1 = n // 2
    beta = float(e[n1 - 1])
    d1, d2 = d[:n1].copy(), d[n1:].copy()
    d1[-1] -= abs(beta)
    d2[0] -= abs(beta)
    l1, q1 = dc.dc_eig(d1, e[:n1 - 1])
    l2, q2 = dc.dc_eig(d2, e[n1:])
    Q = np.zeros((n, n))
    Q[:n1, :n1] = q1
    Q[n1:, n1:] = q2
    return np.concatenate([l1, l2]), Q, n1, beta


def _cases():
    g = W.rng(12)
    d1 = np.sort(g.uniform(-1, 1, 10))
    d2 = np.sort(g.uniform(-1, 1, 10))
    d2[4] = d1[6]
    d2[7] = d1[8]
    Qe = np.zeros((20, 20))
    Qe[:10, :10] = W.random_orthogonal(10, g)
    Qe[10:, 10:] = W.random_orthogonal(10, g)
    D8, Q8, b8 = _structured(20, 20, 4, 4, 8)
    D33, Q33, b33 = _structured(40, 40, 17, 16, 33)
    Dl, Ql, n1l, bl = _level_merge(512, 3)
    Dm, Qm, bm = W.merge_problem(24, 23, 4)
    return [("K8", D8, Q8, 20, b8), ("K33", D33, Q33, 40, b33),
            ("equal_poles", np.concatenate([d1, np.sort(d2)]), Qe, 10, 0.7),
            ("dense47", Dm, Qm, 24, bm), ("tridiag_level_512", Dl, Ql, n1l, bl)]


@pytest.mark.parametrize("case", range(5))
def test_merge_extended_against_exact(api, case):
    name, D, Q, n1, beta = _cases()[case]
    n = len(D)
    lam, qo, tr = api.merge_inspect(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta,
                                    opts={"eigvec": EXT})
    lam_x, u_x, info = extended.merge_extended(D, Q, n1, beta)
    K = info["K"]
    assert int(tr["counts"][0]) == K
    assert np.array_equal(tr["zhat"], info["zbar"])                 # the original z is kept
    lam = lam.cpu().numpy()
    qo = qo.cpu().numpy()
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n)
    v[n1 - 1] = 1.0
    v[n1] = np.sign(beta)
    a += abs(beta) * np.outer(v, v)
    assert np.max(np.abs(lam - lam_x)) <= 20 * n * EPS * np.abs(a).sum(1).max()
    assert np.linalg.norm(a @ qo - qo * lam) <= 10 * n * 2 * EPS * np.linalg.norm(a)
    assert np.max(np.abs(qo.T @ qo - np.eye(n))) <= 100 * n * 2 * EPS
    if K == 0:
        return
    # refined roots against the exact ones (same origin; else the same eigenvalue)
    dbar, zbar, rho = info["dbar"], info["zbar"], info["rho"]
    org = tr["origin"].astype(np.int64)
    same = org == info["origin"]
    assert same.sum() >= K - 2
    ex_hi, ex_lo, _ = extended.exact_roots(dbar, zbar, rho, org, tr["tau"])
    lam_m_d = (dbar[org][:, None] - dbar[None, :]) + ex_hi[:, None]
    terms = rho * zbar[None, :] ** 2 / np.abs(lam_m_d)
    fprime = rho * np.sum(zbar[None, :] ** 2 / lam_m_d ** 2, axis=1)
    bound = 4 * (K + 4) * EPS ** 2 * (1.0 + terms.sum(1)) / fprime + (512 * EPS) ** 2 * np.abs(ex_hi) \
        + 2 * EPS ** 2 * np.abs(ex_hi)
    err = np.abs((tr["tau"] - ex_hi) + (tr["tau_lo"] - ex_lo))
    assert np.all(err <= bound), float(np.max(err / bound))
    # the merge output against the oracle's extended merge, column by column
    sgn = np.sign(np.sum(qo * u_x, axis=0))
    sgn[sgn == 0] = 1.0
    assert np.max(np.abs(qo - u_x * sgn[None, :])) <= 20 * n * EPS
    print(name, "K", K, "max root error / bound", float(np.max(err / bound)))


@pytest.mark.parametrize("gen,n,path", [("uniform", 1000, 0), ("toeplitz", 2048, 0), ("hermite", 600, 0),
                                        ("toeplitz", 4096, 1)])
def test_syev_extended_contract(api, gen, n, path):
    """Full solves with extended-precision eigenvectors on both dense product forms:
    eigenvalues against Sturm bisection and the oracle, residual and orthogonality
    within the accuracy contract."""
    d, e = {"uniform": lambda: W.uniform_tridiag(n, 5), "toeplitz": lambda: W.toeplitz_121(n),
            "hermite": lambda: W.hermite(n)}[gen]()
    lam_t, q_t = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"),
                                  opts={"eigvec": EXT, "path": path})
    lam, q = lam_t.cpu().numpy(), q_t.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    e52 = 2.0 ** -52
    idx = np.arange(0, n, max(1, n // 64))
    assert np.max(np.abs(lam[idx] - sturm.bisection_eigvals(d, e, idx))) <= 10 * n * e52 * nrm
    assert metrics.scaled_residual(d, e, lam, q) <= 10
    assert metrics.orthogonality(q) <= 100 * n * e52
    if n <= 1000:
        lref, qref = dc.syev(d, e)
        err, _ = metrics.column_agreement(lref, qref, q, nrm, min_relgap=1e-4)
        assert err <= 1e-7


def test_extended_batched(api):
    """A ragged batch with extended-precision eigenvectors: every problem against the
    oracle and within the accuracy contract."""
    sizes = [300, 77, 512, 1]
    ds, es = [], []
    for k, n in enumerate(sizes):
        d, e = W.normal_tridiag(n, 300 + k)
        ds.append(d)
        es.append(e)
    lam, q, sz, qoff = api.syev_tridiag_batched(ds, es, opts={"eigvec": EXT})
    off = 0
    e52 = 2.0 ** -52
    for p, n in enumerate(sizes):
        lp = lam[off:off + n].cpu().numpy()
        qp = api.batched_block(q, sz, qoff, p).cpu().numpy()
        lref, qref = dc.syev(ds[p], es[p])
        nrm = metrics.tnorm(ds[p], es[p])
        assert np.max(np.abs(lp - lref)) <= 10 * n * e52 * nrm
        assert metrics.scaled_residual(ds[p], es[p], lp, qp) <= 10
        assert metrics.orthogonality(qp) <= 100 * n * e52
        off += n
