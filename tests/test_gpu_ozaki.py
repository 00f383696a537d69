"""The split-precision (bf16 slices on tcgen05) eigenvector product: parity with the
oracle and with the native FP64 product, through the C ABI.

The product changes only the eigenvectors; the accuracy contract is the same as for
the FP64 path (residual <= 10 n eps ||T||, orthogonality <= 100 n eps) and the two
products must agree to a few units of 1e-15 per entry."""
import numpy as np
import pytest

import workloads as W
from oracle import dc, metrics, sturm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52
OZ = 1


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _fortran(q):
    return torch.tensor(q, device="cuda").t().contiguous().t()


@pytest.mark.parametrize("n1,n2,seed", [(512, 512, 0), (700, 731, 1), (1024, 1000, 2), (1500, 1501, 3)])
def test_merge_ozaki_vs_oracle_and_fp64(api, n1, n2, seed):
    D, Q, beta = W.merge_problem(n1, n2, seed)
    n = n1 + n2
    lam_r, u_r, info = dc.merge(D, Q, n1, beta)
    lam_o, q_o, K_o = api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta, opts={"path": OZ})
    lam_f, q_f, K_f = api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta, opts={"path": 0})
    assert K_o == K_f == info["K"]
    assert torch.equal(lam_o, lam_f)
    q_o = q_o.cpu().numpy()
    q_f = q_f.cpu().numpy()
    lam = lam_o.cpu().numpy()
    assert np.max(np.abs(q_o - q_f)) <= 2e-14
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n)
    v[n1 - 1] = 1.0
    v[n1] = np.sign(beta)
    a += abs(beta) * np.outer(v, v)
    assert np.linalg.norm(a @ q_o - q_o * lam) <= 10 * n * EPS * np.linalg.norm(a)
    assert np.max(np.abs(q_o.T @ q_o - np.eye(n))) <= 100 * n * EPS
    err, _ = metrics.column_agreement(lam_r, u_r, q_o, np.abs(a).sum(1).max(), min_relgap=1e-4)
    assert err <= 1e-8


@pytest.mark.parametrize("gen,n", [("toeplitz", 4096), ("uniform", 3000), ("normal", 2500), ("clement", 2049),
                                   ("sht", 3000)])
def test_syev_ozaki(api, gen, n):
    d, e = {"toeplitz": lambda: W.toeplitz_121(n), "uniform": lambda: W.uniform_tridiag(n, 3),
            "normal": lambda: W.normal_tridiag(n, 4), "clement": lambda: W.clement(n),
            "sht": lambda: W.sht(n)}[gen]()
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    lam_o, q_o = api.syev_tridiag(dt, et, opts={"path": OZ})
    lam_f, q_f = api.syev_tridiag(dt, et, opts={"path": 0})
    # above the first split-precision level the merge inputs differ at rounding level,
    # so eigenvalues agree to the contract tolerance and eigenvectors where gaps allow
    lam = lam_o.cpu().numpy()
    q = q_o.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    assert np.max(np.abs(lam - lam_f.cpu().numpy())) <= 10 * n * EPS * nrm
    assert metrics.scaled_residual(d, e, lam, q) <= 10
    assert metrics.orthogonality(q) <= 100 * n * EPS
    err, mask = metrics.column_agreement(lam_f.cpu().numpy(), q_f.cpu().numpy(), q, nrm, min_relgap=1e-4)
    assert err <= 1e-8
    lref = sturm.bisection_eigvals(d, e, np.arange(0, n, max(1, n // 64)))
    assert np.max(np.abs(lam[::max(1, n // 64)] - lref)) <= 10 * n * EPS * nrm


def test_full_size_toeplitz_16384_ozaki(api):
    n = 16384
    d, e = W.toeplitz_121(n)
    lam_t, q_t = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"),
                                  opts={"path": OZ})
    lam = lam_t.cpu().numpy()
    lref, _ = sturm.closed_form_121(n)
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * 4.0
    g = W.rng(7)
    cols = np.sort(g.choice(n, 64, replace=False))
    qs = q_t[:, torch.tensor(cols, device="cuda")]
    gram = (q_t.t() @ qs).cpu().numpy()
    gram[cols, np.arange(64)] -= 1.0
    assert np.max(np.abs(gram)) <= 100 * n * EPS
    qs = qs.cpu().numpy()
    r = metrics.tri_matmul(d, e, qs) - qs * lam[cols][None, :]
    assert np.linalg.norm(r) / np.sqrt(64 / n) <= 10 * n * EPS * 4.0


@pytest.mark.parametrize("slices,tol", [(5, 1e-11), (6, 2e-14), (7, 3e-15)])
def test_merge_slice_counts(api, slices, tol):
    """S digit slices represent each scaled entry to 2^-8S, so the product's distance
    to the FP64 product shrinks by about 2^8 per slice (S = 7 is at FP64 rounding)."""
    n1, n2 = 1024, 1000
    D, Q, beta = W.merge_problem(n1, n2, 5)
    n = n1 + n2
    lam_o, q_o, K_o = api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta,
                                opts={"path": OZ, "ozaki_slices": slices})
    lam_f, q_f, K_f = api.merge(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta, opts={"path": 0})
    assert K_o == K_f and torch.equal(lam_o, lam_f)
    q_o = q_o.cpu().numpy()
    assert np.max(np.abs(q_o - q_f.cpu().numpy())) <= tol
    assert np.max(np.abs(q_o.T @ q_o - np.eye(n))) <= 100 * n * EPS


def test_syev_seven_slices_accuracy(api):
    n = 4096
    d, e = W.toeplitz_121(n)
    lam_t, q_t = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"),
                                  opts={"path": OZ, "ozaki_slices": 7})
    lam, q = lam_t.cpu().numpy(), q_t.cpu().numpy()
    lref, _ = sturm.closed_form_121(n)
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * 4.0
    assert metrics.scaled_residual(d, e, lam, q) <= 1.0     # S = 6 gives about 4 here
    assert metrics.orthogonality(q) <= 100 * n * EPS
