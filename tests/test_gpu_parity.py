"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small and medium sizes are compared element by element with the oracle; the full
benchmark sizes (n = 16384, 32768) are checked on sampled outputs the oracle computes
one by one (Sturm-bisection eigenvalues, closed forms) and on properties that hold at
any size (residual and orthogonality of sampled columns).

Tolerances (the accuracy contract): |lambda - lambda_ref| <= 10 n eps ||T||,
||T Q - Q Lambda||_F / (n eps ||T||) <= 10, ||Q^T Q - I||_max <= 100 n eps, eps = 2^-52.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dc, metrics, sturm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _solve(api, d, e, **opts):
    lam, q = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"),
                              opts=opts or None)
    return lam.cpu().numpy(), q.cpu().numpy()


def _check_full(d, e, lam, q, lref, qref):
    n = len(d)
    nrm = metrics.tnorm(d, e)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * nrm
    assert metrics.scaled_residual(d, e, lam, q) <= 10
    assert metrics.orthogonality(q) <= 100 * n * EPS
    err, mask = metrics.column_agreement(lref, qref, q, nrm, min_relgap=1e-4)
    assert err <= 1e-7
    # sign convention: largest-magnitude entry positive
    idx = np.argmax(np.abs(q), axis=0)
    assert np.all(q[idx, np.arange(n)] > 0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 64, 65, 100, 257, 1000])
def test_syev_uniform_small(api, n):
    d, e = W.uniform_tridiag(n, n)
    lam, q = _solve(api, d, e)
    lref, qref = dc.syev(d, e)
    _check_full(d, e, lam, q, lref, qref)


@pytest.mark.parametrize("gen", ["normal", "graded", "toeplitz", "clement", "hermite", "sht"])
def test_syev_families(api, gen):
    n = 600
    d, e = {"normal": lambda: W.normal_tridiag(n, 1), "graded": lambda: W.graded_tridiag(n, 2),
            "toeplitz": lambda: W.toeplitz_121(n), "clement": lambda: W.clement(n),
            "hermite": lambda: W.hermite(n), "sht": lambda: W.sht(n)}[gen]()
    lam, q = _solve(api, d, e)
    lref, qref = dc.syev(d, e)
    _check_full(d, e, lam, q, lref, qref)


@pytest.mark.parametrize("leaf", [1, 4, 17, 32])
def test_syev_leaf_sizes(api, leaf):
    d, e = W.uniform_tridiag(300, 7)
    lam, q = _solve(api, d, e, leaf=leaf)
    lref, qref = dc.syev(d, e, leaf=leaf)
    _check_full(d, e, lam, q, lref, qref)


def test_syev_c1_config(api):
    """n = 1024, d, e ~ U[-1, 1], leaf 32: full eigenpairs against the oracle."""
    d, e = W.uniform_tridiag(1024, 0)
    lam, q = _solve(api, d, e)
    lref, qref = dc.syev(d, e)
    _check_full(d, e, lam, q, lref, qref)


def _merge_ref(D, Q, n1, beta):
    lam, u, info = dc.merge(D, Q, n1, beta)
    return lam, u, info


@pytest.mark.parametrize("n1,n2,seed", [(16, 16, 0), (33, 40, 1), (100, 57, 2), (300, 301, 3),
                                        (1, 1, 4), (1, 9, 5), (130, 129, 6)])
def test_merge_parity(api, n1, n2, seed):
    D, Q, beta = W.merge_problem(n1, n2, seed)
    lam_r, u_r, info = _merge_ref(D, Q, n1, beta)
    lam, qo, K = api.merge(torch.tensor(D, device="cuda"),
                           torch.tensor(np.asfortranarray(Q), device="cuda").t().contiguous().t(),
                           n1, beta)
    lam = lam.cpu().numpy()
    qo = qo.cpu().numpy()
    n = n1 + n2
    assert K == info["K"]
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n)
    v[n1 - 1] = 1.0
    v[n1] = np.sign(beta) if beta != 0 else 1.0
    a += abs(beta) * np.outer(v, v)
    nrm = np.abs(a).sum(1).max()
    assert np.max(np.abs(lam - lam_r)) <= 10 * n * EPS * nrm
    assert np.linalg.norm(a @ qo - qo * lam) <= 10 * n * EPS * np.linalg.norm(a)
    assert np.max(np.abs(qo.T @ qo - np.eye(n))) <= 100 * n * EPS
    err, _ = metrics.column_agreement(lam_r, u_r, qo, nrm, min_relgap=1e-4)
    assert err <= 1e-8


def test_merge_deflation_type1(api):
    g = W.rng(3)
    n1, n2 = 20, 12
    Q = np.zeros((32, 32))
    Q[:n1 - 1, :n1 - 1] = W.random_orthogonal(n1 - 1, g)
    Q[n1 - 1, n1 - 1] = 1.0
    Q[n1:, n1:] = W.random_orthogonal(n2, g)
    D = np.concatenate([np.sort(g.uniform(-1, 1, n1)), np.sort(g.uniform(-1, 1, n2))])
    lam_r, u_r, info = dc.merge(D, Q, n1, -0.6)
    lam, qo, K = api.merge(torch.tensor(D, device="cuda"),
                           torch.tensor(Q, device="cuda").t().contiguous().t(), n1, -0.6)
    assert K == info["K"] < 32
    assert np.max(np.abs(lam.cpu().numpy() - lam_r)) <= 1e-14
    qo = qo.cpu().numpy()
    err, _ = metrics.column_agreement(lam_r, u_r, qo, 2.0, min_relgap=1e-6)
    assert err <= 1e-10


def test_merge_deflation_type2_equal_poles(api):
    g = W.rng(12)
    d1 = np.sort(g.uniform(-1, 1, 10))
    d2 = np.sort(g.uniform(-1, 1, 10))
    d2[4] = d1[6]
    d2[7] = d1[8]
    d2 = np.sort(d2)
    D = np.concatenate([d1, d2])
    Q = np.zeros((20, 20))
    Q[:10, :10] = W.random_orthogonal(10, g)
    Q[10:, 10:] = W.random_orthogonal(10, g)
    lam_r, u_r, info = dc.merge(D, Q, 10, 0.7)
    assert len(info["rotations"]) >= 2
    lam, qo, K = api.merge(torch.tensor(D, device="cuda"),
                           torch.tensor(Q, device="cuda").t().contiguous().t(), 10, 0.7)
    assert K == info["K"]
    lam = lam.cpu().numpy()
    qo = qo.cpu().numpy()
    assert np.max(np.abs(lam - lam_r)) <= 1e-14
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(20)
    v[9] = v[10] = 1.0
    a += 0.7 * np.outer(v, v)
    assert np.linalg.norm(a @ qo - qo * lam) <= 1e-13
    assert np.max(np.abs(qo.T @ qo - np.eye(20))) <= 1e-13


def test_merge_zero_coupling(api):
    D, Q, _ = W.merge_problem(12, 13, 9)
    lam, qo, K = api.merge(torch.tensor(D, device="cuda"),
                           torch.tensor(Q, device="cuda").t().contiguous().t(), 12, 0.0)
    assert K == 0
    lam_r, u_r, _ = dc.merge(D, Q, 12, 0.0)
    assert np.array_equal(lam.cpu().numpy(), lam_r)
    assert np.array_equal(np.abs(qo.cpu().numpy()), np.abs(u_r))


def test_nonfinite_input_reported(api):
    d, e = W.uniform_tridiag(100, 1)
    d[17] = np.nan
    with pytest.raises(api.TdcError, match="non-finite"):
        _solve(api, d, e)
    # the context stays usable
    d, e = W.uniform_tridiag(50, 2)
    lam, q = _solve(api, d, e)
    assert metrics.scaled_residual(d, e, lam, q) <= 10


def test_secular_iteration_cap_reported(api):
    d, e = W.uniform_tridiag(200, 3)
    with pytest.raises(api.TdcError, match="secular"):
        _solve(api, d, e, max_secular_iter=1)


def test_batched_ragged(api):
    sizes = [1, 2, 31, 32, 33, 64, 100, 257, 513, 40]
    ds, es = [], []
    for k, n in enumerate(sizes):
        d, e = W.normal_tridiag(n, 100 + k)
        ds.append(d)
        es.append(e)
    lam, q, sz, qoff = api.syev_tridiag_batched(ds, es)
    lam = lam.cpu().numpy()
    off = 0
    for p, n in enumerate(sizes):
        lp = lam[off:off + n]
        qp = api.batched_block(q, sz, qoff, p).cpu().numpy()
        lref, qref = dc.syev(ds[p], es[p])
        _check_full(ds[p], es[p], lp, qp, lref, qref)
        off += n


def test_host_pipeline_matches_device_entry(api):
    """tdc_syev_tridiag_host_async with two solves in flight: every result is the
    device entry's, bit for bit, including slots reused by later submissions."""
    n = 500
    probs = [W.uniform_tridiag(n, 40 + k) for k in range(5)]
    pipe = api.HostPipeline(n, depth=2)
    got = []
    for k, (d, e) in enumerate(probs):
        slot = pipe.submit(torch.tensor(d).pin_memory(), torch.tensor(np.append(e, 0.0)).pin_memory())
        if k >= 1:
            prev = (slot + 1) % 2
            lam_p, q_p = pipe.result(prev)
            got.append((k - 1, lam_p.numpy().copy(), q_p.numpy().copy()))
    lam_p, q_p = pipe.result((len(probs) - 1) % 2)
    got.append((len(probs) - 1, lam_p.numpy().copy(), q_p.numpy().copy()))
    pipe.wait_all()
    assert len(got) == len(probs)
    for k, lam_h, q_h in got:
        lam_d, q_d = _solve(api, *probs[k])
        assert np.array_equal(lam_h, lam_d)
        assert np.array_equal(q_h, q_d)


def test_host_entry_matches_device_entry(api):
    n = 300
    d, e = W.uniform_tridiag(n, 11)
    hs = api.HostSolver(n)
    lam_h, q_h = hs(torch.tensor(d).pin_memory(), torch.tensor(e).pin_memory())
    lam_d, q_d = _solve(api, d, e)
    assert np.array_equal(lam_h.numpy(), lam_d)
    assert np.array_equal(q_h.numpy(), q_d)


# --------------------------------------------------------------------------- full sizes
def _sampled_checks(d, e, lam, q_dev, sample_cols, sample_eigs):
    n = len(d)
    nrm = metrics.tnorm(d, e)
    ref = sturm.bisection_eigvals(d, e, sample_eigs)
    assert np.max(np.abs(lam[sample_eigs] - ref)) <= 10 * n * EPS * nrm
    assert np.all(np.diff(lam) >= 0)
    qs = q_dev[:, torch.tensor(sample_cols, device=q_dev.device)]
    g = (q_dev.t() @ qs).cpu().numpy()
    g[sample_cols, np.arange(len(sample_cols))] -= 1.0
    assert np.max(np.abs(g)) <= 100 * n * EPS
    qs = qs.cpu().numpy()
    r = metrics.tri_matmul(d, e, qs) - qs * lam[sample_cols][None, :]
    # per-column share of the Frobenius residual bound
    assert np.linalg.norm(r) / np.sqrt(len(sample_cols) / n) <= 10 * n * EPS * nrm


def test_full_size_toeplitz_16384(api):
    n = 16384
    d, e = W.toeplitz_121(n)
    lam_t, q_t = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"))
    lam = lam_t.cpu().numpy()
    lref, _ = sturm.closed_form_121(n)
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * 4.0
    g = W.rng(5)
    cols = np.sort(g.choice(n, 64, replace=False))
    _sampled_checks(d, e, lam, q_t, cols, cols[:16])
    # closed-form sine vectors for well-separated sampled columns
    j = np.arange(1, n + 1)[:, None]
    k = (cols + 1)[None, :]
    qref = np.sqrt(2.0 / (n + 1)) * np.sin(j * k * np.pi / (n + 1)) * ((-1.0) ** (j - 1))
    qs = q_t[:, torch.tensor(cols, device="cuda")].cpu().numpy()
    # Davis-Kahan: a unit vector q with residual r = T q - mu q (mu its Rayleigh
    # quotient) makes an angle theta with the exact eigenvector of the eigenvalue
    # nearest mu with sin(theta) <= ||r|| / gap, gap = the distance from mu to the rest
    # of the spectrum (closed form); 1 - cos(theta) <= sin(theta)^2
    tq = metrics.tri_matmul(d, e, qs)
    mu = np.sum(qs * tq, axis=0) / np.sum(qs * qs, axis=0)
    res = np.linalg.norm(tq - qs * mu[None, :], axis=0) / np.linalg.norm(qs, axis=0)
    others = np.abs(lref[None, :] - mu[:, None])
    others[np.arange(len(cols)), cols] = np.inf
    gap = others.min(axis=1)
    dots = np.abs(np.sum(qs * qref, axis=0)) / np.linalg.norm(qs, axis=0)
    assert np.all(1.0 - dots <= (res / gap) ** 2 + 4 * n * EPS)


@pytest.mark.parametrize("gen", ["uniform", "graded"])
def test_full_size_32768(api, gen):
    n = 32768
    d, e = (W.uniform_tridiag if gen == "uniform" else W.graded_tridiag)(n, 0)
    lam_t, q_t = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"))
    lam = lam_t.cpu().numpy()
    g = W.rng(6)
    cols = np.sort(g.choice(n, 48, replace=False))
    _sampled_checks(d, e, lam, q_t, cols, cols[:12])
    del q_t
    torch.cuda.empty_cache()



def test_bounded_wait_times_out_with_status(api):
    """The split-precision product's bounded mbarrier wait, on a barrier nothing arrives
    on, with a 2 ms limit: it gives up, reports status bit 8 and returns; the context
    stays usable (a solve right after is correct)."""
    from paper_1612_07526_gb300 import _lib
    lib = _lib.load()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    rc = lib.tdc_diag_wait_timeout(2_000_000, api._vp(st), api._vp(out), api._stream(None))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) & 8 and int(out.item()) == 0
    assert lib.tdc_diag_wait_timeout(10, api._vp(st), api._vp(out), api._stream(None)) == -1
    d, e = W.uniform_tridiag(120, 4)
    lam, q = _solve(api, d, e)
    assert metrics.scaled_residual(d, e, lam, q) <= 10
