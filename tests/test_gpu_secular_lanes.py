"""Secular roots with 1, 2, 4, 8, 16 or 32 lanes per root (Section 1's secular equation).

Each mapping is forced through tdc_opts.secular_lanes and checked against the
oracle (the DC oracle's eigenpairs, Sturm-count bisection for the eigenvalues) on
problems that span one-lane-group warps, ragged last warps and the last root's
special interval.  The automatic choice (by the level's root count) only picks fewer
than 32 lanes on levels with tens of thousands of roots, so a large batch checks it:
a sample of problems against the oracle, residual and orthogonality of every problem
on the GPU, and results that differ from the forced warp-per-root run (so a grouped
mapping really ran)."""
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


def _gen(gen, n):
    if gen == "uniform":
        return W.uniform_tridiag(n, 21)
    if gen == "toeplitz":
        return W.toeplitz_121(n)
    return W.normal_tridiag(n, 22)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("gen,n", [("uniform", 700), ("normal", 1000), ("toeplitz", 600), ("normal", 45)])
def test_forced_lanes_match_oracle(api, lanes, gen, n):
    d, e = _gen(gen, n)
    lam, q = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"),
                              opts={"secular_lanes": lanes})
    lam, q = lam.cpu().numpy(), q.cpu().numpy()
    nrm = metrics.tnorm(d, e)
    lref, qref = dc.syev(d, e)
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * nrm
    idx = np.unique(np.linspace(0, n - 1, 40).astype(int))
    assert np.max(np.abs(lam[idx] - sturm.bisection_eigvals(d, e, idx))) <= 10 * n * EPS * nrm
    assert metrics.scaled_residual(d, e, lam, q) <= 10
    assert metrics.orthogonality(q) <= 100 * n * EPS
    err, _ = metrics.column_agreement(lref, qref, q, nrm, min_relgap=1e-4)
    assert err <= 1e-7


def test_bad_lanes_rejected(api):
    d, e = W.normal_tridiag(50, 1)
    with pytest.raises(ValueError):
        api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"),
                         opts={"secular_lanes": 3})


def test_auto_lanes_large_batch(api):
    # about 1500 problems of order 200..400: the lowest levels hold a few hundred
    # thousand roots, enough for the grouped mappings
    sizes, probs = W.batched_normal(1500, seed=17, lo=200, hi=400)
    ds = [p[0] for p in probs]
    es = [p[1] for p in probs]
    lam_a, q_a, sz, qoff = api.syev_tridiag_batched(ds, es)
    lam_w, _, _, _ = api.syev_tridiag_batched(ds, es, opts={"secular_lanes": 32})
    assert not torch.equal(lam_a, lam_w)
    off = np.concatenate([[0], np.cumsum(sizes)])
    scale = max(metrics.tnorm(d, e) for d, e in zip(ds, es))
    assert torch.max(torch.abs(lam_a - lam_w)).item() <= 10 * 400 * EPS * scale
    for p in (0, 1, 700, 1499):
        n = int(sizes[p])
        lref, qref = dc.syev(ds[p], es[p])
        lp = lam_a[off[p]:off[p] + n].cpu().numpy()
        qp = api.batched_block(q_a, sz, qoff, p).cpu().numpy()
        nrm = metrics.tnorm(ds[p], es[p])
        assert np.max(np.abs(lp - lref)) <= 10 * n * EPS * nrm
        err, _ = metrics.column_agreement(lref, qref, qp, nrm, min_relgap=1e-4)
        assert err <= 1e-7
    worst_res, worst_orth = 0.0, 0.0
    for p in range(len(sizes)):
        n = int(sizes[p])
        d = torch.tensor(ds[p], device="cuda")
        e = torch.tensor(es[p], device="cuda")
        qp = api.batched_block(q_a, sz, qoff, p)
        lp = lam_a[off[p]:off[p] + n]
        tq = d[:, None] * qp
        tq[:-1] += e[:, None] * qp[1:]
        tq[1:] += e[:, None] * qp[:-1]
        nrm = metrics.tnorm(ds[p], es[p])
        res = torch.linalg.matrix_norm(tq - qp * lp[None, :]).item() / (n * EPS * nrm)
        orth = torch.max(torch.abs(qp.t() @ qp - torch.eye(n, dtype=qp.dtype, device="cuda"))).item()
        worst_res = max(worst_res, res)
        worst_orth = max(worst_orth, orth / (n * EPS))
    assert worst_res <= 10
    assert worst_orth <= 100
