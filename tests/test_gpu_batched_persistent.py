"""The persistent batched solve (tdc_batched_plan_execute_persistent): one kernel launch in
which every CTA takes whole problems from a work queue and runs all their phases.
Checked through the C ABI against the CPU oracle problem by problem, against the
level-by-level execute of the same plan (same arithmetic except the lanes per secular
root, so eigenvalues within the contract and eigenvectors where the gaps allow), and
as a captured CUDA graph (bit for bit: each problem is solved by one CTA with a fixed
order of operations, whichever CTA takes it)."""
import numpy as np
import pytest

import workloads as W
from oracle import dc, metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _problems(sizes, seed):
    ds, es = [], []
    for k, n in enumerate(sizes):
        d, e = W.normal_tridiag(int(n), seed + k)
        ds.append(d)
        es.append(e)
    return ds, es


def _check(ds, es, sizes, lam, q, plan, sample=None):
    off = 0
    for p, n in enumerate(sizes):
        n = int(n)
        if sample is None or p in sample:
            lp = lam[off:off + n].cpu().numpy()
            qp = q[int(plan.qoff[p]):int(plan.qoff[p]) + n * n].view(n, n).t().cpu().numpy()
            lref, qref = dc.syev(ds[p], es[p])
            nrm = metrics.tnorm(ds[p], es[p])
            assert np.all(np.diff(lp) >= 0)
            assert np.max(np.abs(lp - lref)) <= 10 * n * EPS * nrm
            assert metrics.scaled_residual(ds[p], es[p], lp, qp) <= 10
            assert metrics.orthogonality(qp) <= 100 * n * EPS
            err, _ = metrics.column_agreement(lref, qref, qp, nrm, min_relgap=1e-4)
            assert err <= 1e-7
            idx = np.argmax(np.abs(qp), axis=0)
            assert np.all(qp[idx, np.arange(n)] > 0)
        off += n


@pytest.mark.parametrize("leaf", [32, 8, 1])
def test_persistent_ragged_against_oracle(api, leaf):
    sizes = [1, 2, 3, 31, 32, 33, 64, 100, 257, 513, 1000, 2048]
    ds, es = _problems(sizes, 700)
    plan = api.BatchedPlan(sizes, opts={"path": 0, "leaf": leaf})
    d_cat, e_cat = plan.pack(ds, es)
    lam, q = plan.outputs()
    plan.execute_persistent(d_cat, e_cat, lam, q)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    _check(ds, es, sizes, lam, q, plan)


def test_persistent_agrees_with_level_execute_and_replays(api):
    sizes, probs = W.batched_normal(300, seed=3)
    ds = [p[0] for p in probs]
    es = [p[1] for p in probs]
    plan = api.BatchedPlan(sizes, opts={"path": 0})
    d_cat, e_cat = plan.pack(ds, es)
    lam_l, q_l = plan.outputs()
    plan.execute(d_cat, e_cat, lam_l, q_l)
    lam_p, q_p = plan.outputs()
    plan.execute_persistent(d_cat, e_cat, lam_p, q_p)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    off = 0
    for p, n in enumerate(sizes):
        n = int(n)
        nrm = metrics.tnorm(ds[p], es[p])
        a = lam_l[off:off + n].cpu().numpy()
        b = lam_p[off:off + n].cpu().numpy()
        assert np.max(np.abs(a - b)) <= 10 * n * EPS * nrm
        if p % 25 == 0:
            qa = q_l[int(plan.qoff[p]):int(plan.qoff[p]) + n * n].view(n, n).t().cpu().numpy()
            qb = q_p[int(plan.qoff[p]):int(plan.qoff[p]) + n * n].view(n, n).t().cpu().numpy()
            err, _ = metrics.column_agreement(a, qa, qb, nrm, min_relgap=1e-4)
            assert err <= 1e-7
            assert metrics.scaled_residual(ds[p], es[p], b, qb) <= 10
            assert metrics.orthogonality(qb) <= 100 * n * EPS
        off += n
    _check(ds, es, sizes, lam_p, q_p, plan, sample={0, 1, 2, 150, 299})
    # the persistent execute captured in a CUDA graph and replayed: bit for bit
    lam_g, q_g = plan.outputs()
    plan.capture(d_cat, e_cat, lam_g, q_g, persistent=True)
    lam_g.zero_()
    q_g.zero_()
    plan.replay()
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    assert torch.equal(lam_g, lam_p) and torch.equal(q_g, q_p)


def test_persistent_extended_precision(api):
    sizes = [40, 300, 700, 1]
    ds, es = _problems(sizes, 900)
    plan = api.BatchedPlan(sizes, opts={"path": 0, "eigvec": 1})
    d_cat, e_cat = plan.pack(ds, es)
    lam, q = plan.outputs()
    plan.execute_persistent(d_cat, e_cat, lam, q)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    _check(ds, es, sizes, lam, q, plan)


def test_persistent_rejects_other_product_paths(api):
    from paper_1612_07526_gb300 import _lib
    plan = api.BatchedPlan([64, 64], opts={"path": 1})
    d_cat, e_cat = plan.pack(*_problems([64, 64], 5))
    lam, q = plan.outputs()
    rc = _lib.load().tdc_batched_plan_execute_persistent(plan.handle, api._vp(d_cat), api._vp(e_cat), api._vp(lam),
                                                         api._vp(q), api._vp(plan.status), api._stream(None))
    assert rc == -1
