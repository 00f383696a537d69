"""Batched plans: tdc_batched_plan_execute matches tdc_syev_tridiag_batched, and its
replay from a captured CUDA graph gives the same results (every problem checked
against the oracle for a sample, residual and orthogonality for all)."""
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


@pytest.mark.parametrize("path", [0, 1])
def test_plan_execute_and_graph_replay(api, path):
    sizes, probs = W.batched_normal(96, seed=3, lo=32, hi=1200)
    ds = [p[0] for p in probs]
    es = [p[1] for p in probs]
    plan = api.BatchedPlan(sizes, opts={"path": path})
    d_cat, e_cat = plan.pack(ds, es)
    lam1, q1 = plan.outputs()
    plan.execute(d_cat, e_cat, lam1, q1)
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    lam_b, q_b, _, _ = api.syev_tridiag_batched(ds, es, opts={"path": path})
    assert torch.equal(lam1, lam_b) and torch.equal(q1, q_b)
    lam2, q2 = plan.outputs()
    plan.capture(d_cat, e_cat, lam2, q2)
    lam2.zero_()
    q2.zero_()
    plan.replay()
    torch.cuda.synchronize()
    assert torch.equal(lam2, lam1) and torch.equal(q2, q1)
    lam = lam1.cpu().numpy()
    for p, n in enumerate(sizes):
        o = plan.off[p]
        lp = lam[o:o + n]
        qp = api.batched_block(q1, sizes, plan.qoff, p).cpu().numpy()
        assert metrics.scaled_residual(ds[p], es[p], lp, qp) <= 10
        assert metrics.orthogonality(qp) <= 100 * n * EPS
        if p % 16 == 0:
            lref, _ = dc.syev(ds[p], es[p])
            assert np.max(np.abs(lp - lref)) <= 10 * n * EPS * metrics.tnorm(ds[p], es[p])


@pytest.mark.parametrize("gen,n", [("uniform", 3000), ("toeplitz", 2500)])
def test_single_problem_plan_matches_direct(api, gen, n):
    """The one-problem batched plan replayed from a CUDA graph (the bench's timed step)
    gives the direct solve's eigenpairs bit for bit."""
    d, e = W.uniform_tridiag(n, 13) if gen == "uniform" else W.toeplitz_121(n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    lam_d, q_d = api.syev_tridiag(dt, et)
    plan = api.BatchedPlan([n])
    e_cat = torch.zeros(n, dtype=torch.float64, device="cuda")
    e_cat[:n - 1] = et
    lam, q = plan.outputs()
    plan.capture(dt, e_cat, lam, q)
    lam.zero_()
    q.zero_()
    plan.replay()
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    assert torch.equal(lam, lam_d)
    assert torch.equal(q.view(n, n).t(), q_d)
