"""FP64 product tile shapes and their autotuner.  Every shape sums each output
element over k in the same order, so all twelve shapes must give bit-identical
eigenpairs; the solve itself is checked against the oracle's pins (Sturm-count
bisection for the eigenvalues, residual and orthogonality bounds).  The autotuner
must return valid shapes and leave the results unchanged, for single solves and
for batched plans replayed from a CUDA graph."""
import numpy as np
import pytest

import workloads as W
from oracle import metrics, sturm

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
        return W.uniform_tridiag(n, 5)
    if gen == "toeplitz":
        return W.toeplitz_121(n)
    return W.normal_tridiag(n, 6)


@pytest.mark.parametrize("gen,n", [("uniform", 700), ("toeplitz", 600), ("normal", 1000), ("uniform", 97)])
def test_tile_shapes_bit_identical(api, gen, n):
    d, e = _gen(gen, n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    ref = None
    for cfg in range(len(api._lib.TILE_SHAPES)):
        lam, q = api.syev_tridiag(dt, et, opts={"tile_cfg": cfg})
        if ref is None:
            ref = (lam.clone(), q.clone())
            lh, qh = lam.cpu().numpy(), q.cpu().numpy()
            nrm = metrics.tnorm(d, e)
            idx = np.unique(np.linspace(0, n - 1, 40).astype(int))
            assert np.max(np.abs(lh[idx] - sturm.bisection_eigvals(d, e, idx))) <= 10 * n * EPS * nrm
            assert metrics.orthogonality(qh) <= 100 * n * EPS
            assert metrics.scaled_residual(d, e, lh, qh) <= 10
        else:
            assert torch.equal(lam, ref[0]), f"eigenvalues differ for tile shape {cfg}"
            assert torch.equal(q, ref[1]), f"eigenvectors differ for tile shape {cfg}"


def test_autotune_single(api):
    n = 2048
    d, e = W.uniform_tridiag(n, 11)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    lam0, q0 = api.syev_tridiag(dt, et, opts={"tile_cfg": 2})
    shapes = api.autotune(dt, et)
    assert len(shapes) == 6                       # merge levels 64 .. 2048 above leaves of 32
    assert all(0 <= s < len(api._lib.TILE_SHAPES) for s in shapes)
    lam1, q1 = api.syev_tridiag(dt, et)          # tile_cfg = -1: the tuned shapes
    assert torch.equal(lam0, lam1) and torch.equal(q0, q1)


def test_autotune_batched_plan_graph(api):
    sizes, probs = W.batched_normal(64, seed=9, lo=32, hi=900)
    ds = [p[0] for p in probs]
    es = [p[1] for p in probs]
    plan = api.BatchedPlan(sizes)
    d_cat, e_cat = plan.pack(ds, es)
    lam, q = plan.outputs()
    shapes = plan.autotune(d_cat, e_cat, lam, q)
    assert len(shapes) >= 1 and all(0 <= s < len(api._lib.TILE_SHAPES) for s in shapes)
    lam_b, q_b, _, _ = api.syev_tridiag_batched(ds, es, opts={"tile_cfg": 0})
    lam2, q2 = plan.outputs()
    plan.capture(d_cat, e_cat, lam2, q2)
    lam2.zero_()
    q2.zero_()
    plan.replay()
    torch.cuda.synchronize()
    assert int(plan.status.abs().sum()) == 0
    assert torch.equal(lam2, lam_b) and torch.equal(q2, q_b)
