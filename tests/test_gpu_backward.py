"""The hand-written backward (band-only adjoint of the eigendecomposition) against the
oracle's dense FP64 reference gradient, finite differences through the GPU forward,
and the Hellmann-Feynman special case.  Loss of the differentiable configuration:
sum_i w_i lambda_i + ||Q[:, :m]^T G||_F^2."""
import numpy as np
import pytest

import workloads as W
from oracle import backward

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _loss_torch(lam, q, w, G):
    m = G.shape[1]
    return (w * lam).sum() + ((q[:, :m].t() @ G) ** 2).sum()


@pytest.mark.parametrize("n,m", [(200, 8), (1024, 64)])
def test_backward_matches_dense_reference(api, n, m):
    d, e = W.normal_tridiag(n, 40 + n)
    w = W.gaussian(n, 41)
    G = W.gaussian((n, m), 42)
    dt = torch.tensor(d, device="cuda", requires_grad=True)
    et = torch.tensor(e, device="cuda", requires_grad=True)
    wt, Gt = torch.tensor(w, device="cuda"), torch.tensor(G, device="cuda")
    lam, q = api.eigh_tridiag(dt, et)
    _loss_torch(lam, q, wt, Gt).backward()
    gd, ge = dt.grad.cpu().numpy(), et.grad.cpu().numpy()
    lam_n, q_n = lam.detach().cpu().numpy(), q.detach().cpu().numpy()
    gl, gq = backward.config_loss_grads(lam_n, q_n, w, G)
    rd, re = backward.band_gradient(lam_n, q_n, gl, gq)
    scale = max(np.abs(rd).max(), np.abs(re).max())
    assert np.max(np.abs(gd - rd)) <= 1e-9 * scale
    assert np.max(np.abs(ge - re)) <= 1e-9 * scale


def test_backward_finite_differences(api):
    n, m = 300, 16
    d, e = W.normal_tridiag(n, 50)
    w = W.gaussian(n, 51)
    G = W.gaussian((n, m), 52)
    wt, Gt = torch.tensor(w, device="cuda"), torch.tensor(G, device="cuda")
    dt = torch.tensor(d, device="cuda", requires_grad=True)
    et = torch.tensor(e, device="cuda", requires_grad=True)
    lam, q = api.eigh_tridiag(dt, et)
    _loss_torch(lam, q, wt, Gt).backward()
    grad = np.concatenate([dt.grad.cpu().numpy(), et.grad.cpu().numpy()])

    def loss(x):
        l, qq = api.syev_tridiag(torch.tensor(x[:n], device="cuda"), torch.tensor(x[n:], device="cuda"))
        return float(_loss_torch(l, qq, wt, Gt))

    x0 = np.concatenate([d, e])
    g = W.rng(53)
    h = 1e-6
    for _ in range(6):
        u = g.standard_normal(2 * n - 1)
        u /= np.linalg.norm(u)
        fd = (loss(x0 + h * u) - loss(x0 - h * u)) / (2 * h)
        assert abs(fd - grad @ u) <= 1e-5 * (1.0 + abs(grad @ u))


def test_backward_hellmann_feynman(api):
    n = 512
    d, e = W.normal_tridiag(n, 60)
    w = W.gaussian(n, 61)
    lam, q = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"))
    gd, ge = api.syev_backward(lam, q, g_lam=torch.tensor(w, device="cuda"))
    qn = q.cpu().numpy()
    assert np.allclose(gd.cpu().numpy(), (qn * qn) @ w, atol=1e-12, rtol=0)
    assert np.allclose(ge.cpu().numpy(), 2 * (qn[:-1] * qn[1:]) @ w, atol=1e-12, rtol=0)


def test_backward_config_size_finite_differences(api):
    """n = 4096, G 4096 x 64: unit random directions by central differences (the step
    stays far below the eigenvalue gaps), and the dense FP64 reference gradient."""
    n, m = 4096, 64
    d, e = W.normal_tridiag(n, 70)
    w = W.gaussian(n, 71)
    G = W.gaussian((n, m), 72)
    wt, Gt = torch.tensor(w, device="cuda"), torch.tensor(G, device="cuda")
    dt = torch.tensor(d, device="cuda", requires_grad=True)
    et = torch.tensor(e, device="cuda", requires_grad=True)
    lam, q = api.eigh_tridiag(dt, et)
    _loss_torch(lam, q, wt, Gt).backward()
    grad = np.concatenate([dt.grad.cpu().numpy(), et.grad.cpu().numpy()])

    def loss(x):
        l, qq = api.syev_tridiag(torch.tensor(x[:n], device="cuda"), torch.tensor(x[n:], device="cuda"))
        return float(_loss_torch(l, qq, wt, Gt))

    x0 = np.concatenate([d, e])
    g = W.rng(73)
    h = 1e-6
    for _ in range(2):
        u = g.standard_normal(2 * n - 1)
        u /= np.linalg.norm(u)
        fd = (loss(x0 + h * u) - loss(x0 - h * u)) / (2 * h)
        assert abs(fd - grad @ u) <= 1e-5 * (1.0 + abs(grad @ u))
    lam_n, q_n = lam.detach().cpu().numpy(), q.detach().cpu().numpy()
    gl, gq = backward.config_loss_grads(lam_n, q_n, w, G)
    rd, re = backward.band_gradient(lam_n, q_n, gl, gq)
    scale = max(np.abs(rd).max(), np.abs(re).max())
    assert np.max(np.abs(grad[:n] - rd)) <= 1e-9 * scale
    assert np.max(np.abs(grad[n:] - re)) <= 1e-9 * scale
    # the same gradient with the products on the split-precision path (7 slices)
    gd_s, ge_s = api.syev_backward(lam.detach(), q.detach(), torch.tensor(gl, device="cuda"),
                                   torch.tensor(gq, device="cuda"), opts={"path": 1})
    assert np.max(np.abs(gd_s.cpu().numpy() - rd)) <= 1e-9 * scale
    assert np.max(np.abs(ge_s.cpu().numpy() - re)) <= 1e-9 * scale


def _batched_case(api, sizes, m, seed):
    """A batch solved by the batched plan, the configuration's loss per problem
    (w_p, G_p with m columns, m <= n_p), its (lambda_bar, Qbar) in the batch packing."""
    ds, es, ws, Gs = [], [], [], []
    for k, n in enumerate(sizes):
        d, e = W.normal_tridiag(int(n), seed + 10 * k)
        ds.append(d)
        es.append(e)
        ws.append(W.gaussian(int(n), seed + 10 * k + 1))
        Gs.append(W.gaussian((int(n), min(m, int(n))), seed + 10 * k + 2))
    lam, q, sz, qoff = api.syev_tridiag_batched(ds, es)
    gl_cat = torch.tensor(np.concatenate(ws), device="cuda")
    gq_cat = torch.zeros_like(q)
    for p, n in enumerate(sizes):
        qp = api.batched_block(q, sz, qoff, p)
        Gp = torch.tensor(Gs[p], device="cuda")
        mm = Gp.shape[1]
        blk = gq_cat[int(qoff[p]):int(qoff[p]) + int(n) * int(n)].view(int(n), int(n)).t()
        blk[:, :mm] = 2.0 * Gp @ (Gp.t() @ qp[:, :mm])
    return ds, es, ws, Gs, lam, q, sz, qoff, gl_cat, gq_cat


@pytest.mark.parametrize("sizes,m", [([1, 2, 33, 200, 64, 300, 513], 16), ([512] * 4, 64)])
def test_backward_batched_matches_single_and_reference(api, sizes, m):
    """The batched backward equals the single-problem entry bit for bit (same kernels,
    same summation order per problem) and the dense FP64 reference gradient."""
    ds, es, ws, Gs, lam, q, sz, qoff, gl_cat, gq_cat = _batched_case(api, sizes, m, 80)
    gd, ge = api.syev_backward_batched(sz, lam, q, gl_cat, gq_cat, max_cols=m)
    off = 0
    for p, n in enumerate(sizes):
        n = int(n)
        lam_p = lam[off:off + n]
        q_p = api.batched_block(q, sz, qoff, p)
        gq_p = gq_cat[int(qoff[p]):int(qoff[p]) + n * n].view(n, n).t()
        gd1, ge1 = api.syev_backward(lam_p.contiguous(), q_p, gl_cat[off:off + n].contiguous(), gq_p)
        assert torch.equal(gd[off:off + n], gd1)
        assert torch.equal(ge[off:off + n - 1], ge1)
        lam_n, q_n = lam_p.cpu().numpy(), q_p.cpu().numpy()
        rd, re = backward.band_gradient(lam_n, q_n, ws[p], gq_p.cpu().numpy())
        scale = max(np.abs(rd).max(), np.abs(re).max() if n > 1 else 0.0)
        assert np.max(np.abs(gd[off:off + n].cpu().numpy() - rd)) <= 1e-9 * scale
        if n > 1:
            assert np.max(np.abs(ge[off:off + n - 1].cpu().numpy() - re)) <= 1e-9 * scale
        off += n


def test_backward_batched_lambda_only_and_workspace_limit(api):
    """Qbar absent: the Hellmann-Feynman gradient per problem; a workspace sized for
    fewer nonzero columns than Qbar has is reported (3), not overrun."""
    import ctypes
    from paper_1612_07526_gb300 import _lib
    sizes = [40, 100, 7]
    ds, es, ws, Gs, lam, q, sz, qoff, gl_cat, gq_cat = _batched_case(api, sizes, 8, 90)
    gd, ge = api.syev_backward_batched(sz, lam, q, gl_cat, None)
    off = 0
    for p, n in enumerate(sizes):
        qn = api.batched_block(q, sz, qoff, p).cpu().numpy()
        assert np.allclose(gd[off:off + n].cpu().numpy(), (qn * qn) @ ws[p], atol=1e-12, rtol=0)
        assert np.allclose(ge[off:off + n - 1].cpu().numpy(), 2 * (qn[:-1] * qn[1:]) @ ws[p], atol=1e-12, rtol=0)
        off += n
    lib = _lib.load()
    szc = np.ascontiguousarray(sz, dtype=np.int64)
    sp = szc.ctypes.data_as(ctypes.c_void_p)
    nb = lib.tdc_backward_batched_workspace_bytes(len(sizes), sp, 2, None)      # room for 2 columns each
    wsb = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = torch.empty(int(szc.sum()), dtype=torch.float64, device="cuda")
    rc = lib.tdc_syev_tridiag_backward_batched(len(sizes), sp, api._vp(lam), api._vp(q), api._vp(gl_cat),
                                               api._vp(gq_cat), api._vp(out), api._vp(out.clone()), None,
                                               api._vp(wsb), nb, None, api._stream(None))
    assert rc == 3


@pytest.mark.parametrize("n,m", [(200, 8), (1024, 64), (1000, 37)])
def test_backward_split_products(api, n, m):
    """The backward with its two products on the split-precision tensor-core path
    (opts path 1, 7 slices): within 1e-10 of the FP64 backward (the products' error of
    about 2^-56 relative to their row and column scales, times the eigenvector term's
    1/gap amplification, below 1e4 at these sizes) and within the dense reference's
    bound; ragged sizes exercise partial tiles in rows, columns and k."""
    d, e = W.normal_tridiag(n, 140 + n)
    w = W.gaussian(n, 141)
    G = W.gaussian((n, m), 142)
    lam, q = api.syev_tridiag(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"))
    lam_n, q_n = lam.cpu().numpy(), q.cpu().numpy()
    gl, gq = backward.config_loss_grads(lam_n, q_n, w, G)
    glt, gqt = torch.tensor(gl, device="cuda"), torch.tensor(gq, device="cuda")
    gd0, ge0 = api.syev_backward(lam, q, glt, gqt)
    gd1, ge1 = api.syev_backward(lam, q, glt, gqt, opts={"path": 1})
    rd, re = backward.band_gradient(lam_n, q_n, gl, gq)
    scale = max(np.abs(rd).max(), np.abs(re).max())
    assert torch.max(torch.abs(gd1 - gd0)).item() <= 1e-10 * scale
    assert torch.max(torch.abs(ge1 - ge0)).item() <= 1e-10 * scale
    assert np.max(np.abs(gd1.cpu().numpy() - rd)) <= 1e-9 * scale
    assert np.max(np.abs(ge1.cpu().numpy() - re)) <= 1e-9 * scale


def test_backward_batched_split_products(api):
    """The batched backward on the split path: each problem equals the single-problem
    split backward bit for bit (its slices and tiles do not depend on the batch) and
    stays within 1e-10 of the FP64 batched backward."""
    sizes, m = [1, 2, 33, 200, 64, 300, 513], 16
    ds, es, ws, Gs, lam, q, sz, qoff, gl_cat, gq_cat = _batched_case(api, sizes, m, 180)
    gd0, ge0 = api.syev_backward_batched(sz, lam, q, gl_cat, gq_cat, max_cols=m)
    gd, ge = api.syev_backward_batched(sz, lam, q, gl_cat, gq_cat, max_cols=m, opts={"path": 1})
    scale = max(torch.max(torch.abs(gd0)).item(), torch.max(torch.abs(ge0)).item())
    assert torch.max(torch.abs(gd - gd0)).item() <= 1e-10 * scale
    assert torch.max(torch.abs(ge - ge0)).item() <= 1e-10 * scale
    off = 0
    for p, n in enumerate(sizes):
        n = int(n)
        q_p = api.batched_block(q, sz, qoff, p)
        gq_p = gq_cat[int(qoff[p]):int(qoff[p]) + n * n].view(n, n).t()
        gd1, ge1 = api.syev_backward(lam[off:off + n].contiguous(), q_p, gl_cat[off:off + n].contiguous(), gq_p,
                                     opts={"path": 1})
        assert torch.equal(gd[off:off + n], gd1)
        assert torch.equal(ge[off:off + n - 1], ge1)
        off += n
