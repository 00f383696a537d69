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
