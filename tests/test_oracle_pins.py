"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, Sturm counts, brute-force characteristic polynomials, a LAPACK
library cross-check, invariants, special cases).  No GPU."""
import os

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import workloads as W
from oracle import backward, dc, hss, metrics, sturm

EPS = 2.0 ** -52
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return np.array([float(l) for l in f if l.strip() and not l.startswith("#")])


# --------------------------------------------------------------------------- full DC
def test_golden_toeplitz_n8():
    d, e = W.toeplitz_121(8)
    lam, q = dc.syev(d, e, leaf=2)                 # forces three merge levels
    ref = _golden("toeplitz121_n8.txt")
    assert np.max(np.abs(lam - ref)) <= 10 * 8 * EPS * 4.0


def test_golden_clement_n7():
    d, e = W.clement(7)
    lam, _ = dc.syev(d, e, leaf=2)
    ref = _golden("clement_n7.txt")
    nrm = metrics.tnorm(d, e)
    assert np.max(np.abs(lam - ref)) <= 10 * 7 * EPS * nrm
    assert np.allclose(sturm.clement_eigvals(7), ref)


@pytest.mark.parametrize("n", [64, 200, 1024])
def test_closed_form_121(n):
    d, e = W.toeplitz_121(n)
    lam, q = dc.syev(d, e)
    lref, qref = sturm.closed_form_121(n)
    nrm = 4.0
    assert np.max(np.abs(lam - lref)) <= 10 * n * EPS * nrm
    err, mask = metrics.column_agreement(lref, qref, q, nrm, min_relgap=1e-6)
    gap = np.min(np.diff(lref))
    assert err <= 100 * n * EPS * nrm / gap
    assert metrics.orthogonality(q) <= 100 * n * EPS
    assert metrics.scaled_residual(d, e, lam, q) <= 10


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (5, 2), (7, 3), (8, 4), (8, 5)])
def test_charpoly_bruteforce(n, seed):
    d, e = W.uniform_tridiag(n, seed)
    roots = sturm.charpoly_roots(d, e)
    assert roots.shape[0] == n
    lam, q = dc.syev(d, e, leaf=1 if n > 1 else 1)
    nrm = metrics.tnorm(d, e)
    assert np.max(np.abs(lam - roots)) <= 1e-9 * nrm      # root finding on the polynomial
    assert metrics.scaled_residual(d, e, lam, q) <= 10


def test_sturm_bisection_against_closed_form_and_charpoly():
    d, e = W.toeplitz_121(100)
    lref, _ = sturm.closed_form_121(100)
    assert np.max(np.abs(sturm.bisection_eigvals(d, e) - lref)) <= 10 * EPS * 4.0
    d, e = W.uniform_tridiag(7, 11)
    assert np.max(np.abs(sturm.bisection_eigvals(d, e) - sturm.charpoly_roots(d, e))) <= 1e-9


@pytest.mark.parametrize("gen,n", [("uniform", 300), ("normal", 257), ("graded", 300)])
def test_sturm_counts_and_invariants(gen, n):
    d, e = {"uniform": lambda: W.uniform_tridiag(n, 3),
            "normal": lambda: W.normal_tridiag(n, 4),
            "graded": lambda: W.graded_tridiag(n, 5)}[gen]()
    lam, q = dc.syev(d, e)
    nrm = metrics.tnorm(d, e)
    tol = 10 * n * EPS * nrm
    below = sturm.sturm_count(d, e, lam - tol)
    above = sturm.sturm_count(d, e, lam + tol)
    k = np.arange(n)
    assert np.all(below <= k) and np.all(above >= k + 1)
    assert np.max(np.abs(lam - sturm.bisection_eigvals(d, e))) <= tol
    assert metrics.scaled_residual(d, e, lam, q) <= 10
    assert metrics.orthogonality(q) <= 100 * n * EPS


def test_library_dstevd_crosscheck():
    n = 700
    d, e = W.uniform_tridiag(n, 9)
    lam, q = dc.syev(d, e)
    w, z, info = lapack.dstevd(d, e, compute_v=1)
    assert info == 0
    nrm = metrics.tnorm(d, e)
    assert np.max(np.abs(lam - w)) <= 10 * n * EPS * nrm
    err, _ = metrics.column_agreement(w, z, q, nrm, min_relgap=1e-4)
    assert err <= 1e-8


def test_sign_convention():
    d, e = W.uniform_tridiag(100, 1)
    _, q = dc.syev(d, e)
    idx = np.argmax(np.abs(q), axis=0)
    assert np.all(q[idx, np.arange(100)] > 0)


def test_jacobi_leaf():
    a = dc.tridiag_dense(*W.normal_tridiag(31, 2))
    w, v = dc.jacobi_eigh(a)
    assert np.max(np.abs(w - np.linalg.eigvalsh(a))) <= 50 * EPS * np.abs(a).sum(1).max()
    assert np.max(np.abs(v.T @ v - np.eye(31))) <= 1e-13
    assert np.linalg.norm(a @ v - v * w) <= 1e-13 * np.linalg.norm(a)
    w2, _ = dc.jacobi_eigh(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert np.allclose(w2, [-1.0, 3.0], atol=1e-15)


# --------------------------------------------------------------------------- merge pieces
def _secular_case(k, seed):
    g = W.rng(seed)
    d = np.sort(g.uniform(-1, 1, k))
    z = g.standard_normal(k)
    z /= np.linalg.norm(z)
    return d, z, float(g.uniform(0.1, 2.0))


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (17, 2), (200, 3)])
def test_secular_roots_against_dense(k, seed):
    d, z, rho = _secular_case(k, seed)
    o, tau = dc.secular_roots(d, z, rho)
    lam = d[o] + tau
    ev = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(z, z))
    assert np.max(np.abs(lam - ev)) <= 20 * k * EPS * (np.abs(d).max() + rho)
    # interlacing d_i < lambda_i < d_{i+1}, lambda_K <= d_K + rho
    assert np.all(lam > d) and np.all(lam[:-1] < d[1:]) and lam[-1] <= d[-1] + rho
    # the origin is the nearer pole for the inner roots; the last root is right of d_K
    assert np.all(np.abs(tau[:-1]) <= np.diff(d) / 2) and 0 < tau[-1] <= rho


def test_lowner_z_reproduces_spectrum():
    d, z, rho = _secular_case(150, 7)
    o, tau = dc.secular_roots(d, z, rho)
    zh = dc.lowner_z(d, z, rho, o, tau)
    assert np.all(np.sign(zh) == np.sign(z))
    assert np.max(np.abs(zh - z) / np.abs(z)) <= 1e-10       # accurate roots: zhat ~ z
    ev = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(zh, zh))
    assert np.max(np.abs(ev - (d[o] + tau))) <= 1e-13
    # a planted dropped factor is caught: leaving out the (lambda_K - d_j)/rho term
    lam_m_d = (d[o][:, None] - d[None, :]) + tau[:, None]
    bad = zh * zh * rho / lam_m_d[-1]
    assert np.max(np.abs(np.sqrt(bad) - np.abs(z))) > 1e-3


def test_rank_one_vectors_orthonormal_eigenvectors():
    d, z, rho = _secular_case(120, 8)
    o, tau = dc.secular_roots(d, z, rho)
    zh = dc.lowner_z(d, z, rho, o, tau)
    qh = dc.rank_one_vectors(d, zh, o, tau)
    lam = d[o] + tau
    a = np.diag(d) + rho * np.outer(zh, zh)
    assert np.max(np.abs(qh.T @ qh - np.eye(120))) <= 1e-13
    assert np.linalg.norm(a @ qh - qh * lam) <= 1e-13


def test_deflation_type1_exact_zero():
    """Columns whose coupling-row entry is exactly zero give z_j = 0: type-1 deflation,
    and (d_j, column) is an exact eigenpair of the merged matrix."""
    g = W.rng(3)
    n1, n2 = 20, 12
    Q = np.zeros((32, 32))
    Q[:n1 - 1, :n1 - 1] = W.random_orthogonal(n1 - 1, g)   # last row of Q1 is e_{n1}^T
    Q[n1 - 1, n1 - 1] = 1.0
    Q[n1:, n1:] = W.random_orthogonal(n2, g)
    D = np.concatenate([np.sort(g.uniform(-1, 1, n1)), np.sort(g.uniform(-1, 1, n2))])
    beta = -0.6
    lam, u, info = dc.merge(D, Q, n1, beta)
    defl_src = set(info["order"][info["deflated"]].tolist())
    assert set(range(n1 - 1)) <= defl_src
    assert info["K"] == 32 - len(defl_src)
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(32)
    v[n1 - 1] = 1.0
    v[n1] = -1.0
    a += abs(beta) * np.outer(v, v)
    for c in range(n1 - 1):
        x = Q[:, c]
        assert np.linalg.norm(a @ x - D[c] * x) <= 1e-14
    assert np.linalg.norm(a @ u - u * lam) <= 1e-13
    assert np.max(np.abs(np.linalg.eigvalsh(a) - lam)) <= 1e-14


def test_deflation_type2_equal_poles():
    g = W.rng(12)
    n1, n2 = 10, 10
    d1 = np.sort(g.uniform(-1, 1, n1))
    d2 = np.sort(g.uniform(-1, 1, n2))
    d2[4] = d1[6]                             # an exactly repeated pole across the halves
    D = np.concatenate([d1, d2])
    Q = np.zeros((20, 20))
    Q[:10, :10] = W.random_orthogonal(10, g)
    Q[10:, 10:] = W.random_orthogonal(10, g)
    lam, u, info = dc.merge(D, Q, n1, 0.7)
    assert len(info["rotations"]) >= 1
    assert info["K"] <= 19
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(20)
    v[9] = 1.0
    v[10] = 1.0
    a += 0.7 * np.outer(v, v)
    ev = np.linalg.eigvalsh(a)
    assert np.max(np.abs(lam - ev)) <= 1e-13
    assert np.linalg.norm(a @ u - u * lam) <= 1e-13
    assert np.max(np.abs(u.T @ u - np.eye(20))) <= 1e-13


@pytest.mark.parametrize("n1,n2,seed", [(16, 16, 0), (33, 40, 1), (100, 57, 2)])
@pytest.mark.parametrize("neg", [False, True])
def test_merge_against_dense(n1, n2, seed, neg):
    D, Q, beta = W.merge_problem(n1, n2, seed)
    beta = -abs(beta) if neg else abs(beta)
    lam, u, info = dc.merge(D, Q, n1, beta)
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n1 + n2)
    v[n1 - 1] = 1.0
    v[n1] = np.sign(beta)
    a += abs(beta) * np.outer(v, v)
    ev = np.linalg.eigvalsh(a)
    n = n1 + n2
    assert np.max(np.abs(lam - ev)) <= 10 * n * EPS * np.abs(a).sum(1).max()
    assert np.linalg.norm(a @ u - u * lam) <= 10 * n * EPS * np.linalg.norm(a)
    assert np.max(np.abs(u.T @ u - np.eye(n))) <= 100 * n * EPS


# --------------------------------------------------------------------------- HSS
def test_hss_example1_ranks():
    n = 1500
    for which, rmax in ((1, 4), (2, 200)):
        a = W.hss_example1(n, which)
        root, nodes = hss.rand_hss(a, W.gaussian((n, 250), 1), W.gaussian((n, 250), 2), 200, 1e-12)
        r = max(hss.hss_ranks(nodes))
        assert r <= rmax
        rec = hss.hss_to_dense(root)
        assert np.linalg.norm(a - rec) <= 1e-10 * np.linalg.norm(a)
        x = W.gaussian((7, n), 3)
        assert np.linalg.norm(hss.hss_left_multiply(x, root, nodes) - x @ a) <= 1e-10 * np.linalg.norm(x @ a)
    # matrix 1 is rank ~2 off the diagonal (Example 1)
    a = W.hss_example1(n, 1)
    root, nodes = hss.rand_hss(a, W.gaussian((n, 20), 4), W.gaussian((n, 20), 5), 200, 1e-12)
    assert max(hss.hss_ranks(nodes)) <= 3


def test_qhat_off_diagonal_low_rank():
    """Section 2.2 / Fig. 2: N = 1000, d_i = i/N, rho = 1, random unit z."""
    d, z, rho = W.rank_one_example(1000, 0)
    o, tau = dc.secular_roots(d, z, rho)
    zh = dc.lowner_z(d, z, rho, o, tau)
    qh = dc.rank_one_vectors(d, zh, o, tau)
    s = np.linalg.svd(qh[:500, 500:], compute_uv=False)
    assert np.sum(s > 1e-12 * s[0]) < 100
    root, nodes = hss.rand_hss(qh, W.gaussian((1000, 128), 1), W.gaussian((1000, 128), 2), 125, 1e-12)
    assert np.linalg.norm(qh - hss.hss_to_dense(root)) <= 1e-10 * np.linalg.norm(qh)


def test_splitmix64_published_value_and_gaussian_moments():
    # first output of SplitMix64 seeded with 0 (the generator's published reference value)
    assert int(hss.splitmix64(0, 0)) == 0xE220A8397B1DCDAF
    g = hss.gaussian_matrix(7, 1, 2000, 50)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.02
    assert not np.array_equal(g, hss.gaussian_matrix(7, 2, 2000, 50))


def test_merge_hss_matches_dense_merge_at_tolerance():
    """The HSS merge reproduces the dense merge to the compression tolerance; the
    merged matrix's residual and orthogonality stay at that level."""
    D, Q, beta = W.merge_problem(600, 600, 5)
    lam, u, info = dc.merge(D, Q, 600, beta)
    lam_h, u_h, info_h = dc.merge_hss(D, Q, 600, beta, leaf=128, rp=64, tol=1e-12, seed=0x5EED)
    assert np.array_equal(lam, lam_h)
    assert np.max(np.abs(u - u_h)) <= 1e-9
    assert max(info_h["hss_ranks"]) < 64
    assert np.max(np.abs(u_h.T @ u_h - np.eye(1200))) <= 1e-9


def test_interp_decomp_exact_low_rank():
    g = W.rng(3)
    a = g.standard_normal((60, 5)) @ g.standard_normal((5, 40))
    u, idx = hss.interp_decomp(a, 1e-12)
    assert u.shape[1] == 5
    assert np.allclose(u[idx], np.eye(5))
    assert np.linalg.norm(u @ a[idx] - a) <= 1e-10 * np.linalg.norm(a)


# --------------------------------------------------------------------------- backward
def _fd(f, x, direction, h=1e-6):
    return (f(x + h * direction) - f(x - h * direction)) / (2 * h)


def test_backward_finite_differences():
    n = 48
    d, e = W.normal_tridiag(n, 21)
    w = W.gaussian(n, 22)
    G = W.gaussian((n, 6), 23)
    lam, q = dc.dc_eig(d, e)
    gl, gq = backward.config_loss_grads(lam, q, w, G)
    gd, ge = backward.band_gradient(lam, q, gl, gq)

    def loss(x):
        l, qq = dc.dc_eig(x[:n], x[n:])
        return backward.config_loss(l, qq, w, G)

    x0 = np.concatenate([d, e])
    grad = np.concatenate([gd, ge])
    g = W.rng(24)
    for _ in range(4):
        u = g.standard_normal(2 * n - 1)
        assert abs(_fd(loss, x0, u) - grad @ u) <= 1e-6 * (1 + abs(grad @ u))


def test_backward_hellmann_feynman():
    n = 40
    d, e = W.normal_tridiag(n, 31)
    lam, q = dc.dc_eig(d, e)
    w = W.gaussian(n, 32)
    gd, ge = backward.band_gradient(lam, q, g_lam=w)
    assert np.allclose(gd, (q * q) @ w, atol=1e-13)
    assert np.allclose(ge, 2 * (q[:-1] * q[1:]) @ w, atol=1e-13)


# --------------------------------------------------------------------------- metrics
def test_tri_matmul_against_dense_product():
    """T Q for T = tridiag(e, d, e) equals the dense product; a band offset by one row
    or a transposed coupling would change entries of this non-symmetric Q."""
    d, e = W.uniform_tridiag(9, 21)
    q = W.rng(22).standard_normal((9, 4))
    t = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.allclose(metrics.tri_matmul(d, e, q), t @ q, rtol=0, atol=1e-15)
    d2, e2 = np.array([1.0, 2.0, 3.0]), np.array([10.0, 20.0])
    q2 = np.array([[1.0], [0.0], [0.0]])               # first column of T: (1, 10, 0)
    assert np.array_equal(metrics.tri_matmul(d2, e2, q2)[:, 0], [1.0, 10.0, 0.0])


def test_scaled_residual_values():
    """Zero for exact eigenpairs of a diagonal T; for a planted residual the value
    ||R||_F / (n eps ||T||_1) computed by hand."""
    d = np.array([3.0, -1.0, 2.0])
    e = np.zeros(2)
    lam = d.copy()
    q = np.eye(3)
    assert metrics.scaled_residual(d, e, lam, q) == 0.0
    lam_bad = lam + np.array([0.0, 2.0 ** -40, 0.0])   # residual column (0, -2^-40, 0), exact
    assert metrics.scaled_residual(d, e, lam_bad, q) == 2.0 ** -40 / (3 * EPS * 3.0)
    assert metrics.tnorm([1.0, -2.0, 0.5], [4.0, -1.0]) == 7.0     # max row sum |e|+|d|+|e|


def test_orthogonality_and_column_agreement_values():
    q = np.linalg.qr(W.rng(23).standard_normal((6, 6)))[0]
    assert metrics.orthogonality(q) <= 10 * EPS
    q2 = q.copy()
    q2[:, 1] *= 1.0 + 1e-9                             # ||q_1||^2 - 1 = 2e-9 + 1e-18
    assert np.isclose(metrics.orthogonality(q2), 2e-9, rtol=1e-6)
    lam = np.arange(6.0)
    flipped = q * np.array([1, -1, 1, -1, 1, 1])[None, :]
    err, mask = metrics.column_agreement(lam, q, flipped, 6.0)
    assert err <= 1e-15 and mask.all()                 # signs are free
    bent = q.copy()
    bent[:, 2] += 1e-7 * q[:, 3]
    err, _ = metrics.column_agreement(lam, q, bent, 6.0)
    assert np.isclose(err, 1e-7, rtol=1e-6)
    lam_close = np.array([0.0, 1.0, 1.0 + 1e-12, 3.0, 4.0, 5.0])
    _, mask = metrics.column_agreement(lam_close, q, q, 6.0, min_relgap=1e-6)
    assert list(mask) == [True, False, False, True, True, True]


# --------------------------------------------------------------------------- extended precision
def test_extended_roots_against_exact_characteristic_polynomial():
    """The exact roots (rational bisection) against the eigenvalues of D + rho z z^T
    taken by sympy from its characteristic polynomial with rational entries, to 60
    digits: tau differs from the polynomial's root by less than 2^-100 |tau|."""
    sympy = pytest.importorskip("sympy")
    from oracle import extended
    g = W.rng(30)
    for k in (3, 5, 6):
        d = np.sort(g.uniform(-1, 1, k))
        z = g.standard_normal(k)
        z /= np.linalg.norm(z)
        rho = 0.75
        org, tau = dc.secular_roots(d, z, rho)
        hi, lo, ex = extended.exact_roots(d, z, rho, org, tau)
        ds = [sympy.Rational(float(x)) for x in d]
        zs = [sympy.Rational(float(x)) for x in z]
        a = sympy.diag(*ds) + sympy.Rational(0.75) * sympy.Matrix(zs) * sympy.Matrix(zs).T
        lam = sympy.symbols("lam")
        roots = sorted(sympy.Poly(a.charpoly(lam).as_expr(), lam).nroots(n=60, maxsteps=200))
        for i in range(k):
            t_ref = roots[i] - ds[int(org[i])]
            t_ex = sympy.Rational(ex[i].numerator, ex[i].denominator)
            assert abs(t_ex - t_ref) <= abs(t_ref) * sympy.Rational(1, 2 ** 100)
            assert abs(hi[i] + lo[i] - float(t_ref)) <= 4 * np.spacing(abs(float(t_ref)))


def test_extended_vectors_orthonormal_and_reconstruct():
    """Eigenvectors from exact roots and the original z: orthonormal to a few units of
    eps and D + rho z z^T = U Lambda U^T, also for clustered poles and graded z."""
    from oracle import extended
    g = W.rng(31)
    for case in range(3):
        k = 24
        d = np.sort(g.uniform(-1, 1, k))
        if case >= 1:
            d[5] = d[4] + 1e-10
            d[13] = d[12] + 3e-12
            d = np.sort(d)
        z = g.standard_normal(k) * (10.0 ** g.uniform(-4, 0, k) if case == 2 else 1.0)
        z /= np.linalg.norm(z)
        rho = 1.3
        df = dc.deflate(d, z, rho)
        d2, z2 = df["d"][df["kept"]], df["z"][df["kept"]]
        org, tau = dc.secular_roots(d2, z2, rho)
        hi, lo, ex = extended.exact_roots(d2, z2, rho, org, tau)
        u = extended.extended_vectors(d2, z2, org, ex)
        kk = len(d2)
        assert np.max(np.abs(u.T @ u - np.eye(kk))) <= 4 * kk * EPS
        lam = d2[org] + hi
        a = np.diag(d2) + rho * np.outer(z2, z2)
        assert np.linalg.norm(u @ np.diag(lam) @ u.T - a) <= 10 * kk * EPS * np.linalg.norm(a)


def test_extended_merge_against_dense_merge():
    """The extended-precision merge gives the same eigenpairs as the Loewner merge
    (eigenvectors where the gaps allow) and satisfies the merge contract."""
    from oracle import extended
    D, Q, beta = W.merge_problem(30, 26, 32)
    lam, u, info = extended.merge_extended(D, Q, 30, beta)
    lam_l, u_l, _ = dc.merge(D, Q, 30, beta)
    n = len(D)
    assert np.array_equal(lam, lam_l)
    a = Q @ np.diag(D) @ Q.T
    v = np.zeros(n)
    v[29] = 1.0
    v[30] = np.sign(beta)
    a += abs(beta) * np.outer(v, v)
    assert np.linalg.norm(a @ u - u * lam) <= 10 * n * EPS * np.linalg.norm(a)
    assert np.max(np.abs(u.T @ u - np.eye(n))) <= 100 * n * EPS
    err, _ = metrics.column_agreement(lam_l, u_l, u, np.abs(a).sum(1).max(), min_relgap=1e-6)
    assert err <= 1e-12
