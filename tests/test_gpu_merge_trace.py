"""Per-merge parity of the intermediate values (tdc_merge_inspect through the C ABI)
with the oracle's steps, one by one:

* the sort of D and z (Eq. 3), deflation (Eq. 5): the permutation, the type-1 and
  type-2 decisions, the rotations (j, k, c, s) in the order applied, the updated d and
  z, the kept and deflated sets and the Gu column groups: bit for bit (both sides
  round every operation of these steps the same way);
* the secular roots (Section 1): the origin bit for bit, except where the oracle's
  f at the interval's midpoint is within its own rounding-error bound of zero (then
  either origin is right and the two lambda must agree instead); tau within the
  bound that first-order perturbation of the monotone secular function gives (below);
* the Loewner z (Remark 1) and the column norms of Qhat within the bound that the
  roots' differences propagate to (below).

Bounds.  On the root's interval f(tau) = 1 + rho sum_j z_j^2 / (delta_j - tau) is
increasing with f' = rho sum_j z_j^2 / (delta_j - tau)^2.  A computed sum of K terms
carries an error of at most E = (K + 2) eps (1 + rho sum_j z_j^2 / |delta_j - tau|)
(each term: one subtraction, one division, one multiplication; K - 1 additions).
Each solver returns a tau where its computed f is within its E of zero or changes
sign, so |tau - tau*| <= E / f' + 1 ulp for each, and the two differ by at most
2 E / f' + 2 ulp (f' and E evaluated at the oracle's tau; a factor 2 covers the
variation of f' between the two).  zhat_j^2 is a product over i of (lambda_i - d_j)
and fixed differences, so its relative change is sum_i |dtau_i| / |lambda_i - d_j|
plus 4 K eps of rounding; zhat_j takes half of that.  The unscaled column i of Qhat
has entries zhat_j / (d_j - lambda_i), so 1 / ||.|| moves by at most
max_j (rel(zhat_j) + |dtau_i| / |d_j - lambda_i|) plus K eps of rounding."""
import numpy as np
import pytest

import workloads as W
from oracle import dc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import api as a
    return a


def _fortran(q):
    return torch.tensor(np.asfortranarray(q), device="cuda").t().contiguous().t()


def structured_merge(n1, n2, a, b, seed):
    """A merge whose z has exactly a + b nonzero entries: Q1 = diag(I, R_a) and
    Q2 = diag(R_b, I) with random orthogonal R, so the last row of Q1 and the first row
    of Q2 are nonzero only in those columns; the other n - a - b entries of z are
    exactly zero (type-1 deflation), so K = a + b when no d_j coincide."""
    g = W.rng(seed)
    Q = np.zeros((n1 + n2, n1 + n2))
    Q[:n1, :n1] = np.eye(n1)
    Q[n1 - a:n1, n1 - a:n1] = W.random_orthogonal(a, g)
    Q[n1:, n1:] = np.eye(n2)
    Q[n1:n1 + b, n1:n1 + b] = W.random_orthogonal(b, g)
    D = np.concatenate([np.sort(g.uniform(-1, 1, n1)), np.sort(g.uniform(-1, 1, n2))])
    beta = float(g.uniform(0.1, 1.0)) * (-1.0 if seed % 2 else 1.0)
    return D, Q, beta


def tridiag_level_merge(n, seed):
    """The top merge of tridiag(e, d, e) with d, e ~ U[-1, 1]: the children solved by
    the oracle, then torn as in Eq. (2) (the heavy-deflation case of the benchmark)."""
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


def equal_pole_merge():
    g = W.rng(12)
    d1 = np.sort(g.uniform(-1, 1, 10))
    d2 = np.sort(g.uniform(-1, 1, 10))
    d2[4] = d1[6]
    d2[7] = d1[8]
    d2 = np.sort(d2)
    Q = np.zeros((20, 20))
    Q[:10, :10] = W.random_orthogonal(10, g)
    Q[10:, 10:] = W.random_orthogonal(10, g)
    return np.concatenate([d1, d2]), Q, 10, 0.7


def _secular_terms(dbar, zbar, rho, origin, tau):
    """Per root i (oracle's origin and tau): f', the evaluation error bound E of the
    module docstring, and lambda_i - d_j for all j (rows i)."""
    base = dbar[origin][:, None] - dbar[None, :]                 # d_org(i) - d_j
    lam_m_d = base + tau[:, None]                                # lambda_i - d_j
    z2 = zbar * zbar
    t = z2[None, :] / lam_m_d                                    # z_j^2 / (lambda_i - d_j)
    fprime = rho * np.sum(t / lam_m_d, axis=1)
    kk = len(dbar)
    E = (kk + 2) * EPS * (1.0 + rho * np.sum(np.abs(t), axis=1))
    return fprime, E, lam_m_d


def _check_trace(D, Q, n1, beta, tr):
    n = len(D)
    lam_r, u_r, info = dc.merge(D, Q, n1, beta)
    z, rho = dc.merge_z(Q, n1, beta)
    order = info["order"]
    df = dc.deflate(D[order], z[order], rho)
    K = info["K"]
    cnt = tr["counts"]
    # deflation: bit for bit
    assert int(cnt[0]) == K
    assert int(cnt[1]) == len(info["deflated"])
    assert int(cnt[2]) == len(info["rotations"])
    assert int(cnt[5]) == int(np.count_nonzero(df["type1"]))
    half = info["half"]
    kept = info["kept"]
    assert int(cnt[3]) == int(np.count_nonzero(half[kept] == 1))
    assert int(cnt[4]) == int(np.count_nonzero(half[kept] == 3))
    assert np.array_equal(tr["perm"], order)
    assert np.array_equal(tr["d_sorted"], df["d"])
    assert np.array_equal(tr["z_sorted"], df["z"])
    assert np.array_equal(tr["kept"], kept)
    assert np.array_equal(tr["deflated"], info["deflated"])
    if info["rotations"]:
        rj, rk, rc, rs = (np.array(x) for x in zip(*info["rotations"]))
        assert np.array_equal(tr["rot_j"], rj) and np.array_equal(tr["rot_k"], rk)
        assert np.array_equal(tr["rot_c"], rc) and np.array_equal(tr["rot_s"], rs)
    assert np.array_equal(tr["dbar"], info["dbar"])
    assert np.array_equal(tr["zbar"], info["zbar"])
    if K == 0:
        return {}
    dbar, zbar = info["dbar"], info["zbar"]
    org_o, tau_o = info["origin"], info["tau"]
    org_g, tau_g = tr["origin"].astype(np.int64), tr["tau"]
    # origin: bit for bit unless the oracle's midpoint test is within its rounding error
    diff = org_g != org_o
    if diff.any():
        i = np.nonzero(diff)[0]
        assert np.all(i < K - 1)
        half_gap = (dbar[i + 1] - dbar[i]) / 2.0
        delta = (dbar[None, :] - dbar[i][:, None]) - half_gap[:, None]
        terms = zbar[None, :] ** 2 / delta
        fmid = 1.0 + rho * np.sum(terms, axis=1)
        emid = (K + 2) * EPS * (1.0 + rho * np.sum(np.abs(terms), axis=1))
        assert np.all(np.abs(fmid) <= emid), "origin differs where the midpoint test is decided"
    fprime, E, lam_m_d = _secular_terms(dbar, zbar, rho, org_o, tau_o)
    lam_o = dbar[org_o] + tau_o
    lam_g = dbar[org_g] + tau_g
    ulp = np.spacing(np.abs(tau_o))
    same = ~diff
    dtau = np.zeros(K)
    dtau[same] = np.abs(tau_g[same] - tau_o[same])
    dtau[diff] = np.abs(lam_g[diff] - lam_o[diff])
    bound_tau = 2.0 * E / fprime + 2.0 * ulp
    assert np.all(dtau <= bound_tau), float(np.max(dtau / bound_tau))
    # Loewner z: first-order propagation of the roots' differences
    prop = 0.5 * np.sum(dtau[:, None] / np.abs(lam_m_d), axis=0)       # per j
    rel_z = np.abs(tr["zhat"] - info["zhat"]) / np.abs(info["zhat"])
    assert np.all(rel_z <= prop + 4 * K * EPS), float(np.max(rel_z / (prop + 4 * K * EPS)))
    # column norms
    delta_u = np.max(dtau[:, None] / np.abs(lam_m_d), axis=1)          # per i
    u = info["zhat"][None, :] / lam_m_d                                 # rows i: column i of Qhat
    sinv_o = 1.0 / np.sqrt(np.sum(u * u, axis=1))
    rel_s = np.abs(tr["sinv"] - sinv_o) / sinv_o
    bound_s = np.max(prop + 4 * K * EPS) + delta_u + 2 * K * EPS
    assert np.all(rel_s <= bound_s), float(np.max(rel_s / bound_s))
    # a few ulp in tau for the well-conditioned roots (the typical case)
    return {"K": K, "max_ulp_tau": float(np.max(dtau[same] / ulp[same])) if same.any() else 0.0,
            "median_ulp_tau": float(np.median(dtau[same] / ulp[same])) if same.any() else 0.0,
            "origin_differs": int(diff.sum())}


def _run(api, D, Q, n1, beta):
    lam, qo, tr = api.merge_inspect(torch.tensor(D, device="cuda"), _fortran(Q), n1, beta)
    return _check_trace(D, Q, n1, beta, tr)


@pytest.mark.parametrize("K,n1,n2,a,b", [(8, 20, 20, 4, 4), (33, 40, 40, 17, 16),
                                         (1000, 700, 700, 500, 500), (4097, 2200, 2200, 2049, 2048)])
def test_merge_trace_structured(api, K, n1, n2, a, b):
    D, Q, beta = structured_merge(n1, n2, a, b, seed=K)
    st = _run(api, D, Q, n1, beta)
    assert st["K"] == K
    assert st["median_ulp_tau"] <= 4.0
    print(st)


@pytest.mark.parametrize("n1,n2,seed", [(300, 301, 3), (1, 9, 5), (64, 64, 11)])
def test_merge_trace_dense(api, n1, n2, seed):
    D, Q, beta = W.merge_problem(n1, n2, seed)
    st = _run(api, D, Q, n1, beta)
    print(st)


def test_merge_trace_equal_poles(api):
    """Type-2 deflation: two pairs of equal poles across the halves give rotations."""
    D, Q, n1, beta = equal_pole_merge()
    _run(api, D, Q, n1, beta)


@pytest.mark.parametrize("n,seed", [(2048, 0), (1024, 5)])
def test_merge_trace_tridiag_level(api, n, seed):
    """The top merge of a U[-1, 1] tridiagonal: heavy deflation, rotations of nearly
    equal poles, small K."""
    D, Q, n1, beta = tridiag_level_merge(n, seed)
    st = _run(api, D, Q, n1, beta)
    print(st)
