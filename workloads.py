"""Seeded synthetic inputs for the tridiagonal divide-and-conquer eigensolver.

This module only draws numbers: it holds none of the solver's arithmetic, so both
the CPU oracle and the GPU library's tests and benchmark may use it.  Every
generator takes an explicit seed and uses numpy's PCG64 bit generator.

Workloads (the shapes and value distributions of the paper's test matrices and of
the benchmark configurations):

* ``uniform_tridiag``   d_i, e_i ~ U[-1, 1] i.i.d.
* ``normal_tridiag``    d_i, e_i ~ N(0, 1) i.i.d.
* ``toeplitz_121``      d_i = 2, e_i = 1 (Example 2 and the Toeplitz-type matrix
                        of Example 3; closed-form spectrum)
* ``graded_tridiag``    d_i = 10^(-8 i/n) U[-1,1], e_i = 10^(-8 i/n) U[-1,1],
                        i 0-based
* ``clement`` / ``hermite`` / ``sht``   the "difficult" matrices of Examples 3-4
* ``batched_sizes``     n log-uniform in [32, 2048]
* ``merge_problem``     a random rank-one merge: two sorted spectra, two random
                        orthogonal blocks and a coupling entry
* ``rank_one_example``  the Section 2.2 Cauchy-like example (d_i = i/N, rho = 1,
                        random unit z)
* ``hss_example1``      the two dense Toeplitz matrices of Example 1
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_tridiag(n: int, seed: int):
    g = rng(seed)
    d = g.uniform(-1.0, 1.0, size=n)
    e = g.uniform(-1.0, 1.0, size=max(n - 1, 0))
    return d, e


def normal_tridiag(n: int, seed: int):
    g = rng(seed)
    d = g.standard_normal(n)
    e = g.standard_normal(max(n - 1, 0))
    return d, e


def toeplitz_121(n: int):
    return np.full(n, 2.0), np.ones(max(n - 1, 0))


def graded_tridiag(n: int, seed: int):
    g = rng(seed)
    i = np.arange(n, dtype=np.float64)
    scale_d = 10.0 ** (-8.0 * i / n)
    scale_e = 10.0 ** (-8.0 * i[: max(n - 1, 0)] / n)
    d = scale_d * g.uniform(-1.0, 1.0, size=n)
    e = scale_e * g.uniform(-1.0, 1.0, size=max(n - 1, 0))
    return d, e


def clement(n: int):
    """Clement-type matrix: zero diagonal, off-diagonal sqrt(i (n - i)), i = 1..n-1."""
    i = np.arange(1, n, dtype=np.float64)
    return np.zeros(n), np.sqrt(i * (n - i))


def hermite(n: int):
    """Hermite-type matrix: zero diagonal, off-diagonal sqrt(i), i = 1..n-1."""
    return np.zeros(n), np.sqrt(np.arange(1, n, dtype=np.float64))


def sht(n: int, m: int | None = None):
    """Spherical-harmonic-transform tridiagonal of Example 4 (j = 0..n-1, l from m)."""
    if m is None:
        m = n
    m = float(m)

    def c(l):
        return np.sqrt((l - m + 1) * (l - m + 2) * (l + m + 1) * (l + m + 2)
                       / ((2 * l + 1) * (2 * l + 3) ** 2 * (2 * l + 5)))

    def dd(l):
        return (2 * l * (l + 1) - 2 * m * m - 1) / ((2 * l - 1) * (2 * l + 3))

    j = np.arange(n, dtype=np.float64)
    return dd(m + 2 * j), c(m + 2 * j[:-1])


def batched_sizes(batch: int, seed: int, lo: int = 32, hi: int = 2048):
    g = rng(seed)
    u = g.uniform(math.log(lo), math.log(hi), size=batch)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), lo, hi)


def batched_normal(batch: int, seed: int, lo: int = 32, hi: int = 2048):
    """Ragged batch: sizes log-uniform in [lo, hi], d, e ~ N(0, 1), one seed per problem."""
    sizes = batched_sizes(batch, seed, lo, hi)
    probs = [normal_tridiag(int(n), seed * 100003 + 7 * k + 1) for k, n in enumerate(sizes)]
    return sizes, probs


def random_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    a = g.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


def merge_problem(n1: int, n2: int, seed: int, spread: float = 1.0):
    """Inputs of one rank-one merge: D (each half ascending), block-diagonal Q, beta."""
    g = rng(seed)
    d1 = np.sort(g.uniform(-spread, spread, size=n1))
    d2 = np.sort(g.uniform(-spread, spread, size=n2))
    q = np.zeros((n1 + n2, n1 + n2))
    q[:n1, :n1] = random_orthogonal(n1, g)
    q[n1:, n1:] = random_orthogonal(n2, g)
    beta = float(g.uniform(-1.0, 1.0))
    return np.concatenate([d1, d2]), q, beta


def rank_one_example(N: int = 1000, seed: int = 0):
    """d_i = i / N, rho = 1, z a normalised Gaussian vector (Section 2.2, Fig. 2)."""
    g = rng(seed)
    d = np.arange(1, N + 1, dtype=np.float64) / N
    z = g.standard_normal(N)
    return d, z / np.linalg.norm(z), 1.0


def hss_example1(n: int, which: int, dstep: float = 0.1):
    """Example 1 test matrices: 1 -> a_ii = n^2, a_ij = i - j; 2 -> kinetic-energy matrix."""
    i = np.arange(n, dtype=np.float64)
    diff = i[:, None] - i[None, :]
    if which == 1:
        a = diff.copy()
        np.fill_diagonal(a, float(n) ** 2)
        return a
    with np.errstate(divide="ignore"):
        a = (-1.0) ** np.abs(diff) / (diff ** 2 * dstep ** 2)
    np.fill_diagonal(a, math.pi ** 2 / (6.0 * dstep ** 2))
    return a


def gaussian(shape, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(shape)
