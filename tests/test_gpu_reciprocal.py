"""The reciprocal of the secular sums (Newton-Raphson on the hardware approximation)
against the correctly rounded 1/x: within one unit in the last place over the
exponent range the sums meet, exact at powers of two, 0 above 2^1022."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import _lib
    return _lib.load()


def _rcp(lib, x):
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    rt = torch.empty_like(xt)
    assert lib.tdc_diag_reciprocal(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(rt.data_ptr()),
                                   xt.numel(), None) == 0
    torch.cuda.synchronize()
    return rt.cpu().numpy()


def test_reciprocal_within_one_ulp(lib):
    g = np.random.Generator(np.random.PCG64(5))
    n = 1 << 20
    x = g.uniform(1.0, 2.0, n) * np.exp2(g.integers(-1000, 1000, n)) * np.where(g.random(n) < 0.5, -1.0, 1.0)
    r = _rcp(lib, x)
    ref = 1.0 / x
    assert np.all(np.abs(r - ref) <= np.spacing(np.abs(ref)))
    # nearly all correctly rounded
    assert np.mean(r == ref) > 0.99


def test_reciprocal_special_values(lib):
    k = np.arange(-1000, 1001)
    x = np.concatenate([np.exp2(k.astype(np.float64)), -np.exp2(k.astype(np.float64))])
    r = _rcp(lib, x)
    assert np.array_equal(r, 1.0 / x)
    big = np.array([2.0 ** 1022 * 1.5, -(2.0 ** 1023) * 1.9])
    assert np.array_equal(_rcp(lib, big), np.zeros(2))
    assert lib.tdc_diag_reciprocal(None, None, 0, None) == 0
    assert lib.tdc_diag_reciprocal(None, None, -1, None) == -3


def _rsqrt(lib, x):
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    rt = torch.empty_like(xt)
    assert lib.tdc_diag_rsqrt(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(rt.data_ptr()),
                              xt.numel(), None) == 0
    torch.cuda.synchronize()
    return rt.cpu().numpy()


def test_rsqrt_within_four_ulp(lib):
    """The leaf rotations' 1/sqrt(f^2 + g^2) over the range it is used on."""
    g = np.random.Generator(np.random.PCG64(6))
    n = 1 << 20
    x = g.uniform(1.0, 2.0, n) * np.exp2(g.integers(-1020, 1019, n))
    y = _rsqrt(lib, x)
    ref = 1.0 / np.sqrt(x)                     # within one ulp of 1/sqrt(x) itself
    # the last Newton step y (1.5 - (x / 2) y^2) rounds three times (y^2, the fma, the
    # product): about 1.5 ulp of its own, plus the reference's one ulp
    ulps = np.abs(y - ref) / np.spacing(ref)
    worst = np.argsort(ulps)[-3:]
    assert ulps.max() <= 4, f"worst {ulps[worst]} ulp at x = {x[worst]}"
    # residual of the defining equation: x y^2 - 1 within a few ulp
    assert np.max(np.abs(x * y * y - 1.0)) <= 8 * 2.0 ** -52
    k = np.arange(-1020, 1020, 2).astype(np.float64)
    exact = np.exp2(-k / 2)
    assert np.all(np.abs(_rsqrt(lib, np.exp2(k)) - exact) <= np.spacing(exact))
