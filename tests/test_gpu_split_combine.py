"""The split-precision product's output combination (Eq. (6)'s product in split form):
(acc + tsum 2^-8) 2^e with the conversions and the power-of-two scaling done on the
integer pipes and one FP64 addition.  Checked bit for bit against the same arithmetic
in NumPy (int64 to float64 rounded to nearest, float32 to float64 exactly, one
float64 addition, ldexp), across the int64 range that needs rounding (|acc| > 2^53),
carries into the next power of two, zero and subnormal-float tails, and scalings that
leave the normal range."""
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


def _combine(lib, acc, ts, e):
    a = torch.tensor(acc, dtype=torch.int64, device="cuda")
    t = torch.tensor(ts, dtype=torch.float32, device="cuda")
    ee = torch.tensor(e, dtype=torch.int32, device="cuda")
    r = torch.empty(len(acc), dtype=torch.float64, device="cuda")
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    assert lib.tdc_diag_split_combine(vp(a), vp(t), vp(ee), vp(r), len(acc), None) == 0
    torch.cuda.synchronize()
    return r.cpu().numpy()


def _reference(acc, ts, e):
    x = acc.astype(np.float64) + ts.astype(np.float64) * 2.0 ** -8
    return np.ldexp(x, e)


def test_combine_bit_exact(lib):
    rng = np.random.default_rng(5)
    n = 200_000
    mag = rng.integers(0, 62, n)
    acc = (rng.integers(0, 2**62, n, dtype=np.int64) >> (62 - mag)) * rng.choice([-1, 1], n)
    acc[:64] = [0, 1, -1, 2**53, 2**53 + 1, 2**53 + 2, 2**53 + 3, -(2**53 + 1), 2**54 - 1, 2**62 - 1,
                -(2**62 - 1), 2**63 - 1, -(2**63 - 1), 2**55 + 2**3, 2**55 + 2**2, 2**55 + 3 * 2**2] + \
        list(rng.integers(-2**40, 2**40, 48))
    ts = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 25, n))).astype(np.float32)
    ts[:8] = [0.0, -0.0, 1e-40, -1e-42, 2.0 ** -126, 16777216.0, -1.0, 3.0]
    e = rng.integers(-1100, 60, n).astype(np.int32)
    e[:16] = 0
    got = _combine(lib, acc, ts, e)
    ref = _reference(acc, ts, e)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64)), np.flatnonzero(got.view(np.int64) != ref.view(np.int64))[:10]


def test_combine_rejects_bad_arguments(lib):
    assert lib.tdc_diag_split_combine(None, None, None, None, 0, None) == 0
    assert lib.tdc_diag_split_combine(None, None, None, None, -1, None) == -5
