"""tdc_syev_tridiag_noalloc: the solve for small orders with its workspace in a fixed
array inside the library, for callers that cannot allocate device memory (an
allocator that forbids new device allocations, a plug-in that is handed only its
input and output buffers).  Called through the C ABI, twice in a row, and compared
with tdc_syev_tridiag on a caller-provided workspace.  This file runs last so that a
stop at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import metrics

torch = pytest.importorskip("torch")

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import _lib
    return _lib.load()


def _vp(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def test_noalloc_rejects_out_of_range_orders(lib):
    P = ctypes.c_void_p
    assert lib.tdc_syev_tridiag_noalloc(0, P(8), P(8), P(8), P(8), 1, None, None) == -1
    assert lib.tdc_syev_tridiag_noalloc(513, P(8), P(8), P(8), P(8), 513, None, None) == -1


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_twice(lib):
    from paper_1612_07526_gb300 import _lib
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    for call, (n, seed) in enumerate([(512, 3), (300, 4)]):
        d, e = W.uniform_tridiag(n, seed)
        dt = torch.tensor(d, device="cuda")
        et = torch.tensor(e, device="cuda")
        # the library's own scratch
        lam_a = torch.empty(n, dtype=torch.float64, device="cuda")
        q_a = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device="cuda")
        st_a = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = lib.tdc_syev_tridiag_noalloc(n, _vp(dt), _vp(et), _vp(lam_a), _vp(q_a), n, _vp(st_a), sp)
        assert rc == 0, f"call {call}: rc={rc}"
        # the existing entry point with a caller-provided workspace
        o = _lib.default_opts()
        nb = lib.tdc_workspace_bytes(n, ctypes.byref(o))
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        lam_b = torch.empty(n, dtype=torch.float64, device="cuda")
        q_b = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device="cuda")
        st_b = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = lib.tdc_syev_tridiag(n, _vp(dt), _vp(et), _vp(lam_b), _vp(q_b), n, ctypes.byref(o), _vp(ws),
                                  nb, _vp(st_b), sp)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(st_a.item()) == 0 and int(st_b.item()) == 0
        la, lb = lam_a.cpu().numpy(), lam_b.cpu().numpy()
        qa, qb = q_a.cpu().numpy(), q_b.cpu().numpy()
        nrm = metrics.tnorm(d, e)
        assert np.max(np.abs(la - lb)) <= 10 * n * EPS * nrm
        err, _ = metrics.column_agreement(lb, qb, qa, nrm, min_relgap=1e-4)
        assert err <= 1e-7
        assert metrics.scaled_residual(d, e, la, qa) <= 10
        assert metrics.orthogonality(qa) <= 100 * n * EPS


@pytest.mark.gpu
def test_noalloc_call_takes_no_device_memory(lib):
    """With its outputs allocated beforehand, a call changes the device's free memory by
    nothing (a device allocation would take at least one 2 MiB page), and it records no
    per-phase events even while the library's profiling is on."""
    from paper_1612_07526_gb300 import _lib
    n = 400
    d, e = W.uniform_tridiag(n, 9)
    dt = torch.tensor(d, device="cuda")
    et = torch.tensor(e, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    q = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.tdc_syev_tridiag_noalloc(n, _vp(dt), _vp(et), _vp(lam), _vp(q), n, _vp(st), sp) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    lib.tdc_profile_begin()
    assert lib.tdc_syev_tridiag_noalloc(n, _vp(dt), _vp(et), _vp(lam), _vp(q), n, _vp(st), sp) == 0
    torch.cuda.synchronize()
    prof = _lib.TdcProfile()
    assert lib.tdc_profile_end(ctypes.byref(prof)) == 0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert sum(prof.launches) == 0 and prof.calls == 0
    assert int(st.item()) == 0
    assert metrics.scaled_residual(d, e, lam.cpu().numpy(), q.cpu().numpy()) <= 10
