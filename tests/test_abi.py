"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/tdc.h declares.  No GPU and no compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "tdc.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1612_07526_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tdc_syev_tridiag", "tdc_merge", "tdc_syev_tridiag_batched",
                     "tdc_workspace_bytes", "tdc_syev_tridiag_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1612_07526_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(_declared()) <= bound


def test_opts_struct_layout(lib):
    from paper_1612_07526_gb300 import _lib
    o = _lib.default_opts()
    assert o.leaf == 32 and o.path == 0 and o.hss_tol == 1e-12 and o.max_secular_iter == 64
    assert ctypes.sizeof(_lib.TdcOpts) == 56
    assert o.eigvec == 0 and o.hss_grow == 1


def test_host_side_argument_checks(lib):
    """Invalid arguments are rejected on the host with -i before anything launches."""
    from paper_1612_07526_gb300 import _lib
    o = _lib.default_opts()
    P = ctypes.c_void_p
    assert lib.tdc_syev_tridiag(0, P(8), P(8), P(8), P(8), 1, ctypes.byref(o), P(256), 1 << 20, None, None) == -1
    assert lib.tdc_syev_tridiag(4, None, P(8), P(8), P(8), 4, ctypes.byref(o), P(256), 1 << 20, None, None) == -2
    assert lib.tdc_syev_tridiag(4, P(8), P(8), P(8), P(8), 3, ctypes.byref(o), P(256), 1 << 20, None, None) == -6
    bad = _lib.default_opts(leaf=0)
    assert lib.tdc_syev_tridiag(4, P(8), P(8), P(8), P(8), 4, ctypes.byref(bad), P(256), 1 << 20, None, None) == -7
    assert o.secular_lanes == 0
    for lanes in (3, 5, 64, -1):
        bad = _lib.default_opts(secular_lanes=lanes)
        assert lib.tdc_syev_tridiag(4, P(8), P(8), P(8), P(8), 4, ctypes.byref(bad), P(256), 1 << 20,
                                    None, None) == -7
    assert lib.tdc_syev_tridiag(4, P(8), P(8), P(8), P(8), 4, ctypes.byref(o), P(255), 1 << 20, None, None) == -8
    # workspace too small is reported before any launch
    assert lib.tdc_syev_tridiag(64, P(8), P(8), P(8), P(8), 64, ctypes.byref(o), P(256), 16, None, None) == 3
    assert lib.tdc_merge(0, 3, P(8), P(8), 3, 1.0, P(8), P(8), 3, None, ctypes.byref(o), P(256), 1 << 20,
                         None, None) == -1
    # host and pipeline entries: argument checks come before any CUDA call
    assert lib.tdc_syev_tridiag_host_async(0, P(8), P(8), P(8), P(8), 1, ctypes.byref(o), P(256), 1 << 20,
                                           P(8), None) == -1
    assert lib.tdc_syev_tridiag_host_async(4, P(8), P(8), P(8), P(8), 4, ctypes.byref(o), P(256), 1 << 20,
                                           None, None) == -10
    assert lib.tdc_syev_tridiag_host_async(4, P(8), P(8), P(8), P(8), 4, ctypes.byref(o), P(255), 1 << 20,
                                           P(8), None) == -8
    assert lib.tdc_batched_plan_execute_host(None, P(8), P(8), P(8), P(8), P(8), P(8), P(8), P(8), P(8),
                                             P(8), None) == -1
    assert lib.tdc_diag_reciprocal(None, None, -1, None) == -3
    assert lib.tdc_diag_rsqrt(None, None, -1, None) == -3
    assert lib.tdc_diag_rsqrt(None, P(8), 4, None) == -1
    assert lib.tdc_diag_split_combine(P(8), P(8), P(8), P(8), -1, None) == -5
    assert lib.tdc_diag_split_combine(None, P(8), P(8), P(8), 4, None) == -1
    assert lib.tdc_diag_split_combine(P(8), P(8), P(8), None, 4, None) == -4
    assert lib.tdc_workspace_bytes(0, ctypes.byref(o)) == 0
    assert lib.tdc_workspace_bytes(1024, ctypes.byref(o)) > 2 * 1024 * 1024 * 8


def test_workspace_sizes(lib):
    """Host-only sizing (no CUDA call): the FP64 workspace is the 3 n^2 pool plus
    O(n) vectors, the split path adds its slice arena, the host entry adds n^2 for Q
    and three vectors, a batch needs at least the sum of its problems' pools."""
    from paper_1612_07526_gb300 import _lib
    o = _lib.default_opts()
    for n in (32, 1024, 32768):
        ws = lib.tdc_workspace_bytes(n, ctypes.byref(o))
        pool = 3 * n * n * 8
        assert pool <= ws <= pool + 8 * 1024 * n + (8 << 20)
        hb = lib.tdc_host_buffer_bytes(n, ctypes.byref(o))
        assert hb >= ws + n * n * 8 + 3 * n * 8
    oz = _lib.default_opts(path=1)
    assert lib.tdc_workspace_bytes(32768, ctypes.byref(oz)) > 1.9 * lib.tdc_workspace_bytes(32768, ctypes.byref(o))
    sizes = (ctypes.c_int64 * 3)(100, 2000, 32)
    b = lib.tdc_batched_workspace_bytes(3, sizes, ctypes.byref(o))
    assert b >= 3 * 8 * (100 ** 2 + 2000 ** 2 + 32 ** 2)


def test_struct_layouts_match_the_library():
    """The ctypes mirrors of tdc_opts, tdc_profile and tdc_merge_trace have the sizes the
    library was compiled with."""
    import ctypes
    from paper_1612_07526_gb300 import _lib
    lib = _lib.load()
    assert lib.tdc_struct_bytes(0) == ctypes.sizeof(_lib.TdcOpts)
    assert lib.tdc_struct_bytes(1) == ctypes.sizeof(_lib.TdcProfile)
    assert lib.tdc_struct_bytes(2) == ctypes.sizeof(_lib.TdcMergeTrace)
    assert lib.tdc_struct_bytes(3) == 0
