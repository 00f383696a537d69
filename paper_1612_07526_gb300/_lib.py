"""ctypes binding of libtdc.so (argument marshalling only; every step runs in the
library's CUDA kernels).  Importing this module loads the library and raises if it
is missing: there is no fallback implementation."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdc.so")

PATH_DENSE_FP64 = 0
PATH_DENSE_OZAKI = 1
PATH_HSS = 2
PATH_AUTO = 3


class TdcOpts(ctypes.Structure):
    _fields_ = [
        ("path", ctypes.c_int32),
        ("leaf", ctypes.c_int32),
        ("hss_tol", ctypes.c_double),
        ("hss_leaf", ctypes.c_int32),
        ("hss_rp", ctypes.c_int32),
        ("k_threshold", ctypes.c_int64),
        ("ozaki_slices", ctypes.c_int32),
        ("max_secular_iter", ctypes.c_int32),
        ("tile_cfg", ctypes.c_int32),
        ("secular_lanes", ctypes.c_int32),
        ("eigvec", ctypes.c_int32),
        ("hss_grow", ctypes.c_int32),
    ]


EIGVEC_LOWNER = 0
EIGVEC_EXTENDED = 1


class TdcProfile(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_double * 13),
        ("launches", ctypes.c_int64 * 13),
        ("product_flops", ctypes.c_double),
        ("product_min_bytes", ctypes.c_double),
        ("merges", ctypes.c_int64),
        ("K_total", ctypes.c_int64),
        ("calls", ctypes.c_int64),
        ("fp64_product_flops", ctypes.c_double),
        ("split_product_flops", ctypes.c_double),
        ("split_tensor_flops", ctypes.c_double),
        ("defl_copy_bytes", ctypes.c_double),
        ("secular_flops", ctypes.c_double),
        ("hss_fallbacks", ctypes.c_int64),
        ("hss_regrowths", ctypes.c_int64),
        ("hss_sampling_flops", ctypes.c_double),
        ("level_fp64_min_bytes", ctypes.c_double * 32),
        ("level_fp64_flops", ctypes.c_double * 32),
        ("level_fp64_product_ms", ctypes.c_double * 32),
        ("secular_evals", ctypes.c_int64),
        ("sg_gemm_ms", ctypes.c_double),
        ("sg_tensor_flops", ctypes.c_double),
    ]


class TdcMergeTrace(ctypes.Structure):
    """Device pointers receiving a merge's intermediate values (tdc_merge_inspect)."""
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "counts", "perm", "d_sorted", "z_sorted", "kept", "deflated", "rot_j", "rot_k", "rot_c", "rot_s",
        "dbar", "zbar", "origin", "tau", "zhat", "sinv", "tau_lo")]


PHASES = ["tear+leaves", "deflation", "secular", "lowner+norms", "placement", "product",
          "deflated-copy", "sign", "split-product", "operand-split", "hss-sampling", "hss-compression",
          "hss-multiply"]

_lib = None

# (name, restype, argtypes) of every symbol declared in include/tdc.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_OPT = ctypes.POINTER(TdcOpts)
SIGNATURES = [
    ("tdc_default_opts", None, [_OPT]),
    ("tdc_workspace_bytes", ctypes.c_size_t, [_I64, _OPT]),
    ("tdc_syev_tridiag", ctypes.c_int, [_I64, _P, _P, _P, _P, _I64, _OPT, _P, ctypes.c_size_t, _P, _P]),
    ("tdc_host_buffer_bytes", ctypes.c_size_t, [_I64, _OPT]),
    ("tdc_syev_tridiag_host", ctypes.c_int, [_I64, _P, _P, _P, _P, _I64, _OPT, _P, ctypes.c_size_t, _P]),
    ("tdc_syev_tridiag_host_async", ctypes.c_int, [_I64, _P, _P, _P, _P, _I64, _OPT, _P, ctypes.c_size_t, _P,
                                                   _P]),
    ("tdc_merge_workspace_bytes", ctypes.c_size_t, [_I64, _OPT]),
    ("tdc_merge", ctypes.c_int, [_I64, _I64, _P, _P, _I64, ctypes.c_double, _P, _P, _I64, _P, _OPT,
                                 _P, ctypes.c_size_t, _P, _P]),
    ("tdc_merge_inspect", ctypes.c_int, [_I64, _I64, _P, _P, _I64, ctypes.c_double, _P, _P, _I64, _P, _OPT,
                                         _P, ctypes.c_size_t, _P, _P, ctypes.POINTER(TdcMergeTrace)]),
    ("tdc_batched_workspace_bytes", ctypes.c_size_t, [ctypes.c_int32, _P, _OPT]),
    ("tdc_syev_tridiag_batched", ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _OPT, _P,
                                                ctypes.c_size_t, _P, _P]),
    ("tdc_read_status", ctypes.c_int, [_P, _P]),
    ("tdc_backward_workspace_bytes", ctypes.c_size_t, [_I64, _OPT]),
    ("tdc_batched_plan_create", ctypes.c_int, [ctypes.c_int32, _P, _OPT, _P, ctypes.c_size_t, _P,
                                               ctypes.POINTER(ctypes.c_void_p)]),
    ("tdc_batched_plan_execute", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("tdc_batched_plan_destroy", None, [_P]),
    ("tdc_batched_plan_execute_persistent", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("tdc_batched_plan_execute_host", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("tdc_syev_tridiag_backward", ctypes.c_int, [_I64, _P, _P, _I64, _P, _P, _I64, _P, _P, _OPT, _P,
                                                 ctypes.c_size_t, _P, _P]),
    ("tdc_backward_batched_workspace_bytes", ctypes.c_size_t, [ctypes.c_int32, _P, _I64, _OPT]),
    ("tdc_syev_tridiag_backward_batched", ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _OPT, _P,
                                                         ctypes.c_size_t, _P, _P]),
    ("tdc_syev_tridiag_noalloc", ctypes.c_int, [_I64, _P, _P, _P, _P, _I64, _P, _P]),
    ("tdc_autotune", ctypes.c_int, [_I64, _P, _P, _P, _P, _I64, _OPT, _P, ctypes.c_size_t, _P, ctypes.c_int32,
                                    _P, _P, _P]),
    ("tdc_batched_plan_autotune", ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int32, _P, _P]),
    ("tdc_profile_begin", None, []),
    ("tdc_profile_end", ctypes.c_int, [ctypes.POINTER(TdcProfile)]),
    ("tdc_version", ctypes.c_char_p, []),
    ("tdc_struct_bytes", ctypes.c_size_t, [ctypes.c_int]),
    ("tdc_diag_reciprocal", ctypes.c_int, [_P, _P, _I64, _P]),
    ("tdc_diag_rsqrt", ctypes.c_int, [_P, _P, _I64, _P]),
    ("tdc_diag_wait_timeout", ctypes.c_int, [_I64, _P, _P, _P]),
    ("tdc_diag_split_combine", ctypes.c_int, [_P, _P, _P, _P, _I64, _P]),
]


# FP64 product tile shapes (rows, columns) by tdc_opts.tile_cfg index
TILE_SHAPES = [(128, 128), (128, 64), (64, 64), (64, 32), (32, 32), (128, 32), (64, 16), (128, 16),
               (16, 16), (16, 32), (16, 64), (32, 16)]


def load(path: str = LIB_PATH):
    """Loads libtdc.so (building nothing).  Raises OSError if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libtdc.so not found at {path}: run __graft_entry__.build() first "
                      "(the library has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_opts(**kw) -> TdcOpts:
    o = TdcOpts()
    load().tdc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o
