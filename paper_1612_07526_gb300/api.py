"""PyTorch-facing wrappers of the C ABI in include/tdc.h.

PyTorch supplies device memory and streams; every computation runs inside libtdc's
CUDA kernels.  Matrices are returned as column-major (Fortran-order) float64 CUDA
tensors, so ``Q[:, j]`` is the eigenvector of ``lam[j]``.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

_WS: dict = {}


class TdcError(RuntimeError):
    pass


STATUS_BITS = {1: "secular root iteration cap", 2: "non-finite input", 4: "leaf QL iteration cap",
               8: "device wait timed out"}


def _vp(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def workspace(nbytes: int, device=None, key="default") -> torch.Tensor:
    """A cached device byte buffer of at least nbytes (256-byte aligned)."""
    device = torch.device("cuda") if device is None else torch.device(device)
    k = (key, device.index if device.index is not None else torch.cuda.current_device())
    buf = _WS.get(k)
    if buf is None or buf.numel() < nbytes:
        _WS.pop(k, None)
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
        _WS[k] = buf
    assert buf.data_ptr() % 256 == 0
    return buf


def release_workspaces():
    _WS.clear()


def _check_rc(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"{what}: argument {-rc} is invalid")
    if rc == 3:
        raise TdcError(f"{what}: workspace too small")
    if rc == 4:
        raise TdcError(f"{what}: CUDA launch error")
    if rc != 0:
        raise TdcError(f"{what}: status {rc}")


def _raise_status(bits: int, what: str):
    if bits:
        names = [v for k, v in STATUS_BITS.items() if bits & k]
        raise TdcError(f"{what}: device status {bits} ({', '.join(names)})")


def fortran_empty(rows: int, cols: int, device) -> torch.Tensor:
    return torch.empty_strided((rows, cols), (1, max(rows, 1)), dtype=torch.float64, device=device)


def _opts(opts, **kw):
    if opts is None:
        return _lib.default_opts(**kw)
    if isinstance(opts, dict):
        return _lib.default_opts(**{**opts, **kw})
    return opts


def syev_tridiag(d: torch.Tensor, e: torch.Tensor, opts=None, stream=None, check: bool = True,
                 status: torch.Tensor | None = None, out=None):
    """Eigenvalues (ascending) and eigenvectors of tridiag(e, d, e) on the GPU.

    d: (n,) float64 CUDA, e: (n-1,) float64 CUDA.  Returns (lam, Q) with Q column-major."""
    lib = _lib.load()
    n = int(d.shape[0])
    assert d.dtype == torch.float64 and d.is_cuda and d.is_contiguous()
    assert e.dtype == torch.float64 and e.is_cuda and e.is_contiguous() and e.shape[0] == max(n - 1, 0)
    o = _opts(opts)
    if out is None:
        lam = torch.empty(n, dtype=torch.float64, device=d.device)
        q = fortran_empty(n, n, d.device)
    else:
        lam, q = out
    nb = lib.tdc_workspace_bytes(n, ctypes.byref(o))
    if nb == 0:
        raise ValueError("invalid size or options")
    ws = workspace(nb, d.device)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=d.device)
    rc = lib.tdc_syev_tridiag(n, _vp(d), _vp(e if n > 1 else None), _vp(lam), _vp(q), n,
                              ctypes.byref(o), _vp(ws), ws.numel(), _vp(st), _stream(stream))
    _check_rc(rc, "tdc_syev_tridiag")
    if check:
        _raise_status(lib.tdc_read_status(_vp(st), _stream(stream)), "tdc_syev_tridiag")
    return lam, q


def merge(D: torch.Tensor, Q: torch.Tensor, n1: int, beta: float, opts=None, stream=None,
          check: bool = True):
    """One rank-one merge (Eqs. 3-6) of diag(Q1 D1 Q1^T, Q2 D2 Q2^T) + |beta| v v^T.

    Q is (n, n) column-major (only its two diagonal blocks are read).  Returns
    (lam, Q_out, K)."""
    lib = _lib.load()
    n = int(D.shape[0])
    assert Q.stride() == (1, n) and Q.shape == (n, n) and Q.dtype == torch.float64
    o = _opts(opts)
    lam = torch.empty(n, dtype=torch.float64, device=D.device)
    qo = fortran_empty(n, n, D.device)
    kout = torch.zeros(1, dtype=torch.int64, device=D.device)
    nb = lib.tdc_merge_workspace_bytes(n, ctypes.byref(o))
    if nb == 0:
        raise ValueError("invalid size or options")
    ws = workspace(nb, D.device)
    st = torch.zeros(1, dtype=torch.int32, device=D.device)
    rc = lib.tdc_merge(int(n1), int(n - n1), _vp(D), _vp(Q), n, float(beta), _vp(lam), _vp(qo), n,
                       _vp(kout), ctypes.byref(o), _vp(ws), ws.numel(), _vp(st), _stream(stream))
    _check_rc(rc, "tdc_merge")
    if check:
        _raise_status(lib.tdc_read_status(_vp(st), _stream(stream)), "tdc_merge")
    return lam, qo, int(kout.item()) if check else kout


def syev_tridiag_batched(ds, es, opts=None, stream=None, check: bool = True):
    """Solves len(ds) independent problems in one level-synchronous sweep.

    ds[p]: (n_p,) and es[p]: (n_p - 1,) float64 tensors (CPU or CUDA).  Returns
    (lam_cat, Q_cat, sizes, q_offsets): Q of problem p is the n_p x n_p column-major
    block at q_offsets[p] of Q_cat."""
    lib = _lib.load()
    sizes = np.array([int(x.shape[0]) for x in ds], dtype=np.int64)
    b = len(sizes)
    off = np.zeros(b, dtype=np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    qoff = np.zeros(b, dtype=np.int64)
    qoff[1:] = np.cumsum(sizes * sizes)[:-1]
    dev = torch.device("cuda")
    d_cat = torch.cat([torch.as_tensor(x, dtype=torch.float64) for x in ds]).to(dev)
    e_cat = torch.zeros(int(sizes.sum()), dtype=torch.float64)
    for p in range(b):
        if sizes[p] > 1:
            e_cat[off[p]:off[p] + sizes[p] - 1] = torch.as_tensor(es[p], dtype=torch.float64)
    e_cat = e_cat.to(dev)
    lam = torch.empty(int(sizes.sum()), dtype=torch.float64, device=dev)
    q = torch.empty(int((sizes * sizes).sum()), dtype=torch.float64, device=dev)
    o = _opts(opts)
    nb = lib.tdc_batched_workspace_bytes(b, sizes.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o))
    if nb == 0:
        raise ValueError("invalid sizes or options")
    ws = workspace(nb, dev, key="batched")
    st = torch.zeros(b, dtype=torch.int32, device=dev)
    rc = lib.tdc_syev_tridiag_batched(b, sizes.ctypes.data_as(ctypes.c_void_p),
                                      off.ctypes.data_as(ctypes.c_void_p),
                                      qoff.ctypes.data_as(ctypes.c_void_p), _vp(d_cat), _vp(e_cat),
                                      _vp(lam), _vp(q), ctypes.byref(o), _vp(ws), ws.numel(), _vp(st),
                                      _stream(stream))
    _check_rc(rc, "tdc_syev_tridiag_batched")
    if check:
        bits = st.cpu().numpy()
        if bits.any():
            _raise_status(int(np.bitwise_or.reduce(bits)), "tdc_syev_tridiag_batched")
    return lam, q, sizes, qoff


def batched_block(q_cat: torch.Tensor, sizes, qoff, p: int) -> torch.Tensor:
    n = int(sizes[p])
    return q_cat[int(qoff[p]):int(qoff[p]) + n * n].view(n, n).t()


class HostSolver:
    """The end-to-end call a host-memory user makes: tdc_syev_tridiag_host with a
    device buffer it keeps and page-locked host staging."""

    def __init__(self, n: int, opts=None, device=None):
        self.lib = _lib.load()
        self.n = n
        self.o = _opts(opts)
        nb = self.lib.tdc_host_buffer_bytes(n, ctypes.byref(self.o))
        if nb == 0:
            raise ValueError("invalid size or options")
        self.buf = torch.empty(nb, dtype=torch.uint8, device=device or "cuda")
        self.lam = torch.empty(n, dtype=torch.float64).pin_memory()
        self.q = torch.empty(n * n, dtype=torch.float64).pin_memory()

    def __call__(self, d_host: torch.Tensor, e_host: torch.Tensor, stream=None):
        rc = self.lib.tdc_syev_tridiag_host(self.n, _vp(d_host), _vp(e_host), _vp(self.lam), _vp(self.q),
                                            self.n, ctypes.byref(self.o), _vp(self.buf), self.buf.numel(),
                                            _stream(stream))
        if rc < 0 or rc in (3, 4):
            _check_rc(rc, "tdc_syev_tridiag_host")
        _raise_status(rc, "tdc_syev_tridiag_host")
        return self.lam, self.q.view(self.n, self.n).t()

    @property
    def h2d_bytes(self):
        return 8 * (2 * self.n - 1)

    @property
    def d2h_bytes(self):
        return 8 * (self.n + self.n * self.n)
