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


def autotune(d: torch.Tensor, e: torch.Tensor, opts=None, stream=None):
    """Times every FP64 product tile shape per tree level on this input
    (tdc_autotune) and records the fastest; later solves of the same tree structure
    with tile_cfg = -1 use it.  Returns the shape index per level (leaves to root)."""
    lib = _lib.load()
    n = int(d.shape[0])
    assert d.dtype == torch.float64 and d.is_cuda and d.is_contiguous()
    assert e.dtype == torch.float64 and e.is_cuda and e.is_contiguous() and e.shape[0] == max(n - 1, 0)
    o = _opts(opts)
    lam = torch.empty(n, dtype=torch.float64, device=d.device)
    q = fortran_empty(n, n, d.device)
    nb = lib.tdc_workspace_bytes(n, ctypes.byref(o))
    if nb == 0:
        raise ValueError("invalid size or options")
    ws = workspace(nb, d.device)
    st = torch.zeros(1, dtype=torch.int32, device=d.device)
    shapes = (ctypes.c_int32 * 64)()
    nl = ctypes.c_int32(0)
    rc = lib.tdc_autotune(n, _vp(d), _vp(e if n > 1 else None), _vp(lam), _vp(q), n, ctypes.byref(o), _vp(ws),
                          ws.numel(), shapes, 64, ctypes.byref(nl), _vp(st), _stream(stream))
    _check_rc(rc, "tdc_autotune")
    _raise_status(lib.tdc_read_status(_vp(st), _stream(stream)), "tdc_autotune")
    return [int(shapes[i]) for i in range(min(nl.value, 64))]


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


TRACE_INT32 = ("perm", "kept", "deflated", "rot_j", "rot_k", "origin")


def merge_inspect(D: torch.Tensor, Q: torch.Tensor, n1: int, beta: float, opts=None, stream=None):
    """tdc_merge plus the merge's intermediate values (tdc_merge_inspect).  Returns
    (lam, Q_out, trace) with trace a dict of host numpy arrays cut to their defined
    lengths: counts (K, nd, nrot, c1, c3, type-1 count), perm, d_sorted, z_sorted,
    kept, deflated, rot_j, rot_k, rot_c, rot_s, dbar, zbar, origin, tau, zhat, sinv,
    tau_lo (zeros unless opts.eigvec is extended)."""
    lib = _lib.load()
    n = int(D.shape[0])
    assert Q.stride() == (1, n) and Q.shape == (n, n) and Q.dtype == torch.float64
    o = _opts(opts)
    dev = D.device
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    qo = fortran_empty(n, n, dev)
    bufs = {"counts": torch.zeros(8, dtype=torch.int64, device=dev)}
    tr = _lib.TdcMergeTrace()
    for name, _ in _lib.TdcMergeTrace._fields_:
        if name == "counts":
            continue
        bufs[name] = torch.zeros(n, dtype=torch.int32 if name in TRACE_INT32 else torch.float64, device=dev)
    for name, t in bufs.items():
        setattr(tr, name, t.data_ptr())
    nb = lib.tdc_merge_workspace_bytes(n, ctypes.byref(o))
    if nb == 0:
        raise ValueError("invalid size or options")
    ws = workspace(nb, dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = lib.tdc_merge_inspect(int(n1), int(n - n1), _vp(D), _vp(Q), n, float(beta), _vp(lam), _vp(qo), n,
                               None, ctypes.byref(o), _vp(ws), ws.numel(), _vp(st), _stream(stream),
                               ctypes.byref(tr))
    _check_rc(rc, "tdc_merge_inspect")
    _raise_status(lib.tdc_read_status(_vp(st), _stream(stream)), "tdc_merge_inspect")
    h = {k: v.cpu().numpy() for k, v in bufs.items()}
    K, nd, nrot = int(h["counts"][0]), int(h["counts"][1]), int(h["counts"][2])
    cut = {"perm": n, "d_sorted": n, "z_sorted": n, "kept": K, "deflated": nd, "rot_j": nrot, "rot_k": nrot,
           "rot_c": nrot, "rot_s": nrot, "dbar": K, "zbar": K, "origin": K, "tau": K, "zhat": K, "sinv": K,
           "tau_lo": K}
    for k, m in cut.items():
        h[k] = h[k][:m]
    return lam, qo, h


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


class HostPipeline:
    """A stream of problems of one order n solved from and to host memory with `depth`
    solves in flight.  Each slot holds a one-problem batched plan (built and uploaded
    once), its device arrays, page-locked inputs and outputs and a stream; submit()
    enqueues tdc_batched_plan_execute_host on the slot's stream (copy in, execute, copy
    out, no pageable copy), so the copy-out of one problem overlaps the solve of the
    next.  submit() returns the slot holding that problem's result; result(slot) waits
    for it."""

    def __init__(self, n: int, depth: int = 2, opts=None, device=None):
        self.lib = _lib.load()
        self.n = n
        self.depth = depth
        dev = device or "cuda"
        self.plans = [BatchedPlan([n], opts=opts, device=dev) for _ in range(depth)]
        f64 = dict(dtype=torch.float64)
        self.d_dev = [torch.empty(n, device=dev, **f64) for _ in range(depth)]
        self.e_dev = [torch.empty(n, device=dev, **f64) for _ in range(depth)]
        self.lam_dev = [torch.empty(n, device=dev, **f64) for _ in range(depth)]
        self.q_dev = [torch.empty(n * n, device=dev, **f64) for _ in range(depth)]
        self.d_in = [torch.empty(n, **f64).pin_memory() for _ in range(depth)]
        self.e_in = [torch.zeros(n, **f64).pin_memory() for _ in range(depth)]
        self.lam = [torch.empty(n, **f64).pin_memory() for _ in range(depth)]
        self.q = [torch.empty(n * n, **f64).pin_memory() for _ in range(depth)]
        self.status = torch.zeros(depth, dtype=torch.int32).pin_memory()
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(depth)]
        self.events = [None] * depth
        self.k = 0

    def _finish(self, s):
        if self.events[s] is not None:
            self.events[s].synchronize()
            self.events[s] = None
            _raise_status(int(self.status[s]), "tdc_batched_plan_execute_host")

    def submit(self, d_host: torch.Tensor, e_host: torch.Tensor) -> int:
        s = self.k % self.depth
        self.k += 1
        self._finish(s)                                   # the slot's previous problem
        n = self.n
        self.d_in[s].copy_(torch.as_tensor(d_host, dtype=torch.float64).reshape(-1)[:n])
        if n > 1:
            self.e_in[s][:n - 1].copy_(torch.as_tensor(e_host, dtype=torch.float64).reshape(-1)[:n - 1])
        p = self.plans[s]
        rc = self.lib.tdc_batched_plan_execute_host(
            p.handle, _vp(self.d_in[s]), _vp(self.e_in[s]), _vp(self.lam[s]), _vp(self.q[s]),
            ctypes.c_void_p(self.status.data_ptr() + 4 * s), _vp(self.d_dev[s]), _vp(self.e_dev[s]),
            _vp(self.lam_dev[s]), _vp(self.q_dev[s]), _vp(p.status), _stream(self.streams[s]))
        _check_rc(rc, "tdc_batched_plan_execute_host")
        ev = torch.cuda.Event()
        ev.record(self.streams[s])
        self.events[s] = ev
        return s

    def result(self, s: int):
        self._finish(s)
        return self.lam[s], self.q[s].view(self.n, self.n).t()

    def wait_all(self):
        for s in range(self.depth):
            self._finish(s)

    @property
    def h2d_bytes(self):
        return 8 * 2 * self.n

    @property
    def d2h_bytes(self):
        return 8 * (self.n + self.n * self.n)


def syev_backward(lam: torch.Tensor, q: torch.Tensor, g_lam=None, g_q=None, stream=None, opts=None):
    """(g_d, g_e) of a loss with gradients (g_lam, g_q) at the output (lam, q) of
    syev_tridiag, through tdc_syev_tridiag_backward (band-only adjoint).  opts with
    path 1 runs its two products with Q on the split-precision tensor-core path."""
    lib = _lib.load()
    n = int(lam.shape[0])
    if g_q is not None and g_q.stride() != (1, n):
        g_q = g_q.t().contiguous().t()                 # column-major layout expected by the ABI
    gd = torch.empty(n, dtype=torch.float64, device=lam.device)
    ge = torch.empty(max(n - 1, 0), dtype=torch.float64, device=lam.device)
    o = _opts(opts) if opts is not None else None
    op = ctypes.byref(o) if o is not None else None
    nb = lib.tdc_backward_workspace_bytes(n, op)
    ws = workspace(nb, lam.device, key="backward")
    rc = lib.tdc_syev_tridiag_backward(n, _vp(lam), _vp(q), n, _vp(g_lam), _vp(g_q), n, _vp(gd),
                                       _vp(ge if n > 1 else None), op, _vp(ws), ws.numel(), None,
                                       _stream(stream))
    _check_rc(rc, "tdc_syev_tridiag_backward")
    return gd, ge


def syev_backward_batched(sizes, lam_cat: torch.Tensor, q_cat: torch.Tensor, g_lam_cat=None, g_q_cat=None,
                          max_cols: int = -1, stream=None, opts=None):
    """(g_d_cat, g_e_cat) for a batch in the batched forward's dense packing
    (tdc_syev_tridiag_backward_batched): lam_cat / g_lam_cat hold sum(n) values,
    q_cat / g_q_cat the n_p x n_p column-major blocks back to back; g_e_cat holds
    problem p's n_p - 1 entries at the same offset as its d (its last slot is zero)."""
    lib = _lib.load()
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    b = len(sizes)
    dev = lam_cat.device
    tot = int(sizes.sum())
    gd = torch.empty(tot, dtype=torch.float64, device=dev)
    ge = torch.zeros(tot, dtype=torch.float64, device=dev)
    sp = sizes.ctypes.data_as(ctypes.c_void_p)
    o = _opts(opts) if opts is not None else None
    op = ctypes.byref(o) if o is not None else None
    nb = lib.tdc_backward_batched_workspace_bytes(b, sp, int(max_cols), op)
    if nb == 0:
        raise ValueError("invalid sizes")
    ws = workspace(nb, dev, key="backward_batched")
    rc = lib.tdc_syev_tridiag_backward_batched(b, sp, _vp(lam_cat), _vp(q_cat), _vp(g_lam_cat), _vp(g_q_cat),
                                               _vp(gd), _vp(ge), op, _vp(ws), ws.numel(), None, _stream(stream))
    _check_rc(rc, "tdc_syev_tridiag_backward_batched")
    return gd, ge


class TridiagEigh(torch.autograd.Function):
    """(lam, Q) = eigh of tridiag(e, d, e) with a hand-written backward: the forward
    saves only (lam, Q); the backward recomputes nothing of the merge tree."""

    @staticmethod
    def forward(ctx, d, e, opts=None):
        lam, q = syev_tridiag(d.detach().contiguous(), e.detach().contiguous(), opts=opts)
        ctx.save_for_backward(lam, q)
        ctx.opts = opts
        return lam, q

    @staticmethod
    def backward(ctx, g_lam, g_q):
        lam, q = ctx.saved_tensors
        gd, ge = syev_backward(lam, q, g_lam, g_q, opts=ctx.opts)
        return gd, ge, None


def eigh_tridiag(d: torch.Tensor, e: torch.Tensor, opts=None):
    """Differentiable eigendecomposition of tridiag(e, d, e) (FP64, CUDA tensors)."""
    return TridiagEigh.apply(d, e, opts)


class BatchedPlan:
    """A ragged batch solved repeatedly: tdc_batched_plan_create once, then
    execute (kernel launches only) directly or from a captured CUDA graph."""

    def __init__(self, sizes, opts=None, device=None):
        self.lib = _lib.load()
        self.sizes = np.asarray(sizes, dtype=np.int64)
        self.o = _opts(opts)
        dev = torch.device(device or "cuda")
        b = len(self.sizes)
        nb = self.lib.tdc_batched_workspace_bytes(b, self.sizes.ctypes.data_as(ctypes.c_void_p),
                                                  ctypes.byref(self.o))
        if nb == 0:
            raise ValueError("invalid sizes or options")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.handle = ctypes.c_void_p()
        rc = self.lib.tdc_batched_plan_create(b, self.sizes.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.o),
                                              _vp(self.ws), nb, _stream(None), ctypes.byref(self.handle))
        _check_rc(rc, "tdc_batched_plan_create")
        self.off = np.zeros(b, dtype=np.int64)
        self.off[1:] = np.cumsum(self.sizes)[:-1]
        self.qoff = np.zeros(b, dtype=np.int64)
        self.qoff[1:] = np.cumsum(self.sizes * self.sizes)[:-1]
        self.status = torch.zeros(b, dtype=torch.int32, device=dev)
        self.graph = None

    def pack(self, ds, es, device="cuda"):
        d_cat = torch.cat([torch.as_tensor(x, dtype=torch.float64) for x in ds]).to(device)
        e_cat = torch.zeros(int(self.sizes.sum()), dtype=torch.float64)
        for p, n in enumerate(self.sizes):
            if n > 1:
                e_cat[self.off[p]:self.off[p] + n - 1] = torch.as_tensor(es[p], dtype=torch.float64)
        return d_cat, e_cat.to(device)

    def outputs(self, device="cuda"):
        lam = torch.empty(int(self.sizes.sum()), dtype=torch.float64, device=device)
        q = torch.empty(int((self.sizes * self.sizes).sum()), dtype=torch.float64, device=device)
        return lam, q

    def execute(self, d_cat, e_cat, lam, q, stream=None):
        rc = self.lib.tdc_batched_plan_execute(self.handle, _vp(d_cat), _vp(e_cat), _vp(lam), _vp(q),
                                               _vp(self.status), _stream(stream))
        _check_rc(rc, "tdc_batched_plan_execute")

    def autotune(self, d_cat, e_cat, lam, q, stream=None):
        """Tunes the plan's FP64 product tile shape per level (before capture).
        Returns the shape index per level."""
        shapes = (ctypes.c_int32 * 64)()
        nl = ctypes.c_int32(0)
        rc = self.lib.tdc_batched_plan_autotune(self.handle, _vp(d_cat), _vp(e_cat), _vp(lam), _vp(q), shapes, 64,
                                                ctypes.byref(nl), _stream(stream))
        _check_rc(rc, "tdc_batched_plan_autotune")
        return [int(shapes[i]) for i in range(min(nl.value, 64))]

    def execute_persistent(self, d_cat, e_cat, lam, q, stream=None):
        """The same solve in one persistent kernel launch (tdc_batched_plan_execute_persistent:
        each CTA takes whole problems from a work queue; FP64 product plans only)."""
        rc = self.lib.tdc_batched_plan_execute_persistent(self.handle, _vp(d_cat), _vp(e_cat), _vp(lam), _vp(q),
                                                          _vp(self.status), _stream(stream))
        _check_rc(rc, "tdc_batched_plan_execute_persistent")

    def capture(self, d_cat, e_cat, lam, q, persistent=False):
        """Captures one execute (or one persistent execute) on these buffers into a CUDA
        graph (after a warm-up)."""
        if persistent:
            self.execute_persistent(d_cat, e_cat, lam, q)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.execute_persistent(d_cat, e_cat, lam, q)
            self.graph = g
            return
        self.execute(d_cat, e_cat, lam, q)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.execute(d_cat, e_cat, lam, q)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def __del__(self):
        try:
            if self.handle:
                self.lib.tdc_batched_plan_destroy(self.handle)
        except Exception:
            pass
