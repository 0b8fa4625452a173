"""Python binding of ``include/ib.h`` (ctypes; argument marshalling only).

Every entry point of the C ABI is exposed under the same name.  Tensors are
passed as raw device pointers on torch's current CUDA stream; nothing is
computed here.  The library must have been built (``build_lib.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibwave.so")

IB_OK, IB_ERR_ARG, IB_ERR_RANK, IB_ERR_CUDA, IB_ERR_OOM, IB_ERR_UNSTABLE, IB_ERR_TIMEOUT, IB_ERR_STATE = range(8)
FREE, RIGID = 0, 1
SECOND_ORDER, FIRST_ORDER_STAGGERED = 0, 1

EXPORTS = ["ib_opts_default", "ib_build_stencils", "ib_table_free", "ib_table_stats", "ib_table_export",
           "ib_forward", "ib_checkpoint_bytes", "ib_adjoint", "ib_forward_batch", "ib_sync_status",
           "ib_last_error", "ib_version", "ib_profile_enable", "ib_profile_count", "ib_profile_get",
           "ib_forward_noalloc"]


class IbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("ib status %d: %s" % (status, msg))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("space_order", ctypes.c_int32), ("basis_order", ctypes.c_int32),
                ("min_order", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("radius", ctypes.c_double), ("growth", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("eta_v", ctypes.c_double),
                ("rank_tol", ctypes.c_double)]


class TableInfo(ctypes.Structure):
    _fields_ = [("n_ops", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("rows", ctypes.c_int64 * 8), ("nnz", ctypes.c_int64 * 8),
                ("n_boundary_points", ctypes.c_int64), ("n_rank_failures", ctypes.c_int64),
                ("n_grown", ctypes.c_int64), ("n_reduced", ctypes.c_int64),
                ("table_bytes", ctypes.c_int64), ("setup_seconds", ctypes.c_double)]


class Shot(ctypes.Structure):
    _fields_ = [("vel_dev", ctypes.c_void_p), ("rho_dev", ctypes.c_void_p),
                ("src_dev", ctypes.c_void_p), ("rec_dev", ctypes.c_void_p),
                ("wavelet_dev", ctypes.c_void_p), ("traces_dev", ctypes.c_void_p),
                ("nsrc", ctypes.c_int32), ("nrec", ctypes.c_int32)]


_LIB = None


def load(path=LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("libibwave.so not built (run __graft_entry__.build()): %s" % path)
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.ib_opts_default.argtypes = [ctypes.POINTER(Opts), i32]
    L.ib_opts_default.restype = None
    L.ib_build_stencils.argtypes = [ctypes.POINTER(Grid), vp, i32, i32, ctypes.POINTER(Opts),
                                    ctypes.POINTER(vp), vp]
    L.ib_build_stencils.restype = i32
    L.ib_table_free.argtypes = [vp]
    L.ib_table_free.restype = None
    L.ib_table_stats.argtypes = [vp, ctypes.POINTER(TableInfo)]
    L.ib_table_stats.restype = i32
    L.ib_table_export.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.ib_table_export.restype = i32
    L.ib_forward.argtypes = [vp, ctypes.POINTER(Shot), i32, dbl, i32, vp, i32, vp]
    L.ib_forward.restype = i32
    L.ib_checkpoint_bytes.argtypes = [vp, i32, i32, i32]
    L.ib_checkpoint_bytes.restype = i64
    L.ib_adjoint.argtypes = [vp, ctypes.POINTER(Shot), i32, dbl, i32, vp, i32, vp, vp, vp, vp]
    L.ib_adjoint.restype = i32
    L.ib_forward_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Shot), i32, i32, dbl, i32, vp]
    L.ib_forward_batch.restype = i32
    L.ib_sync_status.argtypes = [vp]
    L.ib_sync_status.restype = i32
    L.ib_last_error.argtypes = []
    L.ib_last_error.restype = ctypes.c_char_p
    L.ib_version.argtypes = []
    L.ib_version.restype = ctypes.c_char_p
    L.ib_profile_enable.argtypes = [i32]
    L.ib_profile_enable.restype = i32
    L.ib_profile_count.argtypes = []
    L.ib_profile_count.restype = i32
    L.ib_profile_get.argtypes = [i32, ctypes.c_char_p, i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                 ctypes.POINTER(dbl)]
    L.ib_profile_get.restype = i32
    L.ib_forward_noalloc.argtypes = [vp, ctypes.POINTER(Shot), dbl, i32, vp]
    L.ib_forward_noalloc.restype = i32
    _LIB = L
    return L


def _check(st, allow=()):
    if st != IB_OK and st not in allow:
        raise IbError(st, load().ib_last_error().decode())
    return st


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def ib_opts_default(space_order):
    o = Opts()
    load().ib_opts_default(ctypes.byref(o), int(space_order))
    return o


class Table:
    """Owner of an ``ib_table*``."""

    def __init__(self, handle, ndim, shape, h, form, status):
        self.handle = handle
        self.ndim = ndim
        self.shape = shape          # array shape [nz][nx] or [nz][ny][nx]
        self.h = h
        self.form = form
        self.status = status

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.ib_table_free(self.handle)
            self.handle = None

    def stats(self):
        return ib_table_stats(self)

    def export(self, op):
        return ib_table_export(self, op)


def ib_build_stencils(sdf, h, bc="free", form="second", space_order=4, opts=None, stream=None,
                      allow_rank_failure=False):
    """sdf: CUDA float64 tensor [nz][nx] or [nz][ny][nx] (metres, > 0 inside)."""
    L = load()
    assert sdf.is_cuda and sdf.dtype == torch.float64 and sdf.is_contiguous()
    g = Grid()
    g.ndim = sdf.dim()
    rev = list(reversed(sdf.shape))
    for a in range(3):
        g.n[a] = rev[a] if a < len(rev) else 1
    g.h = float(h)
    o = opts if opts is not None else ib_opts_default(space_order)
    o.space_order = int(space_order)
    handle = ctypes.c_void_p()
    fm = SECOND_ORDER if form in ("second", SECOND_ORDER) else FIRST_ORDER_STAGGERED
    b = FREE if bc in ("free", FREE) else RIGID
    st = L.ib_build_stencils(ctypes.byref(g), _ptr(sdf), b, fm, ctypes.byref(o), ctypes.byref(handle),
                             _stream(stream))
    if st != IB_OK and not (allow_rank_failure and st == IB_ERR_RANK and handle.value):
        if handle.value:
            L.ib_table_free(handle)
        _check(st)
    return Table(handle, g.ndim, tuple(sdf.shape), float(h), fm, st)


def ib_table_stats(table):
    info = TableInfo()
    _check(load().ib_table_stats(table.handle, ctypes.byref(info)))
    n = info.n_ops
    return dict(n_ops=n, rows=list(info.rows[:n]), nnz=list(info.nnz[:n]),
                n_boundary_points=info.n_boundary_points, n_rank_failures=info.n_rank_failures,
                n_grown=info.n_grown, n_reduced=info.n_reduced, table_bytes=info.table_bytes,
                setup_seconds=info.setup_seconds)


def ib_table_export(table, op):
    st = ib_table_stats(table)
    nr, nz = st["rows"][op], st["nnz"][op]
    row_node = np.zeros(max(nr, 1), np.int64)
    row_ptr = np.zeros(nr + 1, np.int64)
    col = np.zeros((max(nz, 1), 3), np.int32)
    w = np.zeros(max(nz, 1), np.float64)
    info = np.zeros((max(nr, 1), 4), np.int32)
    c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().ib_table_export(table.handle, int(op), c(row_node), c(row_ptr), c(col), c(w), c(info)))
    return dict(row_node=row_node[:nr], row_ptr=row_ptr, col=col[:nz], w=w[:nz], info=info[:nr])


def _shot(vel, rho, src, rec, wavelet, traces):
    s = Shot()
    s.vel_dev = vel.data_ptr()
    s.rho_dev = rho.data_ptr() if rho is not None else None
    s.src_dev = src.data_ptr() if src is not None and src.numel() else None
    s.rec_dev = rec.data_ptr() if rec is not None and rec.numel() else None
    s.wavelet_dev = wavelet.data_ptr() if wavelet is not None else None
    s.traces_dev = traces.data_ptr() if traces is not None and traces.numel() else None
    s.nsrc = src.shape[0] if src is not None else 0
    s.nrec = rec.shape[0] if rec is not None else 0
    return s


def _prec(dtype):
    return 64 if dtype == torch.float64 else 32


def ib_checkpoint_bytes(table, precision, nt, n_ckpt):
    return int(load().ib_checkpoint_bytes(table.handle, int(precision), int(nt), int(n_ckpt)))


def ib_forward(table, vel, wavelet, src, rec, dt, nt, rho=None, ckpt=None, n_ckpt=0, traces=None,
               stream=None):
    """vel, rho, wavelet: CUDA tensors of one float dtype (its precision is used);
    src, rec: CUDA float64 [n][ndim] metres.  Returns traces [nrec][nt]."""
    for t in (vel, wavelet):
        assert t.is_cuda and t.is_contiguous()
    if traces is None:
        traces = torch.zeros((rec.shape[0], nt), dtype=vel.dtype, device=vel.device)
    sh = _shot(vel, rho, src, rec, wavelet, traces)
    _check(load().ib_forward(table.handle, ctypes.byref(sh), _prec(vel.dtype), float(dt), int(nt),
                             _ptr(ckpt), int(n_ckpt), _stream(stream)))
    return traces


def ib_adjoint(table, vel, wavelet, src, rec, dt, nt, ckpt, n_ckpt, residual, want_wavelet_grad=False,
               stream=None):
    """Returns (dJ/dvel [same shape as vel], dJ/dwavelet [nt] or None)."""
    grad = torch.zeros_like(vel)
    gw = torch.zeros(nt, dtype=vel.dtype, device=vel.device) if want_wavelet_grad else None
    sh = _shot(vel, None, src, rec, wavelet, None)
    _check(load().ib_adjoint(table.handle, ctypes.byref(sh), _prec(vel.dtype), float(dt), int(nt),
                             _ptr(ckpt), int(n_ckpt), _ptr(residual.contiguous()), _ptr(grad), _ptr(gw),
                             _stream(stream)))
    return grad, gw


def ib_forward_noalloc(table, vel, wavelet, src, rec, dt, nt, traces, stream=None):
    """ib_forward (2D second-order, FP32) with the library's static scratch: no
    device allocation inside the call; `traces` [nrec][nt] float32 is caller-owned."""
    sh = _shot(vel, None, src, rec, wavelet, traces)
    _check(load().ib_forward_noalloc(table.handle, ctypes.byref(sh), float(dt), int(nt), _stream(stream)))
    return traces


def ib_forward_batch(tables, shots, dt, nt, stream=None):
    """shots: list of dicts with vel, wavelet, src, rec (and traces out)."""
    n = len(tables)
    arr = (ctypes.c_void_p * n)(*[t.handle.value for t in tables])
    sh = (Shot * n)()
    outs = []
    for i, d in enumerate(shots):
        tr = d.get("traces")
        if tr is None:
            tr = torch.zeros((d["rec"].shape[0], nt), dtype=d["vel"].dtype, device=d["vel"].device)
        outs.append(tr)
        sh[i] = _shot(d["vel"], d.get("rho"), d["src"], d["rec"], d["wavelet"], tr)
    _check(load().ib_forward_batch(arr, sh, n, 32, float(dt), int(nt), _stream(stream)))
    return outs


def ib_sync_status(stream=None):
    return _check(load().ib_sync_status(_stream(stream)))


def ib_last_error():
    return load().ib_last_error().decode()


def ib_version():
    return load().ib_version().decode()


def ib_profile_enable(stride):
    return _check(load().ib_profile_enable(int(stride)))


def ib_profile_count():
    return int(load().ib_profile_count())


def ib_profile_get(i):
    name = ctypes.create_string_buffer(64)
    la, sa = ctypes.c_int64(), ctypes.c_int64()
    ms = ctypes.c_double()
    _check(load().ib_profile_get(int(i), name, 64, ctypes.byref(la), ctypes.byref(sa), ctypes.byref(ms)))
    return dict(name=name.value.decode(), launches=la.value, sampled=sa.value, sampled_ms=ms.value)


def ib_profile():
    """All kernels seen since the last ib_profile_enable: name -> counters."""
    return {d["name"]: d for d in (ib_profile_get(i) for i in range(ib_profile_count()))}


class Forward(torch.autograd.Function):
    """traces = F(vel) through the library; backward calls ib_adjoint.

    Usage: Forward.apply(vel, table, wavelet, src, rec, dt, nt, n_ckpt)."""

    @staticmethod
    def forward(ctx, vel, table, wavelet, src, rec, dt, nt, n_ckpt):
        prec = _prec(vel.dtype)
        nbytes = ib_checkpoint_bytes(table, prec, nt, n_ckpt)
        ckpt = torch.empty(nbytes, dtype=torch.uint8, device=vel.device)
        traces = ib_forward(table, vel.contiguous(), wavelet, src, rec, dt, nt, ckpt=ckpt, n_ckpt=n_ckpt)
        ctx.save_for_backward(vel, wavelet, src, rec, ckpt)
        ctx.table, ctx.dt, ctx.nt, ctx.n_ckpt = table, dt, nt, n_ckpt
        return traces

    @staticmethod
    def backward(ctx, grad_traces):
        vel, wavelet, src, rec, ckpt = ctx.saved_tensors
        g, _ = ib_adjoint(ctx.table, vel.contiguous(), wavelet, src, rec, ctx.dt, ctx.nt, ckpt, ctx.n_ckpt,
                          grad_traces.contiguous())
        return g, None, None, None, None, None, None, None
