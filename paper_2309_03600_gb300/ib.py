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
EXTRAP_ND, EXTRAP_1D = 0, 1
SECOND_ORDER, FIRST_ORDER_STAGGERED = 0, 1

EXPORTS = ["ib_opts_default", "ib_build_stencils", "ib_table_free", "ib_table_stats", "ib_table_export",
           "ib_forward", "ib_checkpoint_bytes", "ib_adjoint", "ib_forward_batch", "ib_sync_status",
           "ib_last_error", "ib_version", "ib_profile_enable", "ib_profile_count", "ib_profile_get",
           "ib_forward_noalloc", "ib_mlp_create", "ib_mlp_free", "ib_mlp_info", "ib_mlp_buffers",
           "ib_mlp_sync_weights", "ib_mlp_features", "ib_mlp_forward", "ib_mlp_train_step",
           "ib_mlp_targets", "ib_build_stencils_learned", "ib_table_learned", "ib_forward_batch_ckpt",
           "ib_adjoint_batch", "ib_selftest_bounded_wait", "ib_stability"]


class IbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("ib status %d: %s" % (status, msg))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("space_order", ctypes.c_int32), ("basis_order", ctypes.c_int32),
                ("min_order", ctypes.c_int32), ("extrapolation", ctypes.c_int32),
                ("radius", ctypes.c_double), ("growth", ctypes.c_double),
                ("eta_p", ctypes.c_double), ("eta_v", ctypes.c_double),
                ("rank_tol", ctypes.c_double)]


class TableInfo(ctypes.Structure):
    _fields_ = [("n_ops", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("rows", ctypes.c_int64 * 8), ("nnz", ctypes.c_int64 * 8),
                ("n_boundary_points", ctypes.c_int64), ("n_rank_failures", ctypes.c_int64),
                ("n_grown", ctypes.c_int64), ("n_reduced", ctypes.c_int64),
                ("table_bytes", ctypes.c_int64), ("setup_seconds", ctypes.c_double)]


class MlpConfig(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("space_order", ctypes.c_int32),
                ("n_hidden", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("in_radius", ctypes.c_double), ("out_radius", ctypes.c_double)]


class Shot(ctypes.Structure):
    _fields_ = [("vel_dev", ctypes.c_void_p), ("rho_dev", ctypes.c_void_p),
                ("src_dev", ctypes.c_void_p), ("rec_dev", ctypes.c_void_p),
                ("wavelet_dev", ctypes.c_void_p), ("traces_dev", ctypes.c_void_p),
                ("nsrc", ctypes.c_int32), ("nrec", ctypes.c_int32),
                ("damp_eta", ctypes.c_double), ("damp_width", ctypes.c_int32), ("reserved", ctypes.c_int32)]


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
    L.ib_forward_batch_ckpt.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Shot), i32, i32, dbl, i32,
                                        ctypes.POINTER(vp), i32, vp]
    L.ib_forward_batch_ckpt.restype = i32
    L.ib_adjoint_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Shot), i32, i32, dbl, i32,
                                   ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.ib_adjoint_batch.restype = i32
    L.ib_selftest_bounded_wait.argtypes = [vp]
    L.ib_selftest_bounded_wait.restype = i32
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
    fp = ctypes.POINTER(vp)
    L.ib_mlp_create.argtypes = [ctypes.POINTER(MlpConfig), fp]
    L.ib_mlp_create.restype = i32
    L.ib_mlp_free.argtypes = [vp]
    L.ib_mlp_free.restype = None
    L.ib_mlp_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.ib_mlp_info.restype = i32
    L.ib_mlp_buffers.argtypes = [vp, fp, fp, fp, fp]
    L.ib_mlp_buffers.restype = i32
    L.ib_mlp_sync_weights.argtypes = [vp, vp]
    L.ib_mlp_sync_weights.restype = i32
    L.ib_mlp_features.argtypes = [vp, ctypes.POINTER(Grid), vp, vp, i64, i32, vp, vp]
    L.ib_mlp_features.restype = i32
    L.ib_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    L.ib_mlp_forward.restype = i32
    L.ib_mlp_train_step.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, vp, vp]
    L.ib_mlp_train_step.restype = i32
    L.ib_mlp_targets.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(i64), vp]
    L.ib_mlp_targets.restype = i32
    L.ib_build_stencils_learned.argtypes = [ctypes.POINTER(Grid), vp, i32, ctypes.POINTER(Opts), vp, dbl,
                                            fp, vp]
    L.ib_build_stencils_learned.restype = i32
    L.ib_table_learned.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
    L.ib_table_learned.restype = i32
    L.ib_stability.argtypes = [vp, ctypes.POINTER(Shot), i32, dbl, i32, ctypes.c_uint64, dbl, ctypes.POINTER(dbl), vp]
    L.ib_stability.restype = i32
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


def _grid(sdf, h):
    g = Grid()
    g.ndim = sdf.dim()
    rev = list(reversed(sdf.shape))
    for a in range(3):
        g.n[a] = rev[a] if a < len(rev) else 1
    g.h = float(h)
    return g


def ib_build_stencils_learned(sdf, h, mlp, bc="free", space_order=4, accept_tol=1e-6, opts=None,
                              stream=None):
    """Second-order table whose rows take the network's prediction where it is
    exact to ``accept_tol`` and the constrained fit elsewhere."""
    L = load()
    assert sdf.is_cuda and sdf.dtype == torch.float64 and sdf.is_contiguous()
    g = _grid(sdf, h)
    o = opts if opts is not None else ib_opts_default(space_order)
    o.space_order = int(space_order)
    handle = ctypes.c_void_p()
    b = FREE if bc in ("free", FREE) else RIGID
    st = L.ib_build_stencils_learned(ctypes.byref(g), _ptr(sdf), b, ctypes.byref(o), mlp.handle,
                                     float(accept_tol), ctypes.byref(handle), _stream(stream))
    if st != IB_OK:
        if handle.value:
            L.ib_table_free(handle)
        _check(st)
    return Table(handle, g.ndim, tuple(sdf.shape), float(h), SECOND_ORDER, st)


def ib_table_learned(table):
    """(rows checked, rows accepted, per-row residual as numpy)."""
    nr = ib_table_stats(table)["rows"][0] if ib_table_stats(table)["n_ops"] else 0
    res = np.full(max(nr, 1), np.nan)
    c, a = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ib_table_learned(table.handle, ctypes.byref(c), ctypes.byref(a),
                                   res.ctypes.data_as(ctypes.c_void_p)))
    return c.value, a.value, res[:nr]


class Mlp:
    """Owner of an ``ib_mlp*`` (learned stencil network on the current device)."""

    def __init__(self, ndim, space_order, n_hidden=256, n_layers=4, in_radius=4.0, out_radius=None):
        L = load()
        cfg = MlpConfig()
        cfg.ndim = int(ndim)
        cfg.space_order = int(space_order)
        cfg.n_hidden = int(n_hidden)
        cfg.n_layers = int(n_layers)
        cfg.in_radius = float(in_radius)
        cfg.out_radius = float(out_radius if out_radius is not None else (min(space_order, 4) + 1) / 2.0)
        self.cfg = cfg
        h = ctypes.c_void_p()
        _check(L.ib_mlp_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        n_in, n_out, n_par = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(L.ib_mlp_info(h, ctypes.byref(n_in), ctypes.byref(n_out), ctypes.byref(n_par)))
        self.n_in, self.n_out, self.n_params = n_in.value, n_out.value, n_par.value

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.ib_mlp_free(self.handle)
            self.handle = None

    def buffers(self):
        """Library-owned device buffers as torch views: params, grads, adam_m, adam_v."""
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        _check(load().ib_mlp_buffers(self.handle, *[ctypes.byref(p) for p in ptrs]))
        out = []
        for p in ptrs:
            out.append(_device_view(p.value, self.n_params))
        return out

    def set_params(self, values, stream=None):
        params = self.buffers()[0]
        params.copy_(torch.as_tensor(values, dtype=torch.float32, device=params.device))
        _check(load().ib_mlp_sync_weights(self.handle, _stream(stream)))


def _device_view(ptr, n):
    """torch float32 view of n library-owned device floats (no copy)."""
    class _Arr:
        pass
    a = _Arr()
    a.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f4", "data": (int(ptr), False),
                                  "version": 3, "strides": None}
    return torch.as_tensor(a, device="cuda")


def ib_mlp_features(mlp, sdf, h, nodes, bc="free", stream=None):
    """bfloat16 features [n][n_in] of the nodes (int64 linear indices)."""
    assert nodes.dtype == torch.int64 and nodes.is_cuda
    X = torch.empty((nodes.numel(), mlp.n_in), dtype=torch.bfloat16, device=sdf.device)
    b = FREE if bc in ("free", FREE) else RIGID
    _check(load().ib_mlp_features(mlp.handle, ctypes.byref(_grid(sdf, h)), _ptr(sdf), _ptr(nodes),
                                  int(nodes.numel()), b, _ptr(X), _stream(stream)))
    return X


def ib_mlp_forward(mlp, X, stream=None):
    assert X.dtype == torch.bfloat16 and X.is_contiguous() and X.shape[1] == mlp.n_in
    Y = torch.empty((X.shape[0], mlp.n_out), dtype=torch.float32, device=X.device)
    _check(load().ib_mlp_forward(mlp.handle, _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)))
    return Y


def ib_mlp_train_step(mlp, X, T, idx, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=None, stream=None):
    """One Adam step on rows idx of (X, T); returns the device loss tensor."""
    assert X.dtype == torch.bfloat16 and T.dtype == torch.float32 and idx.dtype == torch.int64
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(load().ib_mlp_train_step(mlp.handle, _ptr(X), _ptr(T), _ptr(idx), int(idx.numel()), float(lr),
                                    float(beta1), float(beta2), float(eps), _ptr(loss), _stream(stream)))
    return loss


def ib_mlp_targets(table, mlp, stream=None):
    """(nodes int64 [n], targets float32 [n][n_out]) of the table's trainable rows."""
    nr = ib_table_stats(table)["rows"][0]
    dev = torch.device("cuda", torch.cuda.current_device())
    nodes = torch.empty(max(nr, 1), dtype=torch.int64, device=dev)
    T = torch.empty((max(nr, 1), mlp.n_out), dtype=torch.float32, device=dev)
    n = ctypes.c_int64()
    _check(load().ib_mlp_targets(table.handle, mlp.handle, _ptr(nodes), _ptr(T), int(nr), ctypes.byref(n),
                                 _stream(stream)))
    return nodes[:n.value], T[:n.value]


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


def _shot(vel, rho, src, rec, wavelet, traces, damp=None):
    """damp: None or (width in nodes, eta_max in 1/s) of the absorbing layer."""
    s = Shot()
    if damp is not None:
        s.damp_width = int(damp[0])
        s.damp_eta = float(damp[1])
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
               damp=None, stream=None):
    """vel, rho, wavelet: CUDA tensors of one float dtype (its precision is used);
    src, rec: CUDA float64 [n][ndim] metres; damp: None or (width, eta_max) of
    the absorbing layer.  Returns traces [nrec][nt]."""
    for t in (vel, wavelet):
        assert t.is_cuda and t.is_contiguous()
    if traces is None:
        traces = torch.zeros((rec.shape[0], nt), dtype=vel.dtype, device=vel.device)
    sh = _shot(vel, rho, src, rec, wavelet, traces, damp)
    _check(load().ib_forward(table.handle, ctypes.byref(sh), _prec(vel.dtype), float(dt), int(nt),
                             _ptr(ckpt), int(n_ckpt), _stream(stream)))
    return traces


def ib_adjoint(table, vel, wavelet, src, rec, dt, nt, ckpt, n_ckpt, residual, want_wavelet_grad=False,
               damp=None, stream=None):
    """Returns (dJ/dvel [same shape as vel], dJ/dwavelet [nt] or None)."""
    grad = torch.zeros_like(vel)
    gw = torch.zeros(nt, dtype=vel.dtype, device=vel.device) if want_wavelet_grad else None
    sh = _shot(vel, None, src, rec, wavelet, None, damp)
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
        sh[i] = _shot(d["vel"], d.get("rho"), d["src"], d["rec"], d["wavelet"], tr, d.get("damp"))
    _check(load().ib_forward_batch(arr, sh, n, 32, float(dt), int(nt), _stream(stream)))
    return outs


def _batch_shots(tables, shots, nt, need_traces=True):
    n = len(tables)
    arr = (ctypes.c_void_p * n)(*[t.handle.value for t in tables])
    sh = (Shot * n)()
    outs = []
    for i, d in enumerate(shots):
        tr = d.get("traces")
        if tr is None and need_traces:
            tr = torch.zeros((d["rec"].shape[0], nt), dtype=d["vel"].dtype, device=d["vel"].device)
        outs.append(tr)
        sh[i] = _shot(d["vel"], d.get("rho"), d["src"], d["rec"], d["wavelet"], tr, d.get("damp"))
    return n, arr, sh, outs


def _ptrs(tensors):
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def ib_forward_batch_ckpt(tables, shots, dt, nt, ckpts, n_ckpt, stream=None):
    """ib_forward_batch that also fills ckpts[i] (uint8 device tensors of
    ib_checkpoint_bytes(tables[i], 32, nt, n_ckpt) bytes)."""
    n, arr, sh, outs = _batch_shots(tables, shots, nt)
    _check(load().ib_forward_batch_ckpt(arr, sh, n, 32, float(dt), int(nt), _ptrs(ckpts), int(n_ckpt),
                                        _stream(stream)))
    return outs


def ib_adjoint_batch(tables, shots, dt, nt, ckpts, n_ckpt, residuals, stream=None):
    """Velocity gradients of all shots (list of float32 tensors, grid shape)."""
    n, arr, sh, _ = _batch_shots(tables, shots, nt, need_traces=False)
    grads = [torch.empty(t.shape, dtype=torch.float32, device=d["vel"].device) for t, d in zip(tables, shots)]
    res = [r.contiguous() for r in residuals]
    _check(load().ib_adjoint_batch(arr, sh, n, 32, float(dt), int(nt), _ptrs(ckpts), int(n_ckpt), _ptrs(res),
                                   _ptrs(grads), _stream(stream)))
    return grads


def ib_selftest_bounded_wait(stream=None):
    """Status of the bounded-wait self-test (IB_ERR_TIMEOUT when the bound works)."""
    return load().ib_selftest_bounded_wait(_stream(stream))


def ib_stability(table, vel, dt, n_steps, rho=None, seed=1, max_gain=100.0, damp=None, stream=None):
    """(per-step growth estimate, status): power iteration of the time stepping
    with the table's operators; status IB_ERR_UNSTABLE when growth^n_steps > max_gain."""
    g = ctypes.c_double(0.0)
    sh = _shot(vel, rho, None, None, None, None, damp)
    st = load().ib_stability(table.handle, ctypes.byref(sh), _prec(vel.dtype), float(dt), int(n_steps),
                             int(seed), float(max_gain), ctypes.byref(g), _stream(stream))
    _check(st, allow=(IB_ERR_UNSTABLE,))
    return g.value, st


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
