"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import sim, stencils
from paper_2309_03600_gb300 import inputs
from gpu_util import compare_tables, cuda, gpu_rows, record, rel_l2, small_hills

# FP64 traces: the library's weights come from its own FP64 factorisation
# (Cholesky factor of the streamed Gram matrix, seminormal equations + one
# refinement) of the same A that the oracle pseudo-inverts by SVD.  Measured
# FP64 trace differences on the GB300 are 3e-15 .. 1.5e-13 (second-order 2D
# and 3D, staggered, many sources and receivers): the bound is about ten
# times the largest.
TOL64 = 1e-12
# FP64 adjoint: measured 4e-15 (gradient) and 2e-14 (wavelet gradient).
TOL64_ADJ = 2e-13
# FP32 traces: the target relative L2 of the method's FP32 propagation.
TOL32 = 1e-5

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")


def circle_sdf(nx, nz, cx, cz, R, h=1.0):
    x = np.arange(nx)[None, :] - cx
    z = np.arange(nz)[:, None] - cz
    return (np.sqrt(x * x + z * z) - R) * h


# ---------------------------------------------------------------------------
# stencil tables
# ---------------------------------------------------------------------------
def _lap_case(sdf, h, M, bc, **kw):
    geom = stencils.Geometry(sdf, h, M)
    opts = stencils.Opts(M, **kw)
    orc = stencils.laplacian_rows(geom, bc, opts)
    o = ib.ib_opts_default(M)
    if "ib_order" in kw:
        o.basis_order = kw["ib_order"]
    t = ib.ib_build_stencils(cuda(sdf), h, bc, "second", M, opts=o)
    gpu = gpu_rows(t.export(0), sdf.shape)
    return orc, gpu, t


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [2, 4, 8])
def test_table_flat2d(bc, M):
    sdf = inputs.flat_surface_sdf((48, 40), 10.0, 12.3 * 10.0)
    orc, gpu, t = _lap_case(sdf, 10.0, M, bc)
    assert len(orc) > 0
    compare_tables(orc, gpu, rtol=1e-9)
    st = t.stats()
    assert st["n_rank_failures"] == 0
    assert st["n_boundary_points"] == 48


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_table_circle2d(bc):
    sdf = circle_sdf(56, 52, 27.3, 25.6, 13.7, h=5.0)
    orc, gpu, _ = _lap_case(sdf, 5.0, 8, bc)
    compare_tables(orc, gpu, rtol=1e-8)


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_table_sinusoid2d_order8(bc):
    w = inputs.workload_sinusoid_staggered(nx=161, nz=101, h=5.0, M=8, nt=10)
    orc, gpu, _ = _lap_case(w["sdf"], 5.0, 8, bc)
    compare_tables(orc, gpu, rtol=1e-8)


def test_table_sinusoid2d_basis8():
    """Full order-8 basis (45 unknowns) on the GPU constructor."""
    w = inputs.workload_sinusoid_staggered(nx=121, nz=81, h=5.0, M=8, nt=10)
    orc, gpu, _ = _lap_case(w["sdf"], 5.0, 8, "free", ib_order=8)
    compare_tables(orc, gpu, rtol=1e-7)


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [4, 8])
def test_table_hills3d(M, bc):
    sdf, _ = small_hills()
    orc, gpu, _ = _lap_case(sdf, 10.0, M, bc)
    assert len(orc) > 300
    compare_tables(orc, gpu, rtol=1e-8)


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [4, 8])
def test_table_staggered2d(bc, M):
    w = inputs.workload_sinusoid_staggered(nx=121, nz=81, h=5.0, M=M, nt=10)
    geom = stencils.Geometry(w["sdf"], 5.0, M)
    opts = stencils.Opts(M)
    t = ib.ib_build_stencils(cuda(w["sdf"]), 5.0, bc, "staggered", M)
    st = t.stats()
    assert st["n_ops"] == 4
    for a in range(2):
        orc = stencils.gradient_rows(geom, a, bc, opts)
        compare_tables(orc, gpu_rows(t.export(a), w["sdf"].shape), rtol=1e-8)
    orc_div = stencils.divergence_rows(geom, bc, opts)
    merged = {}
    for a in range(2):
        for node, (ent, info) in gpu_rows(t.export(2 + a), w["sdf"].shape, comp_prefix=a).items():
            merged.setdefault(node, ({}, info))[0].update(ent)
    compare_tables(orc_div, merged, rtol=1e-8)


# ---------------------------------------------------------------------------
# propagation
# ---------------------------------------------------------------------------
def _run_leap(w, bc, dtype, nt=None):
    nt = nt or w["nt"]
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], bc, "second", w["M"])
    tr = ib.ib_forward(t, cuda(w["vel"], dtype), cuda(w["wavelet"][:nt], dtype), cuda(w["src"]), cuda(w["rec"]),
                       w["dt"], nt)
    ib.ib_sync_status()
    return tr.double().cpu().numpy()


def _oracle_leap(w, bc, nt=None):
    nt = nt or w["nt"]
    s = sim.Leapfrog(w["sdf"], w["vel"], w["h"], w["M"], bc, w["dt"], w["src"], w["rec"])
    return s.forward(w["wavelet"][:nt], nt)


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_forward_flat2d_201(bc):
    """201 x 201, M = 4, 500 steps, flat surface at z = 40.3 h: FP64 traces to
    1e-10 and FP32 traces to 1e-5 relative L2 against the FP64 oracle."""
    w = inputs.workload_flat2d(bc=bc)
    ref = _oracle_leap(w, bc)
    e64 = rel_l2(_run_leap(w, bc, torch.float64), ref)
    e32 = rel_l2(_run_leap(w, bc, torch.float32), ref)
    record("flat2d_201_" + bc, e64=e64, e32=e32)
    assert e64 < TOL64, e64
    assert e32 < TOL32, e32


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_forward_sinusoid2d_order8(bc):
    w = inputs.workload_sinusoid_staggered(nx=161, nz=121, h=5.0, M=8, nt=800)
    w["src"] = np.array([[400.0, 350.0]])
    w["rec"] = w["rec"][:60]
    w["vel"] = w["vel"].astype(np.float64)
    ref = _oracle_leap(w, bc)
    e64 = rel_l2(_run_leap(w, bc, torch.float64), ref)
    e32 = rel_l2(_run_leap(w, bc, torch.float32), ref)
    record("sinusoid2d_order8_" + bc, e64=e64, e32=e32)
    assert e64 < TOL64, e64
    assert e32 < TOL32, e32


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [4, 8])
def test_forward_hills3d(M, bc):
    sdf, zs = small_hills()
    h = 10.0
    nx, ny, nz = 40, 36, 34
    vel = np.full(sdf.shape, 1800.0)
    dt = 0.4 * h / 1800.0
    nt = 160
    src = np.array([[20 * h, 17 * h, 26 * h]])
    rec = np.array([[x * h, y * h, zs[y, x] + 2 * h] for x in range(4, 36, 5) for y in range(4, 32, 5)])
    w = dict(sdf=sdf, vel=vel, h=h, M=M, dt=dt, nt=nt, src=src, rec=rec, wavelet=inputs.ricker(25.0, dt, nt))
    ref = _oracle_leap(w, bc)
    e32 = rel_l2(_run_leap(w, bc, torch.float32), ref)
    e64 = rel_l2(_run_leap(w, bc, torch.float64), ref)
    record("hills3d_M%d_%s" % (M, bc), e64=e64, e32=e32)
    assert e64 < TOL64, e64
    assert e32 < TOL32, e32


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [4, 8])
def test_forward_staggered2d(bc, M):
    w = inputs.workload_sinusoid_staggered(nx=161, nz=121, h=5.0, M=M, nt=600)
    w["src"] = np.array([[400.0, 350.0]])
    w["rec"] = w["rec"][:60]
    s = sim.Staggered(w["sdf"], w["vel"], w["rho"], 5.0, M, bc, w["dt"], w["src"], w["rec"])
    ref = s.forward(w["wavelet"], w["nt"])
    t = ib.ib_build_stencils(cuda(w["sdf"]), 5.0, bc, "staggered", M)
    out = {}
    for dt_ in (torch.float64, torch.float32):
        tr = ib.ib_forward(t, cuda(w["vel"], dt_), cuda(w["wavelet"], dt_), cuda(w["src"]), cuda(w["rec"]),
                           w["dt"], w["nt"], rho=cuda(w["rho"], dt_))
        out[dt_] = tr.double().cpu().numpy()
    e64 = rel_l2(out[torch.float64], ref)
    e32 = rel_l2(out[torch.float32], ref)
    record("staggered2d_M%d_%s" % (M, bc), e64=e64, e32=e32)
    assert e64 < TOL64, e64
    assert e32 < TOL32, e32


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
def _tiny(bc):
    h, c, M = 10.0, 1500.0, 4
    nx, nz = 36, 30
    sdf = inputs.flat_surface_sdf((nx, nz), h, 6.35 * h)
    rng = np.random.default_rng(9)
    vel = c + 100.0 * rng.normal(size=(nz, nx))
    dt = 0.35 * h / vel.max()
    src = np.array([[17.3 * h, 20.6 * h]])
    rec = np.array([[x * h, 9.5 * h] for x in range(8, 28, 3)])
    return sdf, vel, h, M, dt, src, rec


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("n_ckpt", [1, 7])
def test_adjoint_vs_oracle(bc, n_ckpt):
    sdf, vel, h, M, dt, src, rec = _tiny(bc)
    nt = 90
    rng = np.random.default_rng(4)
    wv = inputs.ricker(25.0, dt, nt)
    res = rng.normal(size=(rec.shape[0], nt))
    s = sim.Leapfrog(sdf, vel, h, M, bc, dt, src, rec)
    _, hist = s.forward(wv, nt, keep_history=True)
    g_ref, gw_ref = s.adjoint(res, hist)
    t = ib.ib_build_stencils(cuda(sdf), h, bc, "second", M)
    v = cuda(vel)
    nb = ib.ib_checkpoint_bytes(t, 64, nt, n_ckpt)
    ck = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    ib.ib_forward(t, v, cuda(wv), cuda(src), cuda(rec), dt, nt, ckpt=ck, n_ckpt=n_ckpt)
    g, gw = ib.ib_adjoint(t, v, cuda(wv), cuda(src), cuda(rec), dt, nt, ck, n_ckpt, cuda(res),
                          want_wavelet_grad=True)
    ib.ib_sync_status()
    eg, ew = rel_l2(g.cpu().numpy().ravel(), g_ref), rel_l2(gw.cpu().numpy(), gw_ref)
    record("adjoint64_%s_ck%d" % (bc, n_ckpt), grad=eg, wavelet=ew)
    assert eg < TOL64_ADJ
    assert ew < TOL64_ADJ


def test_adjoint_dot_product_fp32():
    """<F w, r> = <w, F^T r> through the library in FP32."""
    w = inputs.workload_flat2d(nx=121, nz=101, nt=300, z0_cells=20.3, src_cells=(60.0, 55.0),
                               rec_x_cells=(30, 90), rec_z_cells=24)
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    rng = np.random.default_rng(3)
    nt = w["nt"]
    wv = cuda(rng.normal(size=nt), torch.float32)
    r = cuda(rng.normal(size=(w["rec"].shape[0], nt)), torch.float32)
    v = cuda(w["vel"], torch.float32)
    nb = ib.ib_checkpoint_bytes(t, 32, nt, 10)
    ck = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    tr = ib.ib_forward(t, v, wv, cuda(w["src"]), cuda(w["rec"]), w["dt"], nt, ckpt=ck, n_ckpt=10)
    _, gw = ib.ib_adjoint(t, v, wv, cuda(w["src"]), cuda(w["rec"]), w["dt"], nt, ck, 10, r,
                          want_wavelet_grad=True)
    lhs = float((tr.double() * r.double()).sum())
    rhs = float((wv.double() * gw.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def test_autograd_function():
    sdf, vel, h, M, dt, src, rec = _tiny("free")
    nt = 60
    wv = inputs.ricker(25.0, dt, nt)
    t = ib.ib_build_stencils(cuda(sdf), h, "free", "second", M)
    v = cuda(vel).requires_grad_(True)
    tr = ib.Forward.apply(v, t, cuda(wv), cuda(src), cuda(rec), dt, nt, 5)
    loss = 0.5 * (tr ** 2).sum()
    loss.backward()
    s = sim.Leapfrog(sdf, vel, h, M, "free", dt, src, rec)
    ref_tr, hist = s.forward(wv, nt, keep_history=True)
    g_ref, _ = s.adjoint(ref_tr, hist)
    e = rel_l2(v.grad.detach().cpu().numpy().ravel(), g_ref)
    record("autograd64", grad=e)
    assert e < TOL64_ADJ


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------
def test_argument_errors():
    sdf = cuda(inputs.flat_surface_sdf((20, 20), 1.0, 5.3))
    with pytest.raises(ib.IbError) as e:
        ib.ib_build_stencils(sdf, 1.0, "free", "second", 5)
    assert e.value.status == ib.IB_ERR_ARG
    with pytest.raises(ib.IbError) as e:
        ib.ib_build_stencils(sdf, -1.0, "free", "second", 4)
    assert e.value.status == ib.IB_ERR_ARG
    t = ib.ib_build_stencils(sdf, 1.0, "free", "second", 4)
    v = cuda(np.ones((20, 20)))
    with pytest.raises(ib.IbError):
        ib.ib_forward(t, v, cuda(np.zeros(5)), cuda(np.zeros((1, 2))), cuda(np.zeros((1, 2))), -1.0, 5)


def test_forward_many_sources():
    """32 off-grid sources (the most a shot may have, 256 interpolation corners)
    all enter the FP64 traces as in the oracle; a 33rd is an argument error."""
    w = inputs.workload_flat2d(nx=81, nz=71, nt=150, z0_cells=20.3, src_cells=(40.0, 45.0),
                               rec_x_cells=(10, 70), rec_z_cells=30)
    rng = np.random.default_rng(7)
    src = np.stack([rng.uniform(5.0, 75.0, 32) * w["h"], rng.uniform(28.0, 65.0, 32) * w["h"]], axis=1)
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    tr = ib.ib_forward(t, cuda(w["vel"]), cuda(w["wavelet"]), cuda(src), cuda(w["rec"]), w["dt"], 150)
    ref = sim.Leapfrog(w["sdf"], w["vel"], w["h"], w["M"], "free", w["dt"], src, w["rec"]).forward(w["wavelet"], 150)
    assert np.abs(ref).max() > 0
    e = rel_l2(tr.cpu().numpy(), ref)
    record("many_sources64", e64=e)
    assert e < TOL64
    src33 = np.concatenate([src, src[:1]], axis=0)
    with pytest.raises(ib.IbError) as e:
        ib.ib_forward(t, cuda(w["vel"]), cuda(w["wavelet"]), cuda(src33), cuda(w["rec"]), w["dt"], 150)
    assert e.value.status == ib.IB_ERR_ARG


# ---------------------------------------------------------------------------
# batched shots
# ---------------------------------------------------------------------------
def test_forward_batch_matches_single_shots():
    """Shots of different sizes and surfaces in one batched, graph-captured run
    give the traces of separate ib_forward calls (and of the oracle)."""
    shots, tables = [], []
    for k in range(3):
        w = inputs.workload_shot2d(k, nt=300, side=(140, 220))
        t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
        tables.append(t)
        shots.append(dict(vel=cuda(w["vel"], torch.float32), wavelet=cuda(w["wavelet"], torch.float32),
                          src=cuda(w["src"]), rec=cuda(w["rec"]), w=w))
    dt = shots[0]["w"]["dt"]
    outs = ib.ib_forward_batch(tables, shots, dt, 300)
    ib.ib_sync_status()
    for t, sh, tr in zip(tables, shots, outs):
        single = ib.ib_forward(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, 300)
        e = rel_l2(tr.double().cpu().numpy(), single.double().cpu().numpy())
        assert e < 2e-6, e
    w = shots[0]["w"]
    ref = sim.Leapfrog(w["sdf"], w["vel"], w["h"], w["M"], "free", dt, w["src"], w["rec"]).forward(w["wavelet"], 300)
    assert rel_l2(outs[0].double().cpu().numpy(), ref) < TOL32


@pytest.mark.parametrize("shape", range(10))
def test_forward_batch_every_tile_shape(shape, monkeypatch):
    """Each tile shape the batched launch can pick (plain tiles, z-marched
    strips of 64 x 8 tiles with one column per thread and of 64 x 16 tiles with
    two) gives the traces of separate ib_forward calls, on shots whose sides
    are not multiples of any tile; the second shot has an absorbing layer."""
    monkeypatch.setenv("IB_BATCH_SHAPE", str(shape))
    nt = 120
    shots, tables = [], []
    for k, side in enumerate(((64, 90), (150, 230), (131, 131))):
        w = inputs.workload_shot2d(20 + k, nt=nt, side=side)
        t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
        tables.append(t)
        shots.append(dict(vel=cuda(w["vel"], torch.float32), wavelet=cuda(w["wavelet"], torch.float32),
                          src=cuda(w["src"]), rec=cuda(w["rec"]), w=w, damp=(12, 60.0) if k == 1 else None))
    dt = shots[0]["w"]["dt"]
    outs = ib.ib_forward_batch(tables, shots, dt, nt)
    ib.ib_sync_status()
    for t, sh, tr in zip(tables, shots, outs):
        single = ib.ib_forward(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, damp=sh["damp"])
        ref = single.double().cpu().numpy()
        assert np.abs(ref).max() > 0
        assert rel_l2(tr.double().cpu().numpy(), ref) < 2e-6


def test_forward_2d_strips_match_tiles(monkeypatch):
    """The single-shot FP32 2D step on z-marched strips of 64 x 8 tiles
    (IB_STRIP=1, IB_STRIP4=0) gives the traces of the 64 x 8 tile kernel
    (IB_STRIP=0), on a grid that is not a multiple of the strip size."""
    monkeypatch.setenv("IB_STRIP4", "0")
    w = inputs.workload_shot2d(30, nt=200, side=(150, 260))
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    args = (t, cuda(w["vel"], torch.float32), cuda(w["wavelet"], torch.float32), cuda(w["src"]), cuda(w["rec"]),
            w["dt"], 200)
    monkeypatch.setenv("IB_STRIP", "1")
    a = ib.ib_forward(*args).double().cpu().numpy()
    monkeypatch.setenv("IB_STRIP", "0")
    b = ib.ib_forward(*args).double().cpu().numpy()
    assert np.abs(b).max() > 0
    assert rel_l2(a, b) < 2e-6


@pytest.mark.parametrize("damped", [False, True])
def test_forward_2d_strip4_match_tiles(damped, monkeypatch):
    """The single-shot FP32 2D step on strips of 64 x 16 tiles with two columns
    per thread (IB_STRIP=1; the default strips) gives the traces of the 64 x 8
    tile kernel (IB_STRIP=0), on a grid that is not a multiple of the strip
    size, with and without the absorbing layer."""
    w = inputs.workload_shot2d(30, nt=200, side=(150, 260))
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    damp = (16, 60.0) if damped else None
    args = (t, cuda(w["vel"], torch.float32), cuda(w["wavelet"], torch.float32), cuda(w["src"]), cuda(w["rec"]),
            w["dt"], 200)
    monkeypatch.setenv("IB_STRIP", "1")
    monkeypatch.setenv("IB_STRIP4", "1")
    a = ib.ib_forward(*args, damp=damp).double().cpu().numpy()
    monkeypatch.setenv("IB_STRIP", "0")
    monkeypatch.setenv("IB_STRIP4", "0")
    b = ib.ib_forward(*args, damp=damp).double().cpu().numpy()
    ib.ib_sync_status()
    assert np.abs(b).max() > 0
    assert rel_l2(a, b) < 2e-6


def test_adjoint_batch_matches_single_shots():
    """Shots of different sizes run through ib_forward_batch_ckpt and
    ib_adjoint_batch (one graph for the backward pass) give the traces and the
    velocity gradients of separate ib_forward / ib_adjoint calls; the batched
    checkpoints also serve the single-shot adjoint (same layout)."""
    nt, n_ckpt = 240, 7                   # segments of 35 steps, the last one short
    shots, tables = [], []
    for k in range(3):
        w = inputs.workload_shot2d(10 + k, nt=nt, side=(120, 200))
        t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
        tables.append(t)
        shots.append(dict(vel=cuda(w["vel"], torch.float32), wavelet=cuda(w["wavelet"], torch.float32),
                          src=cuda(w["src"]), rec=cuda(w["rec"]), w=w))
    dt = shots[0]["w"]["dt"]
    ckpts = [torch.empty(ib.ib_checkpoint_bytes(t, 32, nt, n_ckpt), dtype=torch.uint8, device="cuda")
             for t in tables]
    outs = ib.ib_forward_batch_ckpt(tables, shots, dt, nt, ckpts, n_ckpt)
    grads = ib.ib_adjoint_batch(tables, shots, dt, nt, ckpts, n_ckpt, outs)
    ib.ib_sync_status()
    for t, sh, tr, gb, ck in zip(tables, shots, outs, grads, ckpts):
        ck1 = torch.empty_like(ck)
        single = ib.ib_forward(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, ckpt=ck1, n_ckpt=n_ckpt)
        assert rel_l2(tr.double().cpu().numpy(), single.double().cpu().numpy()) < 2e-6
        g1, _ = ib.ib_adjoint(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, ck1, n_ckpt, single)
        gref = g1.double().cpu().numpy()
        assert np.abs(gref).max() > 0
        assert rel_l2(gb.double().cpu().numpy(), gref) < 1e-5
        g2, _ = ib.ib_adjoint(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, ck, n_ckpt, tr)
        assert rel_l2(g2.double().cpu().numpy(), gref) < 1e-5


def test_forward_3d_tma_matches_plain_loads(monkeypatch):
    """FP32 3D runs through the TMA-staged kernel by default; IB_NO_TMA=1 selects
    the kernel with plain loads.  Both must give the same traces (nz = 34 also
    leaves a z chunk shorter than the stencil half-width)."""
    sdf, zs = small_hills()
    h = 10.0
    vel = np.full(sdf.shape, 1800.0)
    dt = 0.4 * h / 1800.0
    nt = 120
    src = np.array([[20 * h, 17 * h, 26 * h]])
    rec = np.array([[x * h, y * h, zs[y, x] + 2 * h] for x in range(4, 36, 5) for y in range(4, 32, 5)])
    w = dict(sdf=sdf, vel=vel, h=h, M=8, dt=dt, nt=nt, src=src, rec=rec, wavelet=inputs.ricker(25.0, dt, nt))
    monkeypatch.delenv("IB_NO_TMA", raising=False)
    ib.ib_profile_enable(1)
    tma = _run_leap(w, "free", torch.float32)
    assert "leap3d_tma_f32" in ib.ib_profile()
    monkeypatch.setenv("IB_NO_TMA", "1")
    ib.ib_profile_enable(1)
    plain = _run_leap(w, "free", torch.float32)
    assert "leap3d_f32" in ib.ib_profile()
    ib.ib_profile_enable(0)
    assert rel_l2(tma, plain) < 1e-6


@pytest.mark.parametrize("damped", [False, True])
def test_forward_3d_pairs_match_single_points(damped, monkeypatch):
    """The default FP32 3D kernel computes two x-adjacent points per thread on
    64 x 8 tiles; IB_TMA3_PAIRS=0 selects the kernel with one point per thread
    on 32 x 8 tiles.  Same traces on a grid of 2 ragged x tiles (nx = 70) with
    the source spread over the corner of four tiles, with and without the
    absorbing layer."""
    sdf, zs = small_hills(nx=70, ny=20, nz=30)
    h = 10.0
    vel = np.full(sdf.shape, 1800.0)
    dt = 0.4 * h / 1800.0
    nt = 100
    src = np.array([[63.6 * h, 7.5 * h, 20.2 * h]])
    rec = np.array([[x * h, y * h, zs[y, x] + 2 * h] for x in range(2, 68, 5) for y in range(2, 18, 5)])
    rec = np.concatenate([src, rec])
    w = dict(sdf=sdf, vel=vel, h=h, M=8, dt=dt, nt=nt, src=src, rec=rec, wavelet=inputs.ricker(25.0, dt, nt))
    damp = (5, 1.5 * 1800.0 / (5 * h) * math.log(1e6)) if damped else None
    t = ib.ib_build_stencils(cuda(sdf), h, "free", "second", 8)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("IB_TMA3_PAIRS", mode)
        tr = ib.ib_forward(t, cuda(vel, torch.float32), cuda(w["wavelet"], torch.float32), cuda(src), cuda(rec),
                           dt, nt, damp=damp)
        ib.ib_sync_status()
        out[mode] = tr.double().cpu().numpy()
    assert np.abs(out["0"]).max() > 0
    assert rel_l2(out["1"], out["0"]) < 1e-6
    if not damped:
        ref = _oracle_leap(w, "free")
        e = rel_l2(out["1"], ref)
        record("pairs3d_70x20x30", e32=e)
        assert e < TOL32, e


def test_forward_3d_correction_pass_rounds(monkeypatch):
    """The 3D correction pass takes each lane's entries 4 at a time by default
    and 8 at a time with IB_ADD3_U=8: the same entries in the same order per
    lane, so the traces are identical bit for bit."""
    sdf, zs = small_hills()
    h = 10.0
    vel = np.full(sdf.shape, 1800.0)
    dt = 0.4 * h / 1800.0
    nt = 60
    src = np.array([[20 * h, 17 * h, 26 * h]])
    rec = np.array([[x * h, y * h, zs[y, x] + 2 * h] for x in range(4, 36, 5) for y in range(4, 32, 5)])
    t = ib.ib_build_stencils(cuda(sdf), h, "free", "second", 8)
    out = {}
    for u in ("8", "4"):
        monkeypatch.setenv("IB_ADD3_U", u)
        tr = ib.ib_forward(t, cuda(vel, torch.float32), cuda(inputs.ricker(25.0, dt, nt), torch.float32), cuda(src),
                           cuda(rec), dt, nt)
        ib.ib_sync_status()
        out[u] = tr.cpu().numpy()
    assert np.abs(out["4"]).max() > 0
    assert np.array_equal(out["8"], out["4"])


# ---------------------------------------------------------------------------
# FP32 adjoint against the oracle, and the gradient against finite differences
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def adjoint_case32():
    """A shot of the batched-shot family (order 8, layered velocity, sinusoid
    plus bump surface) at a size the oracle finishes in about a minute: the
    oracle's FP64 traces, the residual against data from a 2 % faster model,
    and the oracle's velocity gradient of the misfit."""
    nt = 300
    w = inputs.workload_shot2d(40, nt=nt, side=(140, 200))
    vel = w["vel"].astype(np.float64)
    s = sim.Leapfrog(w["sdf"], vel, w["h"], w["M"], "free", w["dt"], w["src"], w["rec"])
    tr, hist = s.forward(w["wavelet"], nt, keep_history=True)
    dobs = s.with_velocity(vel * 1.02).forward(w["wavelet"], nt)
    res = tr - dobs
    g_ref, _ = s.adjoint(res, hist)
    return w, nt, res, g_ref


def test_adjoint_fp32_vs_oracle(adjoint_case32):
    """ib_adjoint in FP32 (the batched workload's precision): the velocity
    gradient of the misfit against the oracle's exact discrete adjoint."""
    w, nt, res, g_ref = adjoint_case32
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    v = cuda(w["vel"], torch.float32)
    wv = cuda(w["wavelet"], torch.float32)
    n_ckpt = 10
    ck = torch.zeros(ib.ib_checkpoint_bytes(t, 32, nt, n_ckpt), dtype=torch.uint8, device="cuda")
    ib.ib_forward(t, v, wv, cuda(w["src"]), cuda(w["rec"]), w["dt"], nt, ckpt=ck, n_ckpt=n_ckpt)
    g, _ = ib.ib_adjoint(t, v, wv, cuda(w["src"]), cuda(w["rec"]), w["dt"], nt, ck, n_ckpt,
                         cuda(res, torch.float32))
    ib.ib_sync_status()
    e = rel_l2(g.double().cpu().numpy().ravel(), g_ref)
    record("adjoint32_single", grad=e)
    assert e < TOL32, e


def test_adjoint_batch_fp32_vs_oracle(adjoint_case32):
    """ib_forward_batch_ckpt + ib_adjoint_batch (one graph for the backward
    pass) with a second shot beside it: shot 0's FP32 gradient against the oracle."""
    w, nt, res, g_ref = adjoint_case32
    w2 = inputs.workload_shot2d(41, nt=nt, side=(120, 180))
    tables, shots = [], []
    for ww in (w, w2):
        tables.append(ib.ib_build_stencils(cuda(ww["sdf"]), ww["h"], "free", "second", ww["M"]))
        shots.append(dict(vel=cuda(ww["vel"], torch.float32), wavelet=cuda(ww["wavelet"], torch.float32),
                          src=cuda(ww["src"]), rec=cuda(ww["rec"])))
    n_ckpt = 10
    ckpts = [torch.empty(ib.ib_checkpoint_bytes(t, 32, nt, n_ckpt), dtype=torch.uint8, device="cuda")
             for t in tables]
    outs = ib.ib_forward_batch_ckpt(tables, shots, w["dt"], nt, ckpts, n_ckpt)
    residuals = [cuda(res, torch.float32), outs[1]]
    grads = ib.ib_adjoint_batch(tables, shots, w["dt"], nt, ckpts, n_ckpt, residuals)
    ib.ib_sync_status()
    e = rel_l2(grads[0].double().cpu().numpy().ravel(), g_ref)
    record("adjoint32_batch", grad=e)
    assert e < TOL32, e


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_gradient_vs_finite_difference_gpu(bc):
    """Central finite difference of J(c) = 1/2 |F(c) - d|^2 along a random
    direction, every J through ib_forward (FP64), against <dJ/dc, dc> from
    ib_adjoint."""
    sdf, vel, h, M, dt, src, rec = _tiny(bc)
    nt = 90
    wv = cuda(inputs.ricker(25.0, dt, nt))
    t = ib.ib_build_stencils(cuda(sdf), h, bc, "second", M)
    S, R = cuda(src), cuda(rec)
    dobs = ib.ib_forward(t, cuda(vel * 1.01), wv, S, R, dt, nt)

    def J(v):
        tr = ib.ib_forward(t, cuda(v), wv, S, R, dt, nt)
        return 0.5 * float(((tr - dobs) ** 2).sum()), tr

    _, tr0 = J(vel)
    ck = torch.zeros(ib.ib_checkpoint_bytes(t, 64, nt, 5), dtype=torch.uint8, device="cuda")
    ib.ib_forward(t, cuda(vel), wv, S, R, dt, nt, ckpt=ck, n_ckpt=5)
    g, _ = ib.ib_adjoint(t, cuda(vel), wv, S, R, dt, nt, ck, 5, tr0 - dobs)
    rng = np.random.default_rng(5)
    dv = rng.normal(size=vel.shape) * (sdf > 0)
    eps = 1e-3
    fd = (J(vel + eps * dv)[0] - J(vel - eps * dv)[0]) / (2 * eps)
    an = float((g.cpu().numpy() * dv).sum())
    ib.ib_sync_status()
    record("gradient_fd_" + bc, rel=abs(fd - an) / abs(fd))
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


# ---------------------------------------------------------------------------
# more receivers than threads in a time-step launch
# ---------------------------------------------------------------------------
def _below_surface_points(rng, n, sdf, h, ndim):
    """n random points (metres) inside the array whose nearest node is interior."""
    shape = sdf.shape
    out = []
    while len(out) < n:
        p = np.array([rng.uniform(0, (shape[ndim - 1 - a] - 1)) for a in range(ndim)])
        node = tuple(int(round(x)) for x in reversed(p))
        if sdf[node] > 0:
            out.append(p * h)
    return np.array(out)


def test_forward_many_receivers_2d_and_3d():
    """6000 (2D, 18 blocks of 256 threads) and 8000 (3D, 20 blocks) receivers:
    every trace is recorded, as in the oracle."""
    rng = np.random.default_rng(12)
    w = inputs.workload_flat2d(nx=81, nz=71, nt=120, z0_cells=20.3, src_cells=(40.0, 45.0),
                               rec_x_cells=(10, 70), rec_z_cells=30)
    rec = _below_surface_points(rng, 6000, w["sdf"], w["h"], 2)
    w["rec"] = rec
    ref = _oracle_leap(w, "free")
    e2 = rel_l2(_run_leap(w, "free", torch.float64), ref)
    sdf, zs = small_hills()
    h = 10.0
    rec3 = _below_surface_points(rng, 8000, sdf, h, 3)
    w3 = dict(sdf=sdf, vel=np.full(sdf.shape, 1800.0), h=h, M=8, dt=0.4 * h / 1800.0, nt=100,
              src=np.array([[20 * h, 17 * h, 26 * h]]), rec=rec3)
    w3["wavelet"] = inputs.ricker(25.0, w3["dt"], 100)
    ref3 = _oracle_leap(w3, "free")
    e3 = rel_l2(_run_leap(w3, "free", torch.float32), ref3)
    record("many_receivers", e2d64=e2, e3d32=e3)
    assert e2 < TOL64, e2
    assert e3 < TOL32, e3


def test_staggered_many_receivers():
    """Staggered step with 4000 receivers on a grid of 10 step tiles."""
    w = inputs.workload_sinusoid_staggered(nx=121, nz=81, h=5.0, M=4, nt=200)
    rng = np.random.default_rng(13)
    w["rec"] = _below_surface_points(rng, 4000, w["sdf"], 5.0, 2)
    w["src"] = np.array([[300.0, 300.0]])
    s = sim.Staggered(w["sdf"], w["vel"], w["rho"], 5.0, 4, "free", w["dt"], w["src"], w["rec"])
    ref = s.forward(w["wavelet"], w["nt"])
    t = ib.ib_build_stencils(cuda(w["sdf"]), 5.0, "free", "staggered", 4)
    tr = ib.ib_forward(t, cuda(w["vel"], torch.float64), cuda(w["wavelet"]), cuda(w["src"]), cuda(w["rec"]),
                       w["dt"], w["nt"], rho=cuda(w["rho"], torch.float64))
    ib.ib_sync_status()
    e = rel_l2(tr.cpu().numpy(), ref)
    record("staggered_many_receivers", e64=e)
    assert e < TOL64, e
