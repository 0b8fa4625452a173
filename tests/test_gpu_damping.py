"""GPU: the absorbing layer (second-order form) against the oracle's damped
propagation and adjoint, and its effect on the growing edge mode."""
import math

import numpy as np
import pytest
import torch

from oracle import sim
from paper_2309_03600_gb300 import inputs
from gpu_util import cuda, record, rel_l2, small_hills

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")

TOL64 = 1e-12
TOL32 = 1e-5


def _eta(c, W, h, R=1e-6):
    return 1.5 * c / (W * h) * math.log(1.0 / R)


@pytest.mark.parametrize("strips", ["0", "1"])
def test_forward_damped_2d(strips, monkeypatch):
    """Sinusoid surface, order 8, a layer of 16 nodes: FP64 (tile kernel) and
    FP32 traces (tile kernel or z-marched strips) against the oracle."""
    monkeypatch.setenv("IB_STRIP", strips)
    w = inputs.workload_shot2d(30, nt=500, side=(150, 260))
    damp = (16, _eta(4000.0, 16, w["h"]))
    vel = w["vel"].astype(np.float64)
    s = sim.Leapfrog(w["sdf"], vel, w["h"], w["M"], "free", w["dt"], w["src"], w["rec"], damp=damp)
    ref = s.forward(w["wavelet"], w["nt"])
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    out = {}
    for dt_ in (torch.float64, torch.float32):
        tr = ib.ib_forward(t, cuda(vel, dt_), cuda(w["wavelet"], dt_), cuda(w["src"]), cuda(w["rec"]), w["dt"],
                           w["nt"], damp=damp)
        out[dt_] = tr.double().cpu().numpy()
    ib.ib_sync_status()
    e64, e32 = rel_l2(out[torch.float64], ref), rel_l2(out[torch.float32], ref)
    record("damped2d_strips" + strips, e64=e64, e32=e32)
    assert e64 < TOL64, e64
    assert e32 < TOL32, e32


def test_forward_damped_3d():
    """Gaussian hills, order 8, a layer of 6 nodes on the four sides and the
    bottom: FP32 (TMA kernel) and FP64 traces against the oracle."""
    sdf, zs = small_hills()
    h = 10.0
    vel = np.full(sdf.shape, 1800.0)
    dt = 0.4 * h / 1800.0
    nt = 200
    src = np.array([[20 * h, 17 * h, 26 * h]])
    rec = np.array([[x * h, y * h, zs[y, x] + 2 * h] for x in range(2, 38, 5) for y in range(2, 34, 5)])
    wv = inputs.ricker(25.0, dt, nt)
    damp = (6, _eta(1800.0, 6, h))
    ref = sim.Leapfrog(sdf, vel, h, 8, "free", dt, src, rec, damp=damp).forward(wv, nt)
    t = ib.ib_build_stencils(cuda(sdf), h, "free", "second", 8)
    out = {}
    for dt_ in (torch.float64, torch.float32):
        tr = ib.ib_forward(t, cuda(vel, dt_), cuda(wv, dt_), cuda(src), cuda(rec), dt, nt, damp=damp)
        out[dt_] = tr.double().cpu().numpy()
    ib.ib_sync_status()
    e64, e32 = rel_l2(out[torch.float64], ref), rel_l2(out[torch.float32], ref)
    record("damped3d", e64=e64, e32=e32)
    assert e64 < TOL64, e64
    assert e32 < TOL32, e32


@pytest.fixture(scope="module")
def damped_adjoint_case():
    nt = 300
    w = inputs.workload_shot2d(41, nt=nt, side=(120, 180))
    vel = w["vel"].astype(np.float64)
    damp = (12, _eta(4000.0, 12, w["h"]))
    s = sim.Leapfrog(w["sdf"], vel, w["h"], w["M"], "free", w["dt"], w["src"], w["rec"], damp=damp)
    tr, hist = s.forward(w["wavelet"], nt, keep_history=True)
    dobs = s.with_velocity(vel * 1.02).forward(w["wavelet"], nt)
    res = tr - dobs
    g_ref, gw_ref = s.adjoint(res, hist)
    return w, nt, damp, res, g_ref, gw_ref


def test_adjoint_damped_vs_oracle(damped_adjoint_case):
    """ib_adjoint of the damped map (FP64 and FP32) against the oracle's."""
    w, nt, damp, res, g_ref, gw_ref = damped_adjoint_case
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    errs = {}
    for dt_, prec in ((torch.float64, 64), (torch.float32, 32)):
        v = cuda(w["vel"], dt_)
        wv = cuda(w["wavelet"], dt_)
        ck = torch.zeros(ib.ib_checkpoint_bytes(t, prec, nt, 7), dtype=torch.uint8, device="cuda")
        ib.ib_forward(t, v, wv, cuda(w["src"]), cuda(w["rec"]), w["dt"], nt, ckpt=ck, n_ckpt=7, damp=damp)
        g, gw = ib.ib_adjoint(t, v, wv, cuda(w["src"]), cuda(w["rec"]), w["dt"], nt, ck, 7, cuda(res, dt_),
                              want_wavelet_grad=True, damp=damp)
        errs[prec] = (rel_l2(g.double().cpu().numpy().ravel(), g_ref), rel_l2(gw.double().cpu().numpy(), gw_ref))
    ib.ib_sync_status()
    record("adjoint_damped", g64=errs[64][0], w64=errs[64][1], g32=errs[32][0], w32=errs[32][1])
    assert errs[64][0] < 1e-12 and errs[64][1] < 1e-12, errs
    assert errs[32][0] < TOL32 and errs[32][1] < TOL32, errs


def test_adjoint_batch_damped_vs_oracle(damped_adjoint_case):
    """The batched forward (with checkpoints) and batched adjoint, damped, next
    to an undamped shot: shot 0's FP32 gradient against the oracle."""
    w, nt, damp, res, g_ref, _ = damped_adjoint_case
    w2 = inputs.workload_shot2d(42, nt=nt, side=(120, 180))
    tables, shots = [], []
    for ww, dd in ((w, damp), (w2, None)):
        tables.append(ib.ib_build_stencils(cuda(ww["sdf"]), ww["h"], "free", "second", ww["M"]))
        shots.append(dict(vel=cuda(ww["vel"], torch.float32), wavelet=cuda(ww["wavelet"], torch.float32),
                          src=cuda(ww["src"]), rec=cuda(ww["rec"]), damp=dd))
    ckpts = [torch.empty(ib.ib_checkpoint_bytes(t, 32, nt, 10), dtype=torch.uint8, device="cuda") for t in tables]
    outs = ib.ib_forward_batch_ckpt(tables, shots, w["dt"], nt, ckpts, 10)
    grads = ib.ib_adjoint_batch(tables, shots, w["dt"], nt, ckpts, 10, [cuda(res, torch.float32), outs[1]])
    ib.ib_sync_status()
    e = rel_l2(grads[0].double().cpu().numpy().ravel(), g_ref)
    single = ib.ib_forward(tables[0], shots[0]["vel"], shots[0]["wavelet"], shots[0]["src"], shots[0]["rec"],
                           w["dt"], nt, damp=damp)
    eb = rel_l2(outs[0].double().cpu().numpy(), single.double().cpu().numpy())
    record("adjoint_batch_damped", grad32=e, batch_vs_single=eb)
    assert e < TOL32, e
    assert eb < 2e-6, eb


def test_layer_removes_edge_growth_gpu():
    """Shot 43 of the batched family grows from the corner where its surface
    meets the array edge (oracle: above 1.05 per step); with a layer of 30
    nodes the library's power iteration decays."""
    w = inputs.workload_shot2d(43, nt=10)
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", 8)
    vel = cuda(w["vel"], torch.float32)
    g0, st0 = ib.ib_stability(t, vel, w["dt"], 1000)
    g1, st1 = ib.ib_stability(t, vel, w["dt"], 1000, damp=(30, _eta(4000.0, 30, w["h"], 1e-8)))
    record("edge_growth_shot43", undamped=g0, damped=g1)
    assert st0 == ib.IB_ERR_UNSTABLE and g0 > 1.05
    assert st1 == ib.IB_OK and g1 < 1.0
