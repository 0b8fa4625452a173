"""GPU: the two-step (temporally blocked) 2D FP32 leapfrog kernel
(IB_TEMPORAL_BLOCK=1) against the FP64 oracle and against the one-step
kernels, with odd and even step counts, sources and receivers near tile
edges, the absorbing layer, more receivers than threads, and the fall-back
to one step per launch when a correction reaches beyond the kernel's margin."""
import numpy as np
import pytest
import torch

from oracle import sim
from paper_2309_03600_gb300 import inputs
from gpu_util import cuda, record, rel_l2

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")

TOL32 = 1e-5


def _run(t, w, nt, monkeypatch, tb, damp=None, rec=None):
    monkeypatch.setenv("IB_TEMPORAL_BLOCK", "1" if tb else "0")
    ib.ib_profile_enable(1)
    tr = ib.ib_forward(t, cuda(w["vel"], torch.float32), cuda(w["wavelet"][:nt], torch.float32), cuda(w["src"]),
                       cuda(w["rec"] if rec is None else rec), w["dt"], nt, damp=damp)
    ib.ib_sync_status()
    prof = ib.ib_profile()
    ib.ib_profile_enable(0)
    return tr.double().cpu().numpy(), prof.get("leap2d_tb2_f32", {}).get("launches", 0)


def _receivers(w, rng, n):
    """The shot's surface receivers plus n random nodes below the surface."""
    sdf, h = w["sdf"], w["h"]
    nz, nx = sdf.shape
    pts = []
    while len(pts) < n:
        x, z = rng.uniform(0, nx - 1), rng.uniform(0, nz - 1)
        if sdf[int(round(z)), int(round(x))] > 0:
            pts.append((x * h, z * h))
    return np.concatenate([w["rec"], np.array(pts)])


@pytest.mark.parametrize("bc,damped", [("free", False), ("free", True), ("rigid", False)])
def test_two_step_vs_oracle(bc, damped, monkeypatch):
    """Sinusoid-and-bump surface, order 8, 156 x 150 nodes (3 x 5 tiles of
    64 x 32, ragged in x and z), 401 steps (the last one by the one-step kernel): FP32
    traces within 1e-5 relative L2 of the oracle's FP64 traces."""
    nt = 401
    w = inputs.workload_shot2d(30, nt=nt, side=(150, 260), bc=bc)
    rec = _receivers(w, np.random.default_rng(5), 40)
    damp = (16, inputs.damping_eta(4000.0, 16, w["h"], 1e-6)) if damped else None
    vel = w["vel"].astype(np.float64)
    ref = sim.Leapfrog(w["sdf"], vel, w["h"], w["M"], bc, w["dt"], w["src"], rec, damp=damp).forward(w["wavelet"], nt)
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], bc, "second", w["M"])
    tr, launches = _run(t, w, nt, monkeypatch, True, damp=damp, rec=rec)
    assert launches == nt // 2
    e = rel_l2(tr, ref)
    record("two_step_%s%s" % (bc, "_damped" if damped else ""), e32=e)
    assert e < TOL32, e


@pytest.mark.parametrize("nt", [2, 3, 4, 57, 200])
def test_two_step_vs_one_step(nt, monkeypatch):
    """Every trace column (the launches record two per call, the last ones are
    recorded after the loop) equals the one-step kernels' to FP32 rounding."""
    w = inputs.workload_shot2d(31, nt=max(nt, 20), side=(130, 200))
    # a source one node from a tile corner: its spread reaches four tiles
    w["src"] = np.array([[64.4 * w["h"], 96.3 * w["h"]]])
    w["wavelet"] = inputs.ricker(40.0, w["dt"], max(nt, 20), t0=0.0)
    rec = np.concatenate([w["src"], _receivers(w, np.random.default_rng(6), 30)])
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    a, la = _run(t, w, nt, monkeypatch, True, rec=rec)
    b, lb = _run(t, w, nt, monkeypatch, False, rec=rec)
    assert la == nt // 2 and lb == 0
    assert np.abs(b).max() > 0
    assert np.abs(b[:, -1]).max() > 0
    assert rel_l2(a, b) < 2e-6, rel_l2(a, b)
    # column by column: no column is missed or shifted
    floor = 1e-7 * np.abs(b).max()
    for c in range(nt):
        assert np.linalg.norm(a[:, c] - b[:, c]) <= 1e-5 * np.linalg.norm(b[:, c]) + floor, c


def test_two_step_many_receivers(monkeypatch):
    """5000 receivers on a grid of 2 x 3 tiles (1536 threads per launch):
    every trace is recorded."""
    w = inputs.workload_flat2d(nx=81, nz=71, nt=60, z0_cells=20.3, src_cells=(40.0, 45.0),
                               rec_x_cells=(10, 70), rec_z_cells=30, M=8)
    rec = _receivers(w, np.random.default_rng(7), 5000)
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", 8)
    a, la = _run(t, w, 60, monkeypatch, True, rec=rec)
    b, _ = _run(t, w, 60, monkeypatch, False, rec=rec)
    assert la == 30
    assert np.all(np.abs(b).max(axis=1) > 0)
    assert rel_l2(a, b) < 2e-6


def test_two_step_falls_back_beyond_margin(monkeypatch):
    """A first support radius of 7.5 puts correction columns 7 nodes from
    their row, beyond the kernel's largest margin (6): the run takes one step
    per launch (whose traces match a second one-step run to rounding: the
    correction sums are shared-memory atomics)."""
    w = inputs.workload_shot2d(32, nt=80, side=(120, 160))
    w["wavelet"] = inputs.ricker(40.0, w["dt"], 80, t0=0.0)
    o = ib.ib_opts_default(w["M"])
    o.radius = 7.5
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"], opts=o)
    exp = ib.ib_table_export(t, 0)
    assert np.abs(np.asarray(exp["col"])).max() >= 7
    rec = np.concatenate([w["src"], _receivers(w, np.random.default_rng(8), 20)])
    a, la = _run(t, w, 80, monkeypatch, True, rec=rec)
    b, _ = _run(t, w, 80, monkeypatch, False, rec=rec)
    assert la == 0
    assert np.abs(b).max() > 1e-8
    assert rel_l2(a, b) < 1e-6
