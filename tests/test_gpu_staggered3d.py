"""GPU: the 3D first-order staggered form (p, v_x, v_y, v_z; the paper's 3D
first-order example) against the oracle: gradient and coupled divergence
tables, and traces in FP64 and FP32."""
import numpy as np
import pytest
import torch

from oracle import sim
from paper_2309_03600_gb300 import inputs
from gpu_util import compare_tables, cuda, gpu_rows, record, rel_l2, small_hills

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")


@pytest.fixture(scope="module", params=["free", "rigid"])
def stag3(request):
    """Small Gaussian-hills model, order 4: the oracle's operators (built once)
    and its FP64 traces."""
    bc = request.param
    h, M = 10.0, 4
    sdf, zs = small_hills(nx=30, ny=28, nz=26)
    vel = np.full(sdf.shape, 1800.0)
    rho = np.full(sdf.shape, 1000.0)
    dt = 0.3 * h / 1800.0
    nt = 140
    src = np.array([[15 * h, 14 * h, 19 * h]])
    rec = np.array([[x * h, y * h, zs[y, x] + 2 * h] for x in range(3, 27, 4) for y in range(3, 25, 4)])
    wv = inputs.ricker(25.0, dt, nt)
    s = sim.Staggered(sdf, vel, rho, h, M, bc, dt, src, rec)
    ref = s.forward(wv, nt)
    return dict(bc=bc, h=h, M=M, sdf=sdf, vel=vel, rho=rho, dt=dt, nt=nt, src=src, rec=rec, wv=wv, s=s, ref=ref)


def test_table_staggered3d(stag3):
    """Gradient rows at v_x, v_y, v_z nodes and the coupled divergence rows at
    p nodes (105 unknowns per fit): same nodes, supports, radii, orders and
    weights as the oracle."""
    c = stag3
    t = ib.ib_build_stencils(cuda(c["sdf"]), c["h"], c["bc"], "staggered", c["M"])
    st = t.stats()
    assert st["n_ops"] == 6
    shape = c["sdf"].shape
    for a in range(3):
        compare_tables(c["s"].grad_rows[a], gpu_rows(t.export(a), shape), rtol=1e-8)
    merged = {}
    for a in range(3):
        for node, (ent, info) in gpu_rows(t.export(3 + a), shape, comp_prefix=a).items():
            merged.setdefault(node, ({}, info))[0].update(ent)
    compare_tables(c["s"].div_rows, merged, rtol=1e-8)


def test_forward_staggered3d(stag3):
    """Traces of the 3D staggered step (FP64 and FP32) against the oracle."""
    c = stag3
    t = ib.ib_build_stencils(cuda(c["sdf"]), c["h"], c["bc"], "staggered", c["M"])
    out = {}
    for dt_ in (torch.float64, torch.float32):
        tr = ib.ib_forward(t, cuda(c["vel"], dt_), cuda(c["wv"], dt_), cuda(c["src"]), cuda(c["rec"]), c["dt"],
                           c["nt"], rho=cuda(c["rho"], dt_))
        out[dt_] = tr.double().cpu().numpy()
    ib.ib_sync_status()
    assert np.abs(c["ref"]).max() > 0
    e64, e32 = rel_l2(out[torch.float64], c["ref"]), rel_l2(out[torch.float32], c["ref"])
    record("staggered3d_" + c["bc"], e64=e64, e32=e32)
    assert e64 < 1e-12, e64
    assert e32 < 1e-5, e32
