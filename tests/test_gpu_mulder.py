"""GPU: the per-axis 1D extrapolation variant ("Reduction to 1D") against the
oracle -- tables in 2D and 3D, and traces."""
import numpy as np
import pytest
import torch

from oracle import sim, stencils
from paper_2309_03600_gb300 import inputs
from gpu_util import compare_tables, cuda, gpu_rows, record, rel_l2, small_hills

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")


def _opts(M):
    o = ib.ib_opts_default(M)
    o.extrapolation = ib.EXTRAP_1D
    return o


def _case(sdf, h, M):
    geom = stencils.Geometry(sdf, h, M)
    orc = stencils.laplacian_rows(geom, "free", stencils.Opts(M, extrap="1d"))
    t = ib.ib_build_stencils(cuda(sdf), h, "free", "second", M, opts=_opts(M))
    return orc, gpu_rows(t.export(0), sdf.shape), t


@pytest.mark.parametrize("M", [4, 8])
def test_table_1d_sinusoid2d(M):
    w = inputs.workload_sinusoid_staggered(nx=161, nz=101, h=5.0, M=M, nt=10)
    orc, gpu, t = _case(w["sdf"], 5.0, M)
    assert len(orc) > 100
    # a few rows cancel to zero (weights ~1e-16 on both sides): compare on the
    # scale of the standard stencil's weights (order one in grid units)
    compare_tables(orc, gpu, rtol=1e-11, floor=1.0)


def test_table_1d_hills3d():
    sdf, _ = small_hills()
    orc, gpu, _ = _case(sdf, 10.0, 8)
    assert len(orc) > 300
    compare_tables(orc, gpu, rtol=1e-11, floor=1.0)


def test_forward_1d_sinusoid2d():
    """FP64 and FP32 traces with the 1D rows against the oracle (order 8)."""
    w = inputs.workload_sinusoid_staggered(nx=161, nz=121, h=5.0, M=8, nt=600)
    w["src"] = np.array([[400.0, 350.0]])
    w["rec"] = w["rec"][:60]
    vel = w["vel"].astype(np.float64)
    ref = sim.Leapfrog(w["sdf"], vel, 5.0, 8, "free", w["dt"], w["src"], w["rec"],
                       opts=stencils.Opts(8, extrap="1d")).forward(w["wavelet"], w["nt"])
    t = ib.ib_build_stencils(cuda(w["sdf"]), 5.0, "free", "second", 8, opts=_opts(8))
    out = {}
    for dt_ in (torch.float64, torch.float32):
        out[dt_] = ib.ib_forward(t, cuda(vel, dt_), cuda(w["wavelet"], dt_), cuda(w["src"]), cuda(w["rec"]),
                                 w["dt"], w["nt"]).double().cpu().numpy()
    ib.ib_sync_status()
    e64, e32 = rel_l2(out[torch.float64], ref), rel_l2(out[torch.float32], ref)
    record("forward_1d_sinusoid2d", e64=e64, e32=e32)
    assert e64 < 1e-12, e64
    assert e32 < 1e-5, e32


def test_1d_rejects_rigid_and_staggered():
    sdf = cuda(inputs.flat_surface_sdf((40, 30), 1.0, 9.3))
    for bc, form in (("rigid", "second"), ("free", "staggered")):
        with pytest.raises(ib.IbError) as e:
            ib.ib_build_stencils(sdf, 1.0, bc, form, 4, opts=_opts(4))
        assert e.value.status == ib.IB_ERR_ARG
