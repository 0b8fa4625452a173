"""ib_forward_noalloc: the forward for callers that cannot allocate device memory.

Some callers own every device allocation (a host framework with its own memory
manager or a fixed memory budget, a serving loop that must not allocate once
running).  ib_forward_noalloc keeps its scratch in the library's static device
array; its traces must equal those of ib_forward, call after call.  This file
is collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest
import torch

from paper_2309_03600_gb300 import inputs

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")

TOL32 = 1e-5   # the FP32 tolerance of the other parity tests


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["flat_order4", "sinusoid_order8"])
def test_noalloc_matches_forward_twice(case):
    if case == "flat_order4":
        w = inputs.workload_flat2d(nt=400)
    else:
        w = inputs.workload_sinusoid_staggered(nx=241, nz=161, h=5.0, M=8, nt=500)
        w["src"] = np.array([[600.0, 450.0]])
        w["rec"] = w["rec"][:80]
    t = ib.ib_build_stencils(_cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    vel = _cuda(w["vel"], torch.float32)
    wav = _cuda(w["wavelet"], torch.float32)
    src, rec = _cuda(w["src"]), _cuda(w["rec"])
    ref = ib.ib_forward(t, vel, wav, src, rec, w["dt"], w["nt"])
    for _ in range(2):                     # two calls in a row share the static scratch
        tr = torch.full((rec.shape[0], w["nt"]), float("nan"), dtype=torch.float32, device="cuda")
        ib.ib_forward_noalloc(t, vel, wav, src, rec, w["dt"], w["nt"], tr)
        ib.ib_sync_status()
        assert torch.isfinite(tr).all()
        assert _rel(tr, ref) < TOL32


def test_noalloc_rejects_oversize_grid():
    sdf = inputs.flat_surface_sdf((3000, 2000), 10.0, 100.3)
    t = ib.ib_build_stencils(_cuda(sdf), 10.0, "free", "second", 4)
    vel = torch.full(sdf.shape, 1500.0, dtype=torch.float32, device="cuda")
    wav = torch.zeros(4, dtype=torch.float32, device="cuda")
    src = _cuda(np.array([[1000.0, 1000.0]]))
    rec = _cuda(np.array([[1200.0, 500.0]]))
    tr = torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ib.IbError) as e:
        ib.ib_forward_noalloc(t, vel, wav, src, rec, 1e-3, 4, tr)
    assert e.value.status == ib.IB_ERR_ARG
    assert "static limit" in str(e.value)
