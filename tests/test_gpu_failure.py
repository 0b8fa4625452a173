"""Failure detection on the GPU without a fault: a device wait that nothing
completes gives up after its bound, the host reads IB_ERR_TIMEOUT, and the
context keeps working."""
import pytest
import torch

from paper_2309_03600_gb300 import inputs
from gpu_util import cuda, rel_l2

pytestmark = pytest.mark.gpu

ib = pytest.importorskip("paper_2309_03600_gb300.ib")


def _small_forward():
    w = inputs.workload_flat2d(nx=61, nz=51, nt=60, z0_cells=20.3, src_cells=(30.0, 35.0), rec_x_cells=(10, 50),
                               rec_z_cells=25)
    t = ib.ib_build_stencils(cuda(w["sdf"]), w["h"], "free", "second", w["M"])
    tr = ib.ib_forward(t, cuda(w["vel"], torch.float32), cuda(w["wavelet"], torch.float32), cuda(w["src"]),
                       cuda(w["rec"]), w["dt"], w["nt"])
    return tr.double().cpu().numpy()


def test_bounded_wait_reports_timeout_and_context_survives():
    import time
    before = _small_forward()
    t0 = time.perf_counter()
    st = ib.ib_selftest_bounded_wait()
    print("bounded wait gave up after %.3f s" % (time.perf_counter() - t0))
    assert st == ib.IB_ERR_TIMEOUT
    assert "gave up" in ib.ib_last_error()
    assert ib.ib_sync_status() == ib.IB_OK
    after = _small_forward()
    assert rel_l2(after, before) < 1e-6
