"""Host logic of bench.py's roofline (no GPU): the algorithmic bytes per launch
follow the counting the roofline is defined with -- 16 B per second-order grid
point (read p, p_prev, K; write p_next) plus 6 B per correction entry (FP32
weight + 16-bit footprint code), never the gathered value or unfused re-reads --
and the achieved figure is those bytes over the kernel's average launch time."""
import pytest

import bench


def _w(shape, form="second"):
    return {"shape": shape, "form": form}


def test_kernel_bytes_3d_second_order():
    N = 512 * 512 * 384
    stats = {"nnz": [67381122], "rows": [1048576]}
    kb = bench.kernel_bytes(_w((512, 512, 384)), stats, 4)
    assert kb["leap3d_tma_f32"] == 16 * N
    assert kb["ib_add3_f32"] == 6 * 67381122 + 1048576 * (8 + 8 + 4 + 8)
    assert kb["leap3d_f32"] == 16 * N + 6 * 67381122


def test_kernel_bytes_2d_and_staggered():
    stats = {"nnz": [1000], "rows": [10]}
    kb = bench.kernel_bytes(_w((100, 50)), stats, 4)
    assert kb["leap2d_f32"] == 16 * 5000 + 6 * 1000
    assert kb["leap2d_strip_f32"] == kb["leap2d_f32"]
    kb64 = bench.kernel_bytes(_w((100, 50)), stats, 8)
    assert kb64["leap2d_f64"] == 32 * 5000 + 10 * 1000
    # staggered: 7 fields per point and step (read p, v_x, v_z, rho c^2; write p, v_x, v_z),
    # the time loop as replays of a 50-step graph
    ks = bench.kernel_bytes(_w((100, 50), "staggered"), {"nnz": [600, 400], "rows": [5, 5]}, 4)
    assert ks["stag_graph50_f32"] == 50 * (28 * 5000 + 6 * 1000)


def test_roofline_of_picks_the_dominant_kernel():
    prof = {"a": {"sampled": 4, "sampled_ms": 4.0, "launches": 100},      # 1 ms x 100
            "b": {"sampled": 2, "sampled_ms": 1.0, "launches": 1000},     # 0.5 ms x 1000
            "c": {"sampled": 0, "sampled_ms": 0.0, "launches": 10}}
    kb = {"a": 1e9, "b": 2e9, "c": 5e9}
    r = bench.roofline_of(prof, kb, 5000.0, "measured")
    assert r["kernel"] == "b"
    assert r["avg_launch_us"] == pytest.approx(500.0)
    assert r["achieved"] == pytest.approx(2e9 / 5e-4 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_step_roofline_sums_the_two_kernels():
    prof = {"leap3d_tma_f32": {"sampled": 10, "sampled_ms": 3.25, "launches": 2000},
            "ib_add3_f32": {"sampled": 10, "sampled_ms": 1.41, "launches": 2000}}
    w = _w((512, 512, 384))
    stats = {"nnz": [67381122], "rows": [1048576]}
    r = bench.step_roofline(prof, w, stats, 6788.6, "measured")
    byts = 16.0 * 512 * 512 * 384 + 6 * 67381122
    assert r["algorithmic_bytes_per_step"] == byts
    assert r["avg_step_us"] == pytest.approx(466.0)
    assert r["frac"] == pytest.approx(byts / 466e-6 / 1e9 / 6788.6)


def test_job_value_counts_every_rank():
    assert bench.job_value(4, 1e9, 500.0) == pytest.approx(4 * 1e9 / 0.5)
