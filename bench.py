#!/usr/bin/env python
"""Benchmark: grid-point updates/s of the immersed-boundary wave propagator.

One step = one whole shot through the C ABI: ib_build_stencils (boundary
points, IB rows, constrained FP64 fits, packing) + ib_forward over all time
steps (fused stencil + IB gather, source injection, receiver interpolation).
The default workload is the largest single-GPU grid of the method's
configurations: 3D second-order acoustic, 512 x 512 x 384 nodes, h = 10 m,
space order 8, FP32, 2000 time steps at CFL 0.45, a free surface of 12 seeded
Gaussian hills on a 1 km datum, smooth random velocity 1500-4000 m/s, 10 Hz
Ricker source, 256 x 256 receivers 2 h below the surface (synthetic inputs;
the paper's DEM is not available).

The same JSON line carries, under "workloads", the other timed
configurations of the method: the 1001 x 1001 staggered pressure-velocity
shot, 48 batched 2D shots (batched vs one launch per shot), and their
batched forward + adjoint velocity gradient.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on bounded
crops of the same workload instead, on all host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt updates/s vs HBM roofline (plain vs batched/adjoint); IB setup pts/s"
UNIT = "grid-pt updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hills3d",
                    choices=["stag2d", "hills3d", "flat2d", "batch2d", "adjoint2d", "learned3d", "tb2d"])
    ap.add_argument("--train-topos", type=int, default=24, help="learned3d: training topographies")
    ap.add_argument("--epochs", type=int, default=8, help="learned3d: training epochs")
    ap.add_argument("--accept-tol", type=float, default=1e-6, help="learned3d: exactness threshold")
    ap.add_argument("--nshot", type=int, default=48, help="shots of batch2d / adjoint2d")
    ap.add_argument("--bc", default="free", choices=["free", "rigid"])
    ap.add_argument("--nt", type=int, default=0, help="override time steps (testing only)")
    ap.add_argument("--grid", type=int, nargs="*", default=None,
                    help="override the grid of hills3d (nx ny nz) or tb2d (nx nz) (profiling of smaller cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="time the chosen workload only")
    ap.add_argument("--extra-steps", type=int, default=3, help="timed steps of each extra workload")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def make_workload(name, bc, rank=0, nt=0, grid=None):
    from paper_2309_03600_gb300 import inputs
    if name == "stag2d":
        w = inputs.workload_sinusoid_staggered(bc=bc, seed=2 + 1000 * rank)
        w["form"] = "staggered"
        w["desc"] = ("2D first-order staggered p-v, 1001x1001, h=5 m, order 8, FP32, 3000 steps, "
                     "sinusoid %s surface, 4 layers, 12 Hz Ricker, 500 receivers" % bc)
    elif name == "hills3d":
        kw = dict(nx=grid[0], ny=grid[1], nz=grid[2]) if grid else {}
        w = inputs.workload_hills3d(bc=bc, seed=3 + 1000 * rank, device="cuda", **kw)
        w["form"] = "second"
        w["rho"] = None
        w["desc"] = ("3D second-order, 512x512x384, h=10 m, order 8, FP32, 2000 steps at CFL 0.45, "
                     "12 Gaussian hills %s surface, smooth random velocity, 256x256 receivers" % bc)
    else:
        w = inputs.workload_flat2d(bc=bc)
        w["form"] = "second"
        w["rho"] = None
        w["desc"] = "2D second-order, 201x201, h=10 m, order 4, FP64, 500 steps, flat %s surface z=40.3h" % bc
    if nt:
        w["nt"] = nt
        w["wavelet"] = w["wavelet"][:nt]
    w["dtype"] = "f64" if name == "flat2d" else "f32"
    return w


def max_over_ranks(ms, dist, device):
    """Step time of the whole job: the slowest rank's, returned on every rank."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's step time."""
    return world * units_per_rank / (ms * 1e-3)


def grid_points(w):
    n = 1
    for v in w["shape"]:
        n *= v
    return n


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.idx = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


ENTRY_BYTES = {4: 4 + 2, 8: 8 + 2}   # one weight + one 16-bit footprint code per correction entry


def kernel_bytes(w, stats, precision_bytes=4):
    """Algorithmic DRAM bytes of one launch of each time-step kernel, counted
    as the method's roofline counts them: every field the update must read or
    write once per grid point, plus the correction tables at one weight and
    one 16-bit footprint code per entry.  Second order: read p, p_prev, K and
    write p_next (16 B per point in FP32).  Staggered, per step (v and p
    kernels fused): read p, v_x, v_z, rho c^2, write p, v_x, v_z (28 B).
    Values gathered by the corrections and re-reads of unfused kernels are
    not counted."""
    N = grid_points(w)
    e = precision_bytes
    nnz = sum(stats["nnz"])
    tab = ENTRY_BYTES[e] * nnz
    if w["form"] == "staggered":
        step = 7 * e * N + tab
        # the time loop runs as replays of a captured graph of 50 steps (v + p each)
        return {"stag_graph50_" + ("f64" if e == 8 else "f32"): 50 * step}
    name = "leap%dd_%s" % (len(w["shape"]), "f64" if e == 8 else "f32")
    b = 4 * e * N + tab
    out = {name: b}
    if len(w["shape"]) == 3 and e == 4:
        # the TMA-staged 3D step applies the standard stencil (16 B per point); the
        # corrections follow in their own pass over the rows: the table, plus per
        # row its node, entry range and K and the read-modify-write of the output
        out["leap3d_tma_f32"] = 4 * e * N
        out["ib_add3_f32"] = tab + sum(stats["rows"]) * (8 + 8 + 4 + 8)
    if len(w["shape"]) == 2 and e == 4:
        out["leap2d_strip_f32"] = b
    return out


def step_roofline(prof, w, stats, peak, peak_kind):
    """The whole time step of the 3D workload (stencil kernel + correction pass):
    16 B per point + the table at 6 B per entry over the two kernels' summed
    average launch times."""
    a, b = prof.get("leap3d_tma_f32"), prof.get("ib_add3_f32")
    if not (a and a["sampled"] and b and b["sampled"]):
        return None
    t = (a["sampled_ms"] / a["sampled"] + b["sampled_ms"] / b["sampled"]) * 1e-3
    byts = 16.0 * grid_points(w) + ENTRY_BYTES[4] * sum(stats["nnz"])
    ach = byts / t / 1e9
    return {"bound": "hbm", "kernels": ["leap3d_tma_f32", "ib_add3_f32"], "achieved": ach, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_step": byts,
            "avg_step_us": t * 1e6, "frac_of_nominal_8TBs": ach / 8000.0}


def dram_traffic(kernel):
    """Per-launch DRAM bytes from a committed ncu summary, if it is current."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        ent = d.get(kernel)
        if not ent:
            return None
        import hashlib
        h = hashlib.sha256()
        for f in sorted(ent.get("sources", [])):
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != ent.get("sha256"):
            return None
        return float(ent["bytes_per_launch"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# oracle (CPU) sample
# ---------------------------------------------------------------------------
def oracle_full_sizes(workload, w):
    """(grid points, time steps, IB rows) of the full workload, the rows found by
    the oracle's own node detection on the full mask."""
    from oracle import stencils
    M = w["M"]
    if workload == "stag2d":
        g = stencils.Geometry(w["sdf"], w["h"], M)
        rows = (len(stencils.gradient_ib_nodes(g, 0, M)) + len(stencils.gradient_ib_nodes(g, 1, M))
                + len(stencils.divergence_ib_nodes(g, M)))
    else:
        rows = len(stencils.laplacian_ib_nodes(w["sdf"] > 0, M))
    return grid_points(w), w["nt"], rows


def oracle_sample(workload, bc, Nf, ntf, rows_full, seed=0, build_rows=160):
    """Time the FP64 oracle on a bounded sample of the workload and scale it to
    the full workload: the fit of `build_rows` seeded random IB rows of a crop
    (per-row cost x the full workload's IB rows) + time steps on the crop
    (per point-step cost x points x steps).  Touches no GPU.
    Returns (updates/s for the full workload, description)."""
    import numpy as np
    from paper_2309_03600_gb300 import inputs
    from oracle import operators, propagate, stencils
    rng = np.random.default_rng(1000 + seed)
    if workload == "stag2d":
        M, h, nts = 8, 5.0, 200
        w = inputs.workload_sinusoid_staggered(nx=161, nz=161, h=h, M=M, nt=nts, bc=bc)
        geom = stencils.Geometry(w["sdf"], h, M)
        opts = stencils.Opts(M)
        nodes = stencils.divergence_ib_nodes(geom, M)
        pick = [nodes[i] for i in rng.choice(len(nodes), size=min(build_rows, len(nodes)), replace=False)]
        t0 = time.perf_counter()
        div = stencils.divergence_rows(geom, bc, opts, pick)
        t1 = time.perf_counter()
        G, D, _, _ = operators.staggered_matrices(geom, bc, opts, grad_rows=[{}, {}], div_rows=div)
        bv, kp = propagate.staggered_coefficients(geom, w["vel"], w["rho"], w["dt"])
        S = np.zeros(kp.shape[0])
        R = propagate.multilinear_matrix(w["rec"][:50], h, geom.sdf.shape, geom.mask)
        t2 = time.perf_counter()
        propagate.forward_staggered(G, D, bv, kp, S, w["wavelet"], R, nts)
        t3 = time.perf_counter()
        nrow = len(pick)
    else:
        if workload == "hills3d":
            M, h, nts = 8, 10.0, 200
            nx = ny = 48
            nz = 40
            prm = inputs.hills_params(3, 3 + seed, (nx - 1) * h, (ny - 1) * h, hmin=20, hmax=80, smin=80, smax=200)
            sdf, _ = inputs.heightfield_sdf_3d(nx, ny, nz, h, inputs.hills_surface(prm, datum=150.0, zmin=40.0))
            vel = np.full(sdf.shape, 2000.0)
            dt = 0.45 * h / 2000.0
        else:
            w = inputs.workload_flat2d(bc=bc)
            M, h, nts, sdf, vel, dt = w["M"], w["h"], 500, w["sdf"], w["vel"], w["dt"]
        geom = stencils.Geometry(sdf, h, M)
        opts = stencils.Opts(M)
        nodes = stencils.laplacian_ib_nodes(geom.mask, M)
        pick = [nodes[i] for i in rng.choice(len(nodes), size=min(build_rows, len(nodes)), replace=False)]
        t0 = time.perf_counter()
        rows = stencils.laplacian_rows(geom, bc, opts, pick)
        t1 = time.perf_counter()
        L, _ = operators.laplacian_matrix(geom, bc, opts, ib_rows=rows)
        K = propagate.leapfrog_coefficient(vel, dt, geom.mask)
        S = np.zeros(K.shape[0])
        S[K.shape[0] // 2] = 1.0
        R = propagate.multilinear_matrix(np.array([[h * 10.0] * sdf.ndim]), h, sdf.shape, geom.mask)
        t2 = time.perf_counter()
        propagate.forward_leapfrog(L, K, S, inputs.ricker(10.0, dt, nts), R, nts)
        t3 = time.perf_counter()
        nrow = len(pick)
    npts = int(np.prod(geom.sdf.shape))
    t_row = (t1 - t0) / max(nrow, 1)
    t_pt = (t3 - t2) / (npts * nts)
    total = t_row * rows_full + t_pt * Nf * ntf
    desc = ("oracle fit of %d random IB rows (%.2f s) + %d steps (%.2f s) on a %s crop, scaled to %d IB rows and "
            "%d points x %d steps" % (nrow, t1 - t0, nts, t3 - t2, "x".join(map(str, geom.sdf.shape[::-1])),
                                      rows_full, Nf, ntf))
    return Nf * ntf / total, desc


def _oracle_worker(a):
    return oracle_sample(*a)


def cpu_baseline(workload, bc, sizes, cores=None):
    """The oracle as it stands on the host cores: one single-threaded process per
    core, each timing its own seeded sample (spawned, so no GPU state is
    inherited).  Returns the all-core throughput (sum over processes), the
    1-core throughput (the first process alone, before the others start) and
    the core count."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        Nf, ntf, rows = sizes
        with ctx.Pool(1) as pool:
            v1, desc = pool.map(_oracle_worker, [(workload, bc, Nf, ntf, rows, 0)])[0]
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(workload, bc, Nf, ntf, rows, k) for k in range(cores)])
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": sum(v for v, _ in res), "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1core": v1, "sample": "per process: " + desc}


# ---------------------------------------------------------------------------
def roofline_of(prof, kb, peak, peak_kind, prefer=None):
    """Roofline of the dominant sampled kernel (most total time) among those
    whose algorithmic bytes are known."""
    dom, dom_t = None, -1.0
    for name, d in prof.items():
        if d["sampled"] and name in kb and (prefer is None or name in prefer):
            tot = d["sampled_ms"] / d["sampled"] * d["launches"]
            if tot > dom_t:
                dom, dom_t = name, tot
    if dom is None:
        return None
    avg_s = prof[dom]["sampled_ms"] / prof[dom]["sampled"] * 1e-3
    ach = kb[dom] / avg_s / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": ach / peak, "traffic": dram_traffic(dom), "algorithmic_bytes_per_launch": kb[dom],
            "avg_launch_us": avg_s * 1e6, "frac_of_nominal_8TBs": ach / 8000.0}


def kernel_table(prof):
    return {k: {"launches": d["launches"], "avg_us": 1e3 * d["sampled_ms"] / d["sampled"]}
            for k, d in prof.items() if d["sampled"]}


def run_reference(args):
    """The oracle on the host cores: each step is one all-core sample of the
    workload (see cpu_baseline); rank 0 alone runs."""
    wl = args.workload if args.workload in ("hills3d", "stag2d", "flat2d") else "hills3d"
    if wl == "hills3d":
        from paper_2309_03600_gb300 import inputs
        full = inputs.workload_hills3d(bc=args.bc, device="cpu")
        full["form"] = "second"
    else:
        full = make_workload(wl, args.bc)
    sizes = oracle_full_sizes(wl, full)
    vals, base = [], None
    for i in range(args.warmup + args.steps):
        base = cpu_baseline(wl, args.bc, sizes)
        if i >= args.warmup:
            vals.append(base["value"])
    val = sum(vals) / len(vals)
    ms = 1e3 * sizes[0] * sizes[1] / val
    base["value"] = val
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl, "sample": base["sample"]},
        "cpu_baseline": base,
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


def run_single(args, workload, steps, warmup, world, rank, local, dev, dist, with_e2e, with_cpu):
    """One workload of a single shot per rank: timed build + forward, roofline
    of its dominant step kernel, optionally e2e through host buffers and the
    oracle's CPU baseline.  Returns the result dict (rank 0) or None."""
    import torch
    from paper_2309_03600_gb300 import ib

    w = make_workload(workload, args.bc, rank, args.nt, args.grid if workload == "hills3d" else None)
    dtype = torch.float64 if w["dtype"] == "f64" else torch.float32
    eb = 8 if dtype == torch.float64 else 4
    nt = w["nt"]
    sdf_h = torch.as_tensor(w["sdf"], dtype=torch.float64).pin_memory()
    vel_h = torch.as_tensor(w["vel"], dtype=dtype).pin_memory()
    rho_h = torch.as_tensor(w["rho"], dtype=dtype).pin_memory() if w.get("rho") is not None else None
    wav_h = torch.as_tensor(w["wavelet"], dtype=dtype).pin_memory()
    src_h = torch.as_tensor(w["src"], dtype=torch.float64).pin_memory()
    rec_h = torch.as_tensor(w["rec"], dtype=torch.float64).pin_memory()
    sdf, vel, wav, src, rec = (t.to(dev) for t in (sdf_h, vel_h, wav_h, src_h, rec_h))
    rho = rho_h.to(dev) if rho_h is not None else None
    M = w["M"]
    form = w["form"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    traces = torch.zeros((rec.shape[0], nt), dtype=dtype, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        t = ib.ib_build_stencils(sdf, w["h"], w["bc"], form, M)
        ib.ib_forward(t, vel, wav, src, rec, w["dt"], nt, rho=rho, traces=traces)
        return t

    tab = None
    for _ in range(warmup):
        flush.zero_()
        tab = step()
    torch.cuda.synchronize()

    # ---- timed region: device time per step with events, L2 flushed between steps
    clocks = Clocks(local)
    ib.ib_profile_enable(8)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = []
    wall0 = time.perf_counter()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tab = step()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    prof = ib.ib_profile()
    ib.ib_profile_enable(0)
    # the run must have stayed finite (end-of-run NaN/Inf check and the traces)
    ib.ib_sync_status()
    finite = bool(torch.isfinite(traces).all())
    if not finite:
        raise RuntimeError("non-finite traces in the timed run of " + workload)
    stats = tab.stats()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(sum(ms_steps) / len(ms_steps), dist, dev)
    N = grid_points(w)
    upd_per_step = N * nt
    value = job_value(world, upd_per_step, ms)
    launches = sum(d["launches"] for d in prof.values())
    peak, peak_kind = peaks()
    roof = roofline_of(prof, kernel_bytes(w, stats, eb), peak, peak_kind)
    roof_step = step_roofline(prof, w, stats, peak, peak_kind) if len(w["shape"]) == 3 else None
    # ---- end to end through the C ABI with host buffers
    e2e = None
    if with_e2e:
        traces_h = torch.empty((rec.shape[0], nt), dtype=dtype).pin_memory()
        e2e_ms = []
        h2d = sum(t.numel() * t.element_size() for t in (sdf_h, vel_h, wav_h, src_h, rec_h) if t is not None)
        if rho_h is not None:
            h2d += rho_h.numel() * rho_h.element_size()
        for _ in range(max(2, min(steps, 3))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sd, ve, wa, sr, re_ = (t.to(dev, non_blocking=True) for t in (sdf_h, vel_h, wav_h, src_h, rec_h))
            rh = rho_h.to(dev, non_blocking=True) if rho_h is not None else None
            t = ib.ib_build_stencils(sd, w["h"], w["bc"], form, M)
            tr = ib.ib_forward(t, ve, wa, sr, re_, w["dt"], nt, rho=rh)
            traces_h.copy_(tr, non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        em = max_over_ranks(sum(e2e_ms) / len(e2e_ms), dist, dev)
        e2e = {"value": job_value(world, upd_per_step, em), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(traces_h.numel() * traces_h.element_size()), "ms_per_step": em}
    # ---- CPU oracle baseline (rank 0, one GPU)
    cpu = None
    if with_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(workload, args.bc, oracle_full_sizes(workload, w))
    if rank != 0:
        return None
    setup_rows = sum(stats["rows"])
    return {
        "value": value, "ms_per_step": ms, "dtype": w["dtype"],
        "config": {"workload": workload, "desc": w["desc"], "grid": list(w["shape"]), "nt": nt,
                   "space_order": M, "bc": args.bc, "ib_rows": stats["rows"], "ib_nnz": stats["nnz"],
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "setup": {"ib_rows": setup_rows, "seconds": stats["setup_seconds"],
                  "ib_rows_per_s": setup_rows / max(stats["setup_seconds"], 1e-9),
                  "rows_grown": stats["n_grown"], "rows_order_reduced": stats["n_reduced"],
                  "rank_failures": stats["n_rank_failures"], "boundary_points": stats["n_boundary_points"]},
        "roofline": roof, "roofline_step": roof_step, "kernels": kernel_table(prof), "e2e": e2e,
        "cpu_baseline": cpu, "clocks": clk, "gpu_launches": int(launches), "wall_s": wall, "finite": finite,
    }


TB_GRID = (8192, 4096)


def run_temporal(args, steps, warmup, world, rank, local, dev, dist, grid=None, nt=None):
    """2D second-order FP32 shot, 8192 x 4096 nodes (h = 5 m, order 8,
    sinusoid free surface, 4 layers, 400 steps): the forward call with one
    leapfrog step per launch and with two (IB_TEMPORAL_BLOCK=1), table built
    once outside the timed region, L2 flushed between calls.  The two-step
    kernel moves 20 B per point per launch (p^n, p^{n-1}, K read, p^{n+1},
    p^{n+2} written), 10 B per point and step against the 16 B of one step
    per launch; its effective rate (16 B per point and step over its time) can
    exceed the copy bandwidth and is reported beside the DRAM figure."""
    import torch
    from paper_2309_03600_gb300 import ib, inputs
    nx, nz = grid or TB_GRID
    h, M, nt = 5.0, 8, nt or 400
    sdf = torch.as_tensor(inputs.sinusoid_sdf(nx, nz, h, device=dev), dtype=torch.float64, device=dev).contiguous()
    vel = torch.as_tensor(inputs.layered_velocity((nx, nz), h, [800.0, 2000.0, 4000.0],
                                                  [1500.0, 2200.0, 3000.0, 4000.0]), dtype=torch.float32, device=dev)
    dt = inputs.dt_from_courant(0.4, h, 4000.0)
    wav = torch.as_tensor(inputs.ricker(12.0, dt, nt), dtype=torch.float32, device=dev)
    src = torch.tensor([[nx * h / 2, 600.0 + 1000.0 * rank]], dtype=torch.float64, device=dev)
    rx = np.arange(10, nx - 10, 8) * h
    rec = torch.as_tensor(np.stack([rx, np.full_like(rx, 400.0)], 1), device=dev)
    tab = ib.ib_build_stencils(sdf, h, "free", "second", M)
    stats = tab.stats()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    traces = torch.zeros((rec.shape[0], nt), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    N = nx * nz
    peak, peak_kind = peaks()
    out = {}
    old = os.environ.get("IB_TEMPORAL_BLOCK")
    try:
        for mode in ("one_step", "two_step"):
            os.environ["IB_TEMPORAL_BLOCK"] = "1" if mode == "two_step" else "0"
            for _ in range(warmup):
                flush.zero_()
                ib.ib_forward(tab, vel, wav, src, rec, dt, nt, traces=traces)
            torch.cuda.synchronize()
            ib.ib_profile_enable(8)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            ev = []
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ib.ib_forward(tab, vel, wav, src, rec, dt, nt, traces=traces)
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            prof = ib.ib_profile()
            ib.ib_profile_enable(0)
            ib.ib_sync_status()
            if not bool(torch.isfinite(traces).all()):
                raise RuntimeError("non-finite traces in the two-step measurement")
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / len(ev), dist, dev)
            r = {"value": job_value(world, N * nt, ms), "ms_per_call": ms, "kernels": kernel_table(prof),
                 "gpu_launches": int(sum(d["launches"] for d in prof.values()))}
            if mode == "two_step":
                k = prof.get("leap2d_tb2_f32")
                if k and k["sampled"]:
                    t = k["sampled_ms"] / k["sampled"] * 1e-3
                    ach = 20.0 * N / t / 1e9
                    r["roofline"] = {"bound": "hbm", "kernel": "leap2d_tb2_f32", "achieved": ach, "peak": peak,
                                     "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                                     "algorithmic_bytes_per_launch": 20.0 * N, "avg_launch_us": t * 1e6,
                                     "traffic": dram_traffic("leap2d_tb2_f32"),
                                     "effective_GBs_16B_per_point_step": 32.0 * N / t / 1e9,
                                     "effective_frac": 32.0 * N / t / 1e9 / peak}
            else:
                kb = {"leap2d_strip_f32": 16.0 * N + ENTRY_BYTES[4] * sum(stats["nnz"]),
                      "leap2d_f32": 16.0 * N + ENTRY_BYTES[4] * sum(stats["nnz"])}
                r["roofline"] = roofline_of(prof, kb, peak, peak_kind)
            out[mode] = r
    finally:
        if old is None:
            os.environ.pop("IB_TEMPORAL_BLOCK", None)
        else:
            os.environ["IB_TEMPORAL_BLOCK"] = old
    if rank != 0:
        return None
    return {"value": out["two_step"]["value"], "ms_per_step": out["two_step"]["ms_per_call"],
            "config": {"workload": "tb2d", "grid": [nx, nz], "nt": nt, "space_order": M, "bc": "free",
                       "desc": "2D second-order FP32, %dx%d, h=5 m, order 8, %d steps, sinusoid free "
                               "surface, 4 layers; forward call only (table prebuilt)" % (nx, nz, nt),
                       "ib_rows": stats["rows"], "ib_nnz": stats["nnz"], "l2": "flushed between calls"},
            "one_step": out["one_step"], "two_step": out["two_step"],
            "speedup_two_step": out["one_step"]["ms_per_call"] / out["two_step"]["ms_per_call"],
            "gpu_launches": out["one_step"]["gpu_launches"] + out["two_step"]["gpu_launches"]}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args)

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.workload == "learned3d":
        return run_learned(args, world, rank, local, dev, dist)
    if args.workload == "tb2d":   # the one-step / two-step comparison alone
        r = run_temporal(args, args.steps, args.warmup, world, rank, local, dev, dist,
                         tuple(args.grid) if args.grid else None, args.nt or None)
        if rank == 0:
            print(json.dumps(dict(metric=METRIC, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                                  higher_is_better=True, dtype="f32", data="synthetic", **r)))
        if dist:
            dist.destroy_process_group()
        return 0
    if args.workload in ("batch2d", "adjoint2d"):
        res = run_shots(args, args.workload, args.steps, args.warmup, world, rank, local, dev, dist)
    else:
        res = run_single(args, args.workload, args.steps, args.warmup, world, rank, local, dev, dist,
                         not args.no_e2e, not args.no_cpu_baseline)
    extras = {}
    if not args.no_extras and args.workload == "hills3d" and not args.nt and not args.grid:
        ex_steps = max(1, args.extra_steps)
        for name in ("stag2d", "batch2d", "adjoint2d"):
            if name == "stag2d":
                r = run_single(args, name, ex_steps, max(3, args.warmup), world, rank, local, dev, dist, False,
                               False)
            else:
                r = run_shots(args, name, ex_steps, max(3, args.warmup), world, rank, local, dev, dist)
            if r is not None:
                extras[name] = {k: r[k] for k in ("value", "ms_per_step", "config", "setup", "roofline", "kernels",
                                                  "compare", "clocks", "gpu_launches") if k in r}
        r = run_temporal(args, ex_steps, max(3, args.warmup), world, rank, local, dev, dist)
        if r is not None:
            extras["tb2d"] = r
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    out = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": res["dtype"], "data": "synthetic",
    }
    for k in ("config", "setup", "roofline", "roofline_step", "kernels", "compare", "e2e", "cpu_baseline", "clocks",
              "finite"):
        if k in res:
            out[k] = res[k]
    launches = res["gpu_launches"] + sum(e.get("gpu_launches", 0) for e in extras.values())
    out["gpu_launches"] = int(res["gpu_launches"])
    if extras:
        out["workloads"] = extras
        out["gpu_launches_all_workloads"] = int(launches)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def train_network(args, dev, rank):
    """Train the learned-stencil network on rows the plain constructor fits on
    seeded training topographies (untimed; reported)."""
    import torch
    from paper_2309_03600_gb300 import ib, inputs
    net = ib.Mlp(3, 8, n_hidden=256, n_layers=4)
    net.set_params(inputs.mlp_init(net.n_in, 256, 4, net.n_out, seed=17))
    Xs, Ts = [], []
    t0 = time.perf_counter()
    for k in range(args.train_topos):
        sdf = torch.as_tensor(inputs.training_hills_sdf(1000 + k + 100000 * rank, device="cuda"),
                              dtype=torch.float64, device=dev)
        tab = ib.ib_build_stencils(sdf, 10.0, "free", "second", 8)
        nodes, T = ib.ib_mlp_targets(tab, net)
        Xs.append(ib.ib_mlp_features(net, sdf, 10.0, nodes, bc="free"))
        Ts.append(T)
        del tab, sdf
    X, T = torch.cat(Xs), torch.cat(Ts)
    del Xs, Ts
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    g = torch.Generator(device=dev).manual_seed(0)
    B = 4096
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    n_steps = 0
    loss = None
    first = None
    for ep in range(args.epochs):
        perm = torch.randperm(X.shape[0], device=dev, generator=g)
        for b in range(0, X.shape[0] - B + 1, B):
            loss = ib.ib_mlp_train_step(net, X, T, perm[b:b + B], lr=1e-3 if ep < args.epochs - 2 else 3e-4)
            if first is None:
                first = float(loss.item())
            n_steps += 1
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    info = {"rows": int(X.shape[0]), "topographies": args.train_topos, "epochs": args.epochs,
            "batch": B, "steps": n_steps, "data_seconds": t_data, "train_ms": ms,
            "samples_per_s": n_steps * B / (ms * 1e-3), "first_loss": first,
            "final_loss": float(loss.item()) if loss is not None else None}
    del X, T
    return net, info


def run_learned(args, world, rank, local, dev, dist):
    """learned3d: the network proposes each IB row, the exactness test keeps or
    rejects it, rejected rows are fitted; then 1500 FP32 steps.  One step =
    ib_build_stencils_learned + ib_forward on the 768 x 768 x 384 model."""
    import torch
    from paper_2309_03600_gb300 import ib, inputs
    net, train = train_network(args, dev, rank)
    kw = {}
    if args.grid:
        kw = dict(nx=args.grid[0], ny=args.grid[1], nz=args.grid[2])
    w = inputs.workload_learned3d(seed=5 + 1000 * rank, device="cuda", **kw)
    w["form"] = "second"
    nt = args.nt or w["nt"]
    sdf = torch.as_tensor(w["sdf"], dtype=torch.float64, device=dev)
    vel = torch.as_tensor(w["vel"], dtype=torch.float32, device=dev)
    wav = torch.as_tensor(w["wavelet"][:nt], dtype=torch.float32, device=dev)
    src = torch.as_tensor(w["src"], dtype=torch.float64, device=dev)
    rec = torch.as_tensor(w["rec"], dtype=torch.float64, device=dev)
    traces = torch.zeros((rec.shape[0], nt), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    N = grid_points(w)

    def step():
        t = ib.ib_build_stencils_learned(sdf, w["h"], net, space_order=8, accept_tol=args.accept_tol)
        ib.ib_forward(t, vel, wav, src, rec, w["dt"], nt, traces=traces)
        return t

    for _ in range(args.warmup):
        flush.zero_()
        tab = step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ib.ib_profile_enable(8)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tab = step()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    prof = ib.ib_profile()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / len(ev), dist, dev)
    st = tab.stats()
    checked, accepted, res = ib.ib_table_learned(tab)
    fin = res[np.isfinite(res)] if res.size else res
    # the same geometry through the plain constructor, for comparison
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = ib.ib_build_stencils(sdf, w["h"], "free", "second", 8)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    kernels = {k: {"launches": d["launches"], "avg_us": 1e3 * d["sampled_ms"] / d["sampled"]}
               for k, d in prof.items() if d["sampled"]}
    peak, peak_kind = peaks()
    roof = None
    kb = kernel_bytes(w, st, 4)
    for name in ("leap3d_tma_f32", "leap3d_f32"):
        d = prof.get(name)
        if d and d["sampled"]:
            avg_s = d["sampled_ms"] / d["sampled"] * 1e-3
            ach = kb[name] / avg_s / 1e9
            roof = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                    "unit": "GB/s", "frac": ach / peak, "traffic": dram_traffic(name),
                    "algorithmic_bytes_per_launch": kb[name], "avg_launch_us": avg_s * 1e6,
                    "frac_of_nominal_8TBs": ach / 8000.0}
            break
    if rank != 0:
        return 0
    out = {
        "metric": METRIC, "value": job_value(world, N * nt, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "learned3d", "desc": "3D second-order, %dx%dx%d, h=10 m, order 8, FP32, %d steps, "
                   "60 Gaussian hills free surface; rows proposed by the MLP (4x256, bf16) and kept if the "
                   "exactness residual <= %g" % (w["shape"][0], w["shape"][1], w["shape"][2], nt, args.accept_tol),
                   "grid": list(w["shape"]), "nt": nt, "l2": "flushed between steps (256 MB write)"},
        "setup": {"learned_seconds": st["setup_seconds"], "plain_seconds": t_plain,
                  "ib_rows": st["rows"][0], "rows_checked": checked, "rows_accepted": accepted,
                  "residual_median": float(np.median(fin)) if fin.size else None,
                  "residual_p10": float(np.percentile(fin, 10)) if fin.size else None,
                  "rows_below_1e-4": int((fin <= 1e-4).sum()), "rows_below_1e-2": int((fin <= 1e-2).sum()),
                  "ib_rows_per_s_learned": st["rows"][0] / max(st["setup_seconds"], 1e-9),
                  "ib_rows_per_s_plain": st["rows"][0] / max(t_plain, 1e-9)},
        "training": train,
        "roofline": roof, "kernels": kernels, "e2e": None, "cpu_baseline": None, "clocks": clk,
        "gpu_launches": int(sum(d["launches"] for d in prof.values())),
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def run_shots(args, workload, steps, warmup, world, rank, local, dev, dist):
    """batch2d: many 2D second-order shots (sides in [400, 1200], order 8, FP32,
    2000 steps) in one batched, graph-captured launch per step; one step = the
    forward of all shots (tables built once, reported as setup).  The same shots
    one launch per shot and step are timed once for comparison.
    adjoint2d: the same shots, batched forward with 40 checkpoints + batched
    adjoint (velocity gradient of the L2 misfit, the whole backward pass one
    captured graph); one step = all shots.  The same shots one ib_forward +
    ib_adjoint call per shot are timed once for comparison.
    Returns the result dict (rank 0) or None."""
    import torch
    from paper_2309_03600_gb300 import ib, inputs
    nt = args.nt or 2000
    shots, tables = [], []
    t_setup = 0.0
    for k in range(args.nshot):
        w = inputs.workload_shot2d(k + 1000 * rank, nt=nt, device="cuda")
        t0 = time.perf_counter()
        t = ib.ib_build_stencils(torch.as_tensor(w["sdf"], dtype=torch.float64, device=dev), w["h"], "free",
                                 "second", w["M"])
        torch.cuda.synchronize()
        t_setup += time.perf_counter() - t0
        tables.append(t)
        shots.append(dict(vel=torch.as_tensor(w["vel"], dtype=torch.float32, device=dev),
                          wavelet=torch.as_tensor(w["wavelet"], dtype=torch.float32, device=dev),
                          src=torch.as_tensor(w["src"], dtype=torch.float64, device=dev),
                          rec=torch.as_tensor(w["rec"], dtype=torch.float64, device=dev),
                          N=w["shape"][0] * w["shape"][1], dt=w["dt"], damp=w["damp"]))
    dt = shots[0]["dt"]
    N = sum(sh["N"] for sh in shots)
    nnz = sum(sum(t.stats()["nnz"]) for t in tables)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    n_ckpt = 40
    ckpts = []
    if workload == "adjoint2d":
        for t in tables:
            ckpts.append(torch.empty(ib.ib_checkpoint_bytes(t, 32, nt, n_ckpt), dtype=torch.uint8, device=dev))
    last = {}

    def per_shot_adjoint():
        for t, sh, ck in zip(tables, shots, ckpts):
            tr = ib.ib_forward(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, ckpt=ck,
                               n_ckpt=n_ckpt, damp=sh["damp"])
            ib.ib_adjoint(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, ck, n_ckpt, tr,
                          damp=sh["damp"])

    def step():
        if workload == "batch2d":
            last["out"] = ib.ib_forward_batch(tables, shots, dt, nt)
        else:
            # residual = traces (observed data zero): the misfit gradient of all shots
            outs = ib.ib_forward_batch_ckpt(tables, shots, dt, nt, ckpts, n_ckpt)
            last["out"] = ib.ib_adjoint_batch(tables, shots, dt, nt, ckpts, n_ckpt, outs)

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ib.ib_profile_enable(8)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    prof = ib.ib_profile()
    ib.ib_profile_enable(0)
    ib.ib_sync_status()
    finite = all(bool(torch.isfinite(x).all()) for x in last["out"])
    if not finite:
        raise RuntimeError("non-finite output in the timed run of " + workload)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / len(ev), dist, dev)
    value = job_value(world, N * nt, ms)
    peak, peak_kind = peaks()
    roof = None
    compare = None
    eb = ENTRY_BYTES[4]
    if workload == "batch2d":
        g = prof.get("leap2d_batch_graph_f32")
        if g and g["sampled"]:
            per_launch = g["sampled_ms"] / g["sampled"] / nt * 1e-3
            byts = 16.0 * N + eb * nnz
            ach = byts / per_launch / 1e9
            roof = {"bound": "hbm", "kernel": "leap2d_batch_f32", "achieved": ach, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                    "algorithmic_bytes_per_launch": byts, "avg_launch_us": per_launch * 1e6,
                    "frac_of_nominal_8TBs": ach / 8000.0}
        # the same shots, one launch per shot and time step
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t, sh in zip(tables, shots):
            ib.ib_forward(t, sh["vel"], sh["wavelet"], sh["src"], sh["rec"], dt, nt, damp=sh["damp"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        compare = {"one_shot_per_launch_value": N * nt / (ms1 * 1e-3), "one_shot_per_launch_ms": ms1,
                   "batched_speedup": ms1 / ms}
    else:
        a = prof.get("adj2d_batch_graph_f32")
        if a and a["sampled"]:
            avg = a["sampled_ms"] / a["sampled"] * 1e-3
            # one replay = the backward pass of all shots.  Per step and point: the
            # recompute reads p, p_prev, K and stores p (16 B + the forward table);
            # the adjoint step reads mu, mu_prev, K, the stored p^m, p^{m-1},
            # p^{m-2}, the gradient, and writes mu_next and the gradient (36 B +
            # the transposed table); plus the checkpoint restores (4 fields)
            byts = nt * (N * (16 + 36) + 2 * eb * nnz) + n_ckpt * 4 * N * 4
            ach = byts / avg / 1e9
            roof = {"bound": "hbm", "kernel": "adj2d_batch_graph_f32", "achieved": ach, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                    "algorithmic_bytes_per_launch": byts, "avg_launch_us": avg * 1e6,
                    "frac_of_nominal_8TBs": ach / 8000.0}
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        per_shot_adjoint()
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        compare = {"per_shot_calls_value": N * nt / (ms1 * 1e-3), "per_shot_calls_ms": ms1,
                   "batched_speedup": ms1 / ms}
    if rank != 0:
        return None
    return {
        "value": value, "ms_per_step": ms, "dtype": "f32",
        "config": {"workload": workload, "shots": len(shots), "points": N, "nt": nt, "space_order": 8,
                   "edges": "absorbing layer of 20 nodes on the sides and the bottom (nominal reflection 1e-8)",
                   "step": ("batched forward of all shots (tables prebuilt)" if workload == "batch2d"
                            else "batched forward with 40 checkpoints + batched adjoint gradient, all shots"),
                   "l2": "flushed between steps (256 MB write)"},
        "setup": {"seconds": t_setup, "ib_rows": sum(t.stats()["rows"][0] for t in tables), "ib_nnz": nnz},
        "roofline": roof, "kernels": kernel_table(prof), "compare": compare, "e2e": None, "cpu_baseline": None,
        "clocks": clk, "gpu_launches": int(sum(d["launches"] for d in prof.values())), "finite": finite,
    }


if __name__ == "__main__":
    sys.exit(main())
