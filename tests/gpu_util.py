"""Helpers shared by the GPU parity tests (comparison of library tables and
traces with the oracle)."""
import numpy as np
import torch

from oracle import sim, stencils
from paper_2309_03600_gb300 import inputs


def lin_to_node(lin, shape):
    """Array-order linear index -> logical node (x, [y,] z)."""
    idx = np.unravel_index(int(lin), shape)
    return tuple(int(v) for v in reversed(idx))


def gpu_rows(exp, shape, comp_prefix=None):
    """Table export -> {node: ({offset: w}, info)} with offsets in logical order."""
    ndim = len(shape)
    out = {}
    for r, lin in enumerate(exp["row_node"]):
        node = lin_to_node(lin, shape)
        ent = {}
        for k in range(exp["row_ptr"][r], exp["row_ptr"][r + 1]):
            c = exp["col"][k]
            off = (int(c[0]), int(c[2])) if ndim == 2 else (int(c[0]), int(c[1]), int(c[2]))
            if comp_prefix is not None:
                off = (comp_prefix,) + off
            ent[off] = float(exp["w"][k])
        out[node] = (ent, tuple(int(v) for v in exp["info"][r]))
    return out


def compare_tables(orc, gpu, rtol=1e-8, check_info=True, floor=0.0):
    """Same IB nodes, same support sets, same radius and basis order, weights
    equal to (rtol + 1e-13 cond(A)) * max|w| of the row.  Returns the largest
    relative difference seen."""
    assert set(orc) == set(gpu), (sorted(set(orc) ^ set(gpu))[:10], len(orc), len(gpu))
    worst = 0.0
    for node, (wo, info) in orc.items():
        wg, ginfo = gpu[node]
        assert ginfo[3] == 0, (node, ginfo)
        if check_info:
            assert ginfo[0] == int(round(2 * info["radius"])), (node, ginfo, info["radius"])
            assert ginfo[1] == info["order"], (node, ginfo, info["order"])
        assert set(wo) == set(wg), (node, sorted(set(wo) ^ set(wg)))
        if not wo:
            continue
        # floor: the weight scale below which a row's corrections count as zero
        # (rows whose corrections cancel analytically carry only rounding)
        scale = max(1e-300, floor, max(abs(v) for v in wo.values()))
        d = max(abs(wo[k] - wg[k]) for k in wo) / scale
        worst = max(worst, d)
        # both sides carry rounding error ~ cond(A) * eps: allow 1e-13 * cond on top of rtol
        tol = rtol + 1e-13 * info.get("cond", 1.0)
        assert d <= tol, (node, d, info.get("cond"))
    return worst


def split_div(orc_div, comp):
    """Oracle divergence rows -> rows of one velocity component."""
    out = {}
    for node, (w, info) in orc_div.items():
        out[node] = ({k: v for k, v in w.items() if k[0] == comp}, info)
    return out


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def record(name, **vals):
    """Report a measured parity figure: printed, and appended to the file named by
    the environment variable IB_PARITY_LOG when it is set."""
    import os
    line = "PARITY %s %s" % (name, " ".join("%s=%.3e" % (k, v) for k, v in vals.items()))
    print(line, flush=True)
    path = os.environ.get("IB_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


def small_hills(nx=40, ny=36, nz=34, h=10.0, seed=13):
    """A small seeded Gaussian-hills surface (3D parity cases)."""
    prm = inputs.hills_params(5, seed, (nx - 1) * h, (ny - 1) * h, hmin=20, hmax=90, smin=60, smax=160)
    parts = inputs.hills_surface(prm, datum=160.0, zmin=30.0)
    sdf, zs = inputs.heightfield_sdf_3d(nx, ny, nz, h, parts)
    return sdf, zs
