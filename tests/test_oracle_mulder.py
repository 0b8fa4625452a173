"""Pins of the oracle's per-axis 1D extrapolation, the variant the paper derives
as a sub-case of its method ("Reduction to 1D"; free surface), and of the
paper's comparison of the two (N-D error lower at every grid increment).  No GPU."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import sympy as sy

from oracle import images, operators, sim, stencils
from paper_2309_03600_gb300 import inputs


def test_extrapolation_1d_closed_forms():
    """Order 2: the extrapolant is the line through (u_b, 0) and (u_1, f_1)
    (p = p'' = 0 at u_b), so f~(u_e) = f_1 (u_e - u_b) / (u_1 - u_b).  Order 4: an
    odd cubic a z + b z^3 about u_b (z = u - u_b) through the two interior
    points; its weights follow from the 2 x 2 system in (a, b)."""
    u1, ub, ue = -0.0, 0.37, 2.0
    e = stencils.extrapolation_1d([u1], ub, ue, 2, "free")
    assert abs(e[0] - (ue - ub) / (u1 - ub)) < 1e-14
    pts = [0.0, -1.0]
    e = stencils.extrapolation_1d(pts, ub, ue, 4, "free")
    Z = np.array([[z, z ** 3] for z in (pts[0] - ub, pts[1] - ub)])
    ze = ue - ub
    want = np.array([ze, ze ** 3]) @ np.linalg.inv(Z)
    np.testing.assert_allclose(e, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("M", [4, 8])
def test_1d_flat_polynomial_exactness(M):
    """Flat surface z = z0 (only the z stencils are cut): the 1D rows reproduce
    lap q for every polynomial q odd in z - z0 of degree <= M (it meets p = 0,
    p'' = 0, ... on the surface along the z lines)."""
    nx, nz, z0 = 40, 30, 9.37
    sdf = inputs.flat_surface_sdf((nx, nz), 1.0, z0)
    geom = stencils.Geometry(sdf, 1.0, M)
    L, rows = operators.laplacian_matrix(geom, "free", stencils.Opts(M, extrap="1d"))
    assert all(info["order"] == M for (_, info) in rows.values())
    rng = np.random.default_rng(5)
    coeffs = {(i, j): rng.normal() for i in range(M + 1) for j in range(M + 1 - i) if j % 2 == 1}
    X, Z = np.meshgrid(np.arange(nx, dtype=float), np.arange(nz, dtype=float))
    xs, zs = (X - 20.0) / 10.0, (Z - z0) / 10.0
    q = sum(c * xs ** i * zs ** j for (i, j), c in coeffs.items()) * geom.mask
    lap = np.zeros_like(q)
    for (i, j), c in coeffs.items():
        if i >= 2:
            lap += c * i * (i - 1) * xs ** (i - 2) * zs ** j / 100.0
        if j >= 2:
            lap += c * j * (j - 1) * xs ** i * zs ** (j - 2) / 100.0
    Lq = (L @ q.ravel()).reshape(q.shape)
    ib = np.array([[z, x] for (x, z) in rows])
    keep = (ib[:, 1] >= M) & (ib[:, 1] < nx - M)
    np.testing.assert_allclose(Lq[ib[keep, 0], ib[keep, 1]], lap[ib[keep, 0], ib[keep, 1]],
                               atol=1e-9 * np.abs(q).max())


def _tilted_error(M, h, extrap, ang=17.0, k=2 * np.pi * 1.5, s=0.15, sig=0.15):
    """Whole-field error of the Poisson problem L_mod u_h = lap u on a plane
    tilted by `ang` degrees, u odd in the distance to the plane (it meets every
    free-surface condition there), Gaussian-windowed along and across it."""
    a = math.radians(ang)
    nrm = (math.sin(a), math.cos(a))
    pt = (1.2, 0.55)
    x, z = sy.symbols("x z")
    zeta = (x - pt[0]) * nrm[0] + (z - pt[1]) * nrm[1]
    xi = (x - pt[0]) * nrm[1] - (z - pt[1]) * nrm[0]
    u = sy.sin(k * zeta) * sy.exp(-zeta ** 2 / s ** 2) * sy.exp(-xi ** 2 / sig ** 2)
    uf = sy.lambdify((x, z), u, "numpy")
    ff = sy.lambdify((x, z), sy.diff(u, x, 2) + sy.diff(u, z, 2), "numpy")
    nx, nz = int(round(2.4 / h)) + 1, int(round(1.8 / h)) + 1
    geom = stencils.Geometry(inputs.tilted_plane_sdf((nx, nz), h, np.array(pt), ang), h, M)
    L, _ = operators.laplacian_matrix(geom, "free", stencils.Opts(M, extrap=extrap))
    X, Z = np.meshgrid(np.arange(nx) * h, np.arange(nz) * h)
    keep = np.flatnonzero(geom.mask.ravel())
    uh = spla.spsolve(L.tocsr()[keep][:, keep].tocsc(), ff(X, Z).ravel()[keep])
    return float(np.abs(uh - uf(X, Z).ravel()[keep]).max())


@pytest.mark.parametrize("M", [4, 8])
def test_nd_error_below_1d_on_a_tilted_plane(M):
    """The paper's comparison: the N-D extrapolation gives the lower error at
    every grid increment tested (measured at h = 1/40, 1/80: N-D 8.6e-4, 3.3e-5
    against 1D 2.6e-3, 6.6e-4 at M = 4).  The 1D rows impose p'' = 0 along the
    grid line, which a tilted plane does not satisfy (the mixed derivative of an
    odd field survives), so the 1D field converges at order 2 (measured 1.99)."""
    e_nd = [_tilted_error(M, h, "nd") for h in (1 / 40, 1 / 80)]
    e_1d = [_tilted_error(M, h, "1d") for h in (1 / 40, 1 / 80)]
    assert all(a < b for a, b in zip(e_nd, e_1d)), (e_nd, e_1d)
    assert math.log2(e_1d[0] / e_1d[1]) > 1.7, e_1d


def test_1d_flat_surface_images_201():
    """Config-1 geometry (201 x 201, order 4, flat surface at z = 40.3 h): the
    1D rows match direct minus image within twice the free-space scheme error,
    like the N-D rows (a flat surface cut only along z)."""
    w = inputs.workload_flat2d()
    s = sim.Leapfrog(w["sdf"], w["vel"], w["h"], w["M"], "free", w["dt"], w["src"], w["rec"],
                     opts=stencils.Opts(w["M"], extrap="1d"))
    tr = s.forward(w["wavelet"], w["nt"])
    times = (np.arange(w["nt"]) + 1) * w["dt"]
    an = images.flat_surface_traces(images.ricker_fn(w["f0"]), w["src"][0], w["rec"], times, w["c"], w["z0"],
                                    "free", 2)
    win = times < 0.95
    s0 = sim.Leapfrog(np.full_like(w["sdf"], 1e6), w["vel"], w["h"], w["M"], "free", w["dt"], w["src"], w["rec"])
    tr0 = s0.forward(w["wavelet"], w["nt"])
    r = np.linalg.norm(w["rec"] - w["src"][0], axis=1)[:, None]
    an0 = images.free_space_2d(images.ricker_fn(w["f0"]), r, times[None, :], w["c"])
    e = float(np.linalg.norm(tr[:, win] - an[:, win]) / np.linalg.norm(an[:, win]))
    e0 = float(np.linalg.norm(tr0[:, win] - an0[:, win]) / np.linalg.norm(an0[:, win]))
    assert e <= 2.0 * e0, (e, e0)
