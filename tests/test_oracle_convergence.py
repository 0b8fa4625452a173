"""Whole-field convergence of the modified Laplacian under grid refinement (no GPU),
on an off-grid plane and on a circle.

The paper measures the spatial convergence of its boundary treatment on an
exact solution ("Convergence testing"): just short of order 4 for an order-4
discretisation.  Its exact solution is not available, so this pin uses the
spatial part of that experiment with an exact solution of its own: the
Poisson problem L_mod u_h = lap u on the interior nodes, for a field u that
meets every imposed condition on an off-grid flat surface z = z0,

    free   u = sin(k zeta) exp(-zeta^2 / s^2) exp(-(x - xc)^2 / sigma^2)
    rigid  u = cos(k zeta) exp(-zeta^2 / s^2) exp(-(x - xc)^2 / sigma^2),

zeta = z - z0.  u is odd (free) or even (rigid) in zeta, so u, lap u, lap^2 u,
... (free) or every odd normal derivative of lap^k u (rigid) vanish on the
surface, and u is below 1e-27 at the other array edges (zero halo).  The
whole-field error max |u_h - u| over interior nodes then converges at the
order of the extrapolation basis P (local truncation O(h^{P-1}) on a band one
cell thick contributes O(h^P) to the solution).  Refinement is by 3 with the
surface exactly half-way between nodes on every grid (z0 / h = j + 1/2).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import sympy as sy

from oracle import operators, stencils
from paper_2309_03600_gb300 import inputs


def _exact(bc, z0, xc=1.2, sig=0.15, s=0.15, k=2 * np.pi * 1.5):
    x, z = sy.symbols("x z")
    zeta = z - z0
    base = sy.sin(k * zeta) if bc == "free" else sy.cos(k * zeta)
    u = base * sy.exp(-zeta ** 2 / s ** 2) * sy.exp(-(x - xc) ** 2 / sig ** 2)
    f = sy.diff(u, x, 2) + sy.diff(u, z, 2)
    return sy.lambdify((x, z), u, "numpy"), sy.lambdify((x, z), f, "numpy")


def _whole_field_error(M, P, bc, h, z0=0.35, Lx=2.4, Lz=1.55, rank_tol=None):
    nx = int(round(Lx / h)) + 1
    nz = int(round(Lz / h)) + 1
    geom = stencils.Geometry(inputs.flat_surface_sdf((nx, nz), h, z0), h, M)
    L, _ = operators.laplacian_matrix(geom, bc, stencils.Opts(M, ib_order=P, rank_tol=rank_tol))
    uf, ff = _exact(bc, z0)
    X, Z = np.meshgrid(np.arange(nx) * h, np.arange(nz) * h)
    assert np.abs(uf(X, Z)[:, [0, -1]]).max() < 1e-25 and np.abs(uf(X, Z)[-1, :]).max() < 1e-25
    keep = np.flatnonzero(geom.mask.ravel())
    u = uf(X, Z).ravel()[keep]
    f = ff(X, Z).ravel()[keep]
    uh = spla.spsolve(L.tocsr()[keep][:, keep].tocsc(), f)
    return float(np.abs(uh - u).max())


def _orders(M, P, bc, hs, rank_tol=None):
    e = [_whole_field_error(M, P, bc, h, rank_tol=rank_tol) for h in hs]
    return [float(np.log(a / b) / np.log(3.0)) for a, b in zip(e, e[1:])], e


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_whole_field_order4(bc):
    """Order-4 interior and basis: order >= 4 - 0.7 on both refinements
    (measured 4.56 / 4.37 free, 4.13 / 4.16 rigid)."""
    o, e = _orders(4, 4, bc, (1 / 30, 1 / 90, 1 / 270))
    assert all(x >= 4 - 0.7 for x in o), (o, e)


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_whole_field_order8_basis4(bc):
    """Order-8 interior with the order-4 basis (the default at M = 8): the
    basis order bounds the convergence, >= 4 - 0.7 (measured 4.65 free, 3.55 rigid)."""
    o, e = _orders(8, 4, bc, (1 / 30, 1 / 90))
    assert all(x >= 4 - 0.7 for x in o), (o, e)


@pytest.mark.parametrize("bc,bound", [("free", 8 - 0.7), ("rigid", 8 - 1.5)])
def test_whole_field_order8_basis8(bc, bound):
    """Order-8 interior and basis (ib_order = M) at rank tolerance 1e-3:
    free >= 8 - 0.7 (measured 8.39); rigid >= 8 - 1.5 (measured 7.39, then
    6.69 on the next refinement: the rigid hierarchy imposes M/2 conditions
    per boundary point, the free one M/2 + 1).  The rigid default tolerance
    (1e-2, chosen for the stability of the order-4 basis) rejects the order-8
    fits of some rows near this surface and reduces them to order 4: 3.55."""
    o, e = _orders(8, 8, bc, (1 / 30, 1 / 90), rank_tol=1e-3)
    assert all(x >= bound for x in o), (o, e)
    assert e[-1] < 1e-6 * 10, e


# ---------------------------------------------------------------------------
# a curved surface: a circle of radius R (off-grid centre), domain outside it
# ---------------------------------------------------------------------------
XC, ZC, RC = 1.2, 1.2, 0.37      # circle; the array is [0, 2.4]^2
R1, R2 = 0.62, 1.08              # the exact field is windowed to zero between R1 and R2


def _circle_field(bc):
    """u = (r/R - R/r) cos(theta) (free) or (r/R + R/r) cos(theta) (rigid) about
    the circle's centre.  Both are harmonic, so lap u = lap^2 u = ... = 0
    everywhere; the free one vanishes on r = R and the rigid one has zero
    normal derivative there (d/dr (r/R + R/r) = 0 at r = R), so every
    condition of either hierarchy holds on the whole circle."""
    x, z = sy.symbols("x z", real=True)
    r = sy.sqrt((x - XC) ** 2 + (z - ZC) ** 2)
    u = (r / RC + (-1 if bc == "free" else 1) * RC / r) * (x - XC) / r
    return x, z, r, u


def _circle_geometry(M, h):
    n = int(round(2.4 / h)) + 1
    X, Z = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    rr = np.hypot(X - XC, Z - ZC)
    return X, Z, rr, stencils.Geometry(rr - RC, h, M)


def _circle_truncation(M, P, bc, h):
    """max |L_mod u - lap u| over the IB band (lap u = 0)."""
    x, z, r, u = _circle_field(bc)
    uf = sy.lambdify((x, z), u, "numpy")
    X, Z, rr, geom = _circle_geometry(M, h)
    L, _ = operators.laplacian_matrix(geom, bc, stencils.Opts(M, ib_order=P))
    mask = geom.mask.ravel()
    with np.errstate(all="ignore"):
        U = np.where(mask, uf(X, Z).ravel(), 0.0)      # exterior nodes carry no weight
    res = L.tocsr() @ U
    band = mask & (rr.ravel() < RC + (M // 2 + 1) * h)
    return float(np.abs(res[band]).max())


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_ib_rows_truncation_circle(bc):
    """Local truncation of the modified rows on a curved surface: applied to a
    harmonic field that meets every imposed condition on the circle, the rows
    of the IB band return lap u = 0 up to O(h^(P-1)) (an order-P extrapolant
    enters a second difference).  Order 4, h = 1/30 .. 1/240: overall order
    >= P - 1.5 (measured 2.72 free, 2.59 rigid; a wrong sign or dropped BC row
    leaves an O(1) or O(1/h) defect)."""
    hs = (1 / 30, 1 / 60, 1 / 120, 1 / 240)
    e = [_circle_truncation(4, 4, bc, h) for h in hs]
    assert all(a > b for a, b in zip(e, e[1:])), e
    order = float(np.log(e[0] / e[-1]) / np.log(hs[0] / hs[-1]))
    assert order >= 4 - 1.5, (order, e)


def _circle_whole_field_error(M, P, bc, h):
    x, z, r, u = _circle_field(bc)
    t = (r - R1) / (R2 - R1)
    g = lambda s: sy.exp(-1 / s)
    W = g(1 - t) / (g(1 - t) + g(t))            # C-infinity: 1 for r <= R1, 0 for r >= R2
    uf = sy.lambdify((x, z), u, "numpy")
    wf = sy.lambdify((x, z), W, "numpy")
    ff = sy.lambdify((x, z), sy.diff(u * W, x, 2) + sy.diff(u * W, z, 2), "numpy")
    X, Z, rr, geom = _circle_geometry(M, h)
    L, _ = operators.laplacian_matrix(geom, bc, stencils.Opts(M, ib_order=P))
    inner, outer = rr <= R1, rr >= R2
    band = ~inner & ~outer
    with np.errstate(all="ignore"):
        Wv = np.where(inner, 1.0, np.where(outer, 0.0, wf(X, Z)))
        U = np.where(rr > RC / 2, uf(X, Z), 0.0) * Wv
        F = np.where(band, ff(X, Z), 0.0)         # lap(u W) = 0 where W is constant
    keep = np.flatnonzero(geom.mask.ravel())
    uh = spla.spsolve(L.tocsr()[keep][:, keep].tocsc(), F.ravel()[keep])
    return float(np.abs(uh - U.ravel()[keep]).max())


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_whole_field_circle_order4(bc):
    """Whole-field convergence on a curved surface: the Poisson problem with the
    harmonic field above, windowed to zero (C-infinity) well inside the array,
    outside a circle of radius 0.37 at (1.2, 1.2); order 4, refinement by 2.
    Order >= 4 - 0.7 on each refinement (measured 5.17, 3.81 free; 5.16, 3.84
    rigid; 3.91 / 3.93 on the next one)."""
    hs = (1 / 30, 1 / 60, 1 / 120)
    e = [_circle_whole_field_error(4, 4, bc, h) for h in hs]
    o = [float(np.log(a / b) / np.log(2.0)) for a, b in zip(e, e[1:])]
    assert all(v >= 4 - 0.7 for v in o), (o, e)


def _sphere_truncation(M, P, bc, h, c=0.6, R=0.37):
    """max |L_mod u - lap u| over the IB band of a sphere of radius R at (c, c, c)
    in [0, 1.2]^3 (domain outside it), for the harmonic field
    u = (r/R - (R/r)^2) cos(theta) (free: zero on r = R) or
    u = (r/R + (R/r)^2 / 2) cos(theta) (rigid: zero normal derivative on r = R),
    theta measured from the z axis; lap^k u = 0, so every condition holds."""
    n = int(round(1.2 / h)) + 1
    Z, Y, X = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")
    rr = np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2)
    geom = stencils.Geometry(rr - R, h, M)
    L, _ = operators.laplacian_matrix(geom, bc, stencils.Opts(M, ib_order=P))
    mask = geom.mask.ravel()
    with np.errstate(all="ignore"):
        ct = (Z - c) / rr
        u = (rr / R - (R / rr) ** 2) * ct if bc == "free" else (rr / R + 0.5 * (R / rr) ** 2) * ct
        U = np.where(mask, u.ravel(), 0.0)
    res = L.tocsr() @ U
    band = mask & (rr.ravel() < R + (M // 2 + 1) * h)
    return float(np.abs(res[band]).max())


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_ib_rows_truncation_sphere(bc):
    """The 3D rows on a curved surface: the truncation of the IB band on a
    sphere (5.5 and 11 cells in radius at h = 1/15, 1/30, order 4) falls by
    more than 2^2 (measured 28.7 -> 1.40 free, 36.7 -> 0.45 rigid: orders 4.4
    and 6.4 on these coarse grids, ahead of the asymptotic P - 1)."""
    e = [_sphere_truncation(4, 4, bc, h) for h in (1 / 15, 1 / 30)]
    assert e[1] < e[0] / 4.0, e


def _circle_harmonic(X, Z, sign):
    """f = (r/R + sign R/r) cos(theta) about the circle's centre and its x and z
    derivatives (sign -1: zero on the circle; +1: zero normal derivative)."""
    dx, dz = X - XC, Z - ZC
    r2 = dx * dx + dz * dz
    f = dx / RC + sign * RC * dx / r2
    fx = 1.0 / RC + sign * RC * (r2 - 2 * dx * dx) / (r2 * r2)
    fz = -2.0 * sign * RC * dx * dz / (r2 * r2)
    return f, fx, fz


def _circle_staggered_truncation(M, P, bc, h):
    """Truncation of the modified staggered operators near the circle:
    G_a p - d_a p at the v_a nodes (j + e_a/2) for p = f(-1) (free) or f(+1)
    (rigid), and D v - div v (= 0) at the p nodes for v = grad f(+1), which has
    zero divergence and curl and zero normal component on the circle, so it
    meets every velocity condition of both hierarchies."""
    n = int(round(2.4 / h)) + 1
    X, Z = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    rr = np.hypot(X - XC, Z - ZC)
    geom = stencils.Geometry(rr - RC, h, M)
    G, D, _, _ = operators.staggered_matrices(geom, bc, stencils.Opts(M, ib_order=P))
    near = rr.ravel() < RC + (M // 2 + 2) * h
    sg = -1.0 if bc == "free" else 1.0
    shift = ((0.5 * h, 0.0), (0.0, 0.5 * h))
    out = []
    with np.errstate(all="ignore"):
        p = np.where(geom.mask, _circle_harmonic(X, Z, sg)[0], 0.0).ravel()
        vs = []
        for a, (sx, sz) in enumerate(shift):
            _, fx, fz = _circle_harmonic(X + sx, Z + sz, sg)
            vm = geom.vmask(a).ravel()
            out.append(float(np.abs((G[a] @ p - (fx if a == 0 else fz).ravel())[vm & near]).max()))
            _, gx, gz = _circle_harmonic(X + sx, Z + sz, 1.0)
            vs.append(np.where(vm, (gx if a == 0 else gz).ravel(), 0.0))
        out.append(float(np.abs((D @ np.concatenate(vs))[geom.mask.ravel() & near]).max()))
    return out


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_staggered_rows_truncation_circle(bc):
    """The first-order form's modified gradient and divergence rows on a curved
    surface, order 4: from h = 1/30 to 1/240 each truncation converges at
    order >= P - 1 (measured G_x, G_z, D: 3.70, 3.80, 3.35 free; 4.03, 3.59,
    3.55 rigid; a first derivative of an order-P extrapolant is O(h^P))."""
    hs = (1 / 30, 1 / 60, 1 / 120, 1 / 240)
    e = np.array([_circle_staggered_truncation(4, 4, bc, h) for h in hs])
    orders = np.log(e[0] / e[-1]) / np.log(hs[0] / hs[-1])
    assert np.all(orders >= 4 - 1.0), (orders, e)


def test_nd_rows_beat_1d_on_a_circle():
    """The paper's comparison of the N-D extrapolation with the per-axis 1D one
    ("Reduction to 1D"), on a curved free surface: the 1D rows impose p'' = 0
    along each grid line, which the harmonic field does not satisfy across a
    curved surface, so their truncation in the IB band stays O(1) (measured
    13.1, 10.2, 10.6, 10.6 for h = 1/30 .. 1/240), while the N-D rows converge
    (0.20 .. 6.8e-4)."""
    x, z, r, u = _circle_field("free")
    uf = sy.lambdify((x, z), u, "numpy")
    e = {}
    for ex in ("nd", "1d"):
        e[ex] = []
        for h in (1 / 30, 1 / 120):
            X, Z, rr, geom = _circle_geometry(4, h)
            L, _ = operators.laplacian_matrix(geom, "free", stencils.Opts(4, ib_order=4, extrap=ex))
            mask = geom.mask.ravel()
            with np.errstate(all="ignore"):
                U = np.where(mask, uf(X, Z).ravel(), 0.0)
            band = mask & (rr.ravel() < RC + 3 * h)
            e[ex].append(float(np.abs((L.tocsr() @ U)[band]).max()))
    assert all(a < b for a, b in zip(e["nd"], e["1d"])), e
    assert e["nd"][1] < e["nd"][0] / 16, e
    assert e["1d"][1] > e["1d"][0] / 4, e
