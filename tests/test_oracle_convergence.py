"""Whole-field convergence of the modified Laplacian under grid refinement (no GPU).

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
