"""Pins of the oracle's absorbing layer (no GPU).

The paper's examples use zero Dirichlet edges and note that a damping boundary
of choice combines with the method (Examples section).  The oracle's layer
solves p_tt + eta p_t = c^2 lap p + f near the side edges and the bottom,
centred in time (``oracle.propagate``).  Pinned here: the free decay of the
time derivative against its closed form, the exact adjoint of the damped map,
the absorption of outgoing waves, and the removal of the growing mode that
lives where a surface meets the zero-Dirichlet array edge.
"""
import math

import numpy as np
import pytest

from oracle import propagate, sim, stability, stencils
from paper_2309_03600_gb300 import inputs


def test_profile_shape():
    """a = eta dt / 2 min(1, d^2 / W^2): a_max on the edges and the bottom
    row, zero inside and on the top row away from the sides."""
    nz, nx, W = 30, 40, 5
    a = propagate.damping_coefficient((nz, nx), W, 100.0, 1e-3).reshape(nz, nx)
    amax = 0.5 * 100.0 * 1e-3
    assert a[:, 0].min() == pytest.approx(amax) and a[-1, :].min() == pytest.approx(amax)
    assert a[0, W:nx - W].max() == 0.0 and a[:nz - W, W:nx - W].max() == 0.0
    assert a[10, 2] == pytest.approx(amax * 9 / 25)          # d = 3 from the left edge
    assert a[nz - 4, nx - 4] == pytest.approx(amax * 8 / 25)   # bottom corner: d^2 = 2^2 + 2^2


def test_free_decay_closed_form():
    """With c -> 0 at a layer node the recursion leaves only the damping term:
    the increments d^n = p^n - p^{n-1} shrink by C = (1 - a) / (1 + a) per step,
    so p^n = p^1 (1 - C^n) / (1 - C) exactly, and C is within (eta dt)^3 / 12
    of exp(-eta dt) (the centred difference of p_t + eta p = 0)."""
    nz, nx, h, W, eta = 30, 40, 10.0, 6, 400.0
    sdf = np.full((nz, nx), 1e6)
    vel = np.full((nz, nx), 1e-9)
    dt = 1e-3
    src = np.array([[1.0 * h, 12.0 * h]])          # node (x=1, z=12): d = 5 -> a = a_max 25/36
    s = sim.Leapfrog(sdf, vel, h, 4, "free", dt, src, src, damp=(W, eta))
    nt = 60
    wl = np.zeros(nt)
    wl[0] = 1.0
    tr = s.forward(wl, nt)[0]
    a = 0.5 * eta * dt * 25.0 / 36.0
    C = (1 - a) / (1 + a)
    p1 = dt * dt / h ** 2 / (1 + a)
    n = np.arange(1, nt + 1)
    np.testing.assert_allclose(tr, p1 * (1 - C ** n) / (1 - C), rtol=1e-9)
    assert abs(C - math.exp(-2 * a)) <= (2 * a) ** 3 / 12


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_damped_adjoint_dot_product_and_gradient(bc):
    """The damped map's adjoint: <F w, r> = <w, F^T r> to 1e-12 and the velocity
    gradient against central finite differences of J to 1e-6."""
    h, c, M = 10.0, 1500.0, 4
    nx, nz = 36, 30
    sdf = inputs.flat_surface_sdf((nx, nz), h, 6.35 * h)
    rng = np.random.default_rng(9)
    vel = c + 100.0 * rng.normal(size=(nz, nx))
    dt = 0.35 * h / vel.max()
    src = np.array([[17.3 * h, 20.6 * h]])
    rec = np.array([[x * h, 9.5 * h] for x in range(3, 34, 3)])
    damp = (6, 3.0 * c / (6 * h) * math.log(1e4))
    s = sim.Leapfrog(sdf, vel, h, M, bc, dt, src, rec, damp=damp)
    nt = 90
    wv = rng.normal(size=nt)
    r = rng.normal(size=(rec.shape[0], nt))
    tr, hist = s.forward(wv, nt, keep_history=True)
    _, gw = s.adjoint(r, hist)
    lhs, rhs = float(np.sum(tr * r)), float(np.dot(wv, gw))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
    wv = inputs.ricker(25.0, dt, nt)
    dobs = s.with_velocity(vel * 1.01).forward(wv, nt)
    J = lambda v: 0.5 * float(np.sum((s.with_velocity(v).forward(wv, nt) - dobs) ** 2))
    tr0, hist = s.forward(wv, nt, keep_history=True)
    g, _ = s.adjoint(tr0 - dobs, hist)
    dv = rng.normal(size=vel.shape) * s.geom.mask
    eps = 1e-3
    fd = (J(vel + eps * dv) - J(vel - eps * dv)) / (2 * eps)
    assert abs(fd - float(np.dot(g, dv.ravel()))) <= 1e-6 * abs(fd)


def test_layer_absorbs_edge_reflections():
    """201 x 201, flat free surface: once the direct wave has reached the side
    edges, the late traces near the source carry the edge reflections; a layer
    of 20 nodes cuts them by more than 10x against zero Dirichlet edges."""
    w = inputs.workload_flat2d(nt=1100, rec_x_cells=(90, 110), rec_z_cells=80)
    c, h = w["c"], w["h"]
    out = {}
    for damp in (None, (20, 1.5 * c / (20 * h) * math.log(1e6))):
        s = sim.Leapfrog(w["sdf"], w["vel"], h, w["M"], "free", w["dt"], w["src"], w["rec"], damp=damp)
        out[damp is None] = s.forward(w["wavelet"], w["nt"])
    t = (np.arange(w["nt"]) + 1) * w["dt"]
    late = t > 2 * 95 * h / c + 0.2              # after the first side-edge reflection is back
    und, dmp = np.abs(out[True][:, late]).max(), np.abs(out[False][:, late]).max()
    assert dmp < 0.1 * und, (dmp, und)


def test_layer_removes_edge_growth():
    """The batched-shot family's shot 43: its surface meets the zero-Dirichlet
    array edge, where the modified operator has a growing mode (per step growth
    above 1.05).  With a layer of 30 nodes the power iteration decays."""
    w = inputs.workload_shot2d(43, nt=10)
    geom = stencils.Geometry(w["sdf"], w["h"], 8)
    from oracle import operators
    L, _ = operators.laplacian_matrix(geom, "free", stencils.Opts(8))
    vel = w["vel"].astype(np.float64)
    K = propagate.leapfrog_coefficient(vel, w["dt"], geom.mask)
    r0, _ = stability.leapfrog_growth(L, K, nsteps=600)
    a = propagate.damping_coefficient(geom.sdf.shape, 30, 1.5 * vel.max() / (30 * w["h"]) * math.log(1e8),
                                      w["dt"]) * geom.mask.ravel()
    r1, _ = stability.leapfrog_growth(L, K, nsteps=600, a=a)
    assert r0 > 1.05 and r1 < 1.0, (r0, r1)
