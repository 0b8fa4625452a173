"""Pins of the oracle's geometry, constrained fits and modified stencils (no GPU)."""
from fractions import Fraction
import itertools
import math

import numpy as np
import pytest

from oracle import geometry, operators, stencils, taylor
from paper_2309_03600_gb300 import inputs


def circle_sdf(nx, nz, cx, cz, R, inside=False):
    x = np.arange(nx)[None, :] - cx
    z = np.arange(nz)[:, None] - cz
    r = np.sqrt(x * x + z * z)
    return (R - r) if inside else (r - R)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def test_flat_boundary_points():
    sdf = inputs.flat_surface_sdf((20, 30), 1.0, 10.3)
    bps = geometry.BoundaryPoints(sdf, 1.0, 4)
    assert len(bps.owners) == 20
    for o, xb, n in zip(bps.owners, bps.xb, bps.normal):
        assert o[1] == 10
        np.testing.assert_allclose(xb, [o[0], 10.3], atol=1e-14)
        np.testing.assert_allclose(n, [0.0, 1.0], atol=1e-14)


@pytest.mark.parametrize("M", [4, 8])
def test_circle_boundary_points_on_surface(M):
    R, c = 17.3, (31.2, 29.7)
    sdf = circle_sdf(64, 64, c[0], c[1], R)
    bps = geometry.BoundaryPoints(sdf, 1.0, M)
    assert len(bps.owners) > 80
    for o, xb, n in zip(bps.owners, bps.xb, bps.normal):
        rr = math.hypot(xb[0] - c[0], xb[1] - c[1])
        assert abs(rr - R) < 1e-5
        assert np.max(np.abs(xb - np.array(o))) <= 0.5
        # normal points radially outwards (into the domain r > R)
        radial = (np.array(o) - np.array(c)) / math.hypot(o[0] - c[0], o[1] - c[1])
        assert np.dot(n, radial) > 0.999


def test_eta_exclusion():
    sdf = inputs.flat_surface_sdf((10, 10), 1.0, 4.6)
    bps = geometry.BoundaryPoints(sdf, 1.0, 4)
    # bp at z = 4.6 owned by z = 5 (s = 0.4); node z = 5 is 0.4 away -> excluded at eta 0.5
    assert bps.eta_excluded((3.0, 5.0), 0.5)
    assert not bps.eta_excluded((3.0, 5.0), 0.4)        # strict inequality
    assert not bps.eta_excluded((3.0, 6.0), 0.5)
    assert not bps.eta_excluded((3.0, 5.0), 0.0)


# ---------------------------------------------------------------------------
# fits
# ---------------------------------------------------------------------------
def test_free_space_has_no_ib_rows():
    geom = stencils.Geometry(np.full((30, 30), 1e3), 1.0, 4)
    assert stencils.laplacian_ib_nodes(geom.mask, 4) == []
    L, rows = operators.laplacian_matrix(geom, "free", stencils.Opts(4))
    assert rows == {}
    # interior row = textbook stencil
    i = 15 * 30 + 15
    w = [float(x) for x in taylor.central_second(4)]
    row = L.getrow(i).toarray().ravel()
    assert row[i] == pytest.approx(2 * w[2])
    assert row[i + 1] == pytest.approx(w[3]) and row[i + 30] == pytest.approx(w[3])
    assert row[i - 2] == pytest.approx(w[0]) and row[i - 60] == pytest.approx(w[0])


def _frac_solve(A, b):
    """Exact solution of the square system A x = b (Fractions)."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("z0,M", [(Fraction(9, 4), 2), (Fraction(21, 8), 2), (Fraction(9, 4), 4)])
def test_brute_force_rational_least_squares(bc, z0, M):
    """Flat surface at a rational depth: every entry of A is rational, so the
    minimum-norm solution y = A (A^T A)^{-1} u of A^T y = u (the Moore-Penrose
    form of the correction) is computed exactly and compared."""
    nx, nz = 13, 12
    sdf = inputs.flat_surface_sdf((nx, nz), 1.0, float(z0))
    geom = stencils.Geometry(sdf, 1.0, M)
    opts = stencils.Opts(M, eta_p=0.5)
    rows = stencils.laplacian_rows(geom, bc, opts)
    zi = math.ceil(z0) if math.ceil(z0) != z0 else int(z0) + 1
    node = (6, zi)
    wts, info = rows[node]
    r = info["radius"]
    # independent construction of A and u in exact arithmetic
    idx = taylor.multi_indices(2, M)
    half = Fraction(1, 2)
    eta = half
    bp_z = z0                                    # all boundary points at (i, z0)
    owners_z = [k for k in range(nz) if abs(Fraction(k) - z0) <= half]
    assert len(owners_z) == 1

    def mono(px, pz, k, a=(0, 0)):
        if k[0] < a[0] or k[1] < a[1]:
            return Fraction(0)
        ex, ez = k[0] - a[0], k[1] - a[1]
        return px ** ex / math.factorial(ex) * pz ** ez / math.factorial(ez)

    Arows, pts = [], []
    R = int(math.ceil(r)) + 1
    for dz in range(-R, R + 1):
        for dx in range(-R, R + 1):
            x, z = node[0] + dx, node[1] + dz
            if not (0 <= x < nx and 0 <= z < nz):
                continue
            if 4 * (dx * dx + dz * dz) > 4 * r * r:
                continue
            if not Fraction(z) > z0:
                continue
            if abs(Fraction(z) - bp_z) < eta:
                continue
            pts.append((dx, dz))
    pts.sort(key=lambda p: (p[0] ** 2 + p[1] ** 2, p[1], p[0]))
    for dx, dz in pts:
        Arows.append([mono(Fraction(dx), Fraction(dz), k) for k in idx])
    nbp = 0
    for bx in range(nx):
        px, pz = Fraction(bx - node[0]), bp_z - node[1]
        if px * px + pz * pz > Fraction(r) ** 2:
            continue
        nbp += 1
        if bc == "free":
            for k2 in range(0, M // 2 + 1):          # lap^k2 of a term in 2D
                lapk = {}
                for j in range(k2 + 1):
                    lapk[(2 * j, 2 * (k2 - j))] = math.comb(k2, j)
                Arows.append([sum(c * mono(px, pz, k, a) for a, c in lapk.items()) for k in idx])
        else:
            for k2 in range(0, (M - 1) // 2 + 1):    # d/dz lap^k2 (normal = +z)
                lapk = {}
                for j in range(k2 + 1):
                    lapk[(2 * j, 2 * (k2 - j) + 1)] = math.comb(k2, j)
                Arows.append([sum(c * mono(px, pz, k, a) for a, c in lapk.items()) for k in idx])
    assert nbp == info["n_bp"]
    assert len(pts) == info["n_int"]
    w2 = taylor.central_second(M)
    u = [Fraction(0)] * len(idx)
    H = M // 2
    for a in range(2):
        for kk in list(range(-H, 0)) + list(range(1, H + 1)):
            e = [node[0], node[1]]
            e[a] += kk
            if 0 <= e[0] < nx and 0 <= e[1] < nz and not Fraction(e[1]) > z0:
                o = [Fraction(0), Fraction(0)]
                o[a] = Fraction(kk)
                for j, k in enumerate(idx):
                    u[j] += w2[kk + H] * mono(o[0], o[1], k)
    T = len(idx)
    AtA = [[sum(Arows[r_][i] * Arows[r_][j] for r_ in range(len(Arows))) for j in range(T)]
           for i in range(T)]
    z = _frac_solve(AtA, u)
    y = [sum(Arows[i][j] * z[j] for j in range(T)) for i in range(len(pts))]
    got = np.array([wts[p] for p in pts])
    want = np.array([float(v) for v in y])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13 * np.abs(want).max())


def test_square_case_is_inverse():
    """With as many independent rows as columns the pseudoinverse is the inverse
    (the square-system construction the paper attributes to earlier work)."""
    rng = np.random.default_rng(5)
    A = rng.normal(size=(6, 6))
    u = rng.normal(size=6)
    y = np.linalg.pinv(A).T @ u
    np.testing.assert_allclose(y, np.linalg.solve(A.T, u), rtol=1e-10)


def _odd_poly_value(x, z, z0, coeffs):
    """sum a_ij x^i (z - z0)^j over odd j (free) / even j (rigid)."""
    return sum(c * x ** i * (z - z0) ** j for (i, j), c in coeffs.items())


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [4, 8])
def test_flat_polynomial_exactness(bc, M):
    """A polynomial of degree <= a row's basis order that satisfies every
    imposed condition on the plane (odd in z - z0 for the free surface, even
    for the rigid one) is differentiated exactly by the modified operator:
    L_mod q at that IB row equals lap q.  Checked for every basis order the
    rows were fitted at (the full order, or a reduced one)."""
    nx, nz, z0 = 40, 30, 9.37
    sdf = inputs.flat_surface_sdf((nx, nz), 1.0, z0)
    geom = stencils.Geometry(sdf, 1.0, M)
    opts = stencils.Opts(M)
    L, rows = operators.laplacian_matrix(geom, bc, opts)
    X, Z = np.meshgrid(np.arange(nx, dtype=float), np.arange(nz, dtype=float))
    xs, zs = (X - 20.0) / 10.0, Z / 10.0
    ib = np.array([[z, x] for (x, z) in rows])
    order = np.array([info["order"] for (_, info) in rows.values()])
    assert (order == opts.basis(2)).any()
    par = 1 if bc == "free" else 0
    for P in sorted(set(order.tolist())):
        rng = np.random.default_rng(11 + P)
        coeffs = {(i, j): rng.normal() for i in range(P + 1) for j in range(P + 1 - i) if j % 2 == par}
        q = _odd_poly_value(xs, zs, z0 / 10.0, coeffs) * geom.mask
        # exact Laplacian of q in grid units (x, z scaled by 1/10)
        lap = np.zeros_like(q)
        for (i, j), c in coeffs.items():
            if i >= 2:
                lap += c * i * (i - 1) * xs ** (i - 2) * (zs - z0 / 10.0) ** j / 100.0
            if j >= 2:
                lap += c * j * (j - 1) * xs ** i * (zs - z0 / 10.0) ** (j - 2) / 100.0
        Lq = (L @ q.ravel()).reshape(q.shape)
        got = Lq[ib[:, 0], ib[:, 1]]
        want = lap[ib[:, 0], ib[:, 1]]
        # ignore the columns nearest each side wall (truncated by the array edge)
        keep = (ib[:, 1] >= M) & (ib[:, 1] < nx - M) & (order == P)
        scale = np.abs(q).max()
        np.testing.assert_allclose(got[keep], want[keep], atol=1e-9 * scale)


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_curved_exactness_via_null_space(bc):
    """Curved surface: for random delta in the null space of the node's BC rows,
    q = a . delta satisfies every imposed condition at every boundary point;
    the modified row must reproduce the standard stencil applied to q on the
    full lattice: sum_j c_j q(X_j) = sum_e w_e q(x_e)."""
    sdf = circle_sdf(48, 48, 23.4, 24.1, 12.6)
    geom = stencils.Geometry(sdf, 1.0, 8)
    opts = stencils.Opts(8)
    nodes = stencils.laplacian_ib_nodes(geom.mask, 8)[::7]
    rows = stencils.laplacian_rows(geom, bc, opts, nodes)
    rng = np.random.default_rng(2)
    for node, (wts, info) in rows.items():
        A, u, y = info["A"], info["u"], info["y"]
        n_int = info["n_int"]
        C = A[n_int:]
        _, s, Vt = np.linalg.svd(C) if C.shape[0] else (None, np.zeros(0), np.eye(A.shape[1]))
        rank = int((s > 1e-10 * (s[0] if s.size else 1)).sum())
        N = Vt[rank:].T
        if N.shape[1] == 0:
            continue
        delta = N @ rng.normal(size=N.shape[1])
        qX = A[:n_int] @ delta
        lhs = float(np.dot(y[:n_int], qX))
        rhs = float(np.dot(u, delta))
        assert abs(lhs - rhs) <= 1e-9 * (np.abs(y).sum() * np.abs(qX).max() + abs(rhs))
        # and the exact identity A^T y = u that defines the minimum-norm correction
        np.testing.assert_allclose(A.T @ y, u, atol=1e-9 * np.abs(u).max())


def test_support_grows_when_rank_deficient():
    """A geometry where the initial support cannot constrain the basis: a thin
    wedge of interior points. The radius must grow beyond (M+1)/2 (or the order
    drop) and the final A must have full column rank."""
    ws = inputs.workload_sinusoid_staggered(nx=81, nz=61, h=5.0, M=8, nt=10)
    g2 = stencils.Geometry(ws["sdf"], 5.0, 8)
    rows = stencils.divergence_rows(g2, "free", stencils.Opts(8, ib_order=8),
                                    stencils.divergence_ib_nodes(g2, 8)[:40])
    grown = [info["radius"] > (info["order"] + 1) / 2.0 or info["order"] < 8 for _, info in rows.values()]
    assert any(grown)
    for _, info in rows.values():
        A = info["A"]
        sv = np.linalg.svd(A, compute_uv=False)
        assert A.shape[0] >= A.shape[1] and sv[-1] > 1e-3 * sv[0]


def test_block_structure_coupling():
    """Velocity fit: interior rows touch one component block each; BC rows of
    the free surface span both blocks (multi-field section, appendix)."""
    ws = inputs.workload_sinusoid_staggered(nx=81, nz=61, h=5.0, M=4, nt=10)
    g = stencils.Geometry(ws["sdf"], 5.0, 4)
    nodes = stencils.divergence_ib_nodes(g, 4)[:5]
    rows = stencils.divergence_rows(g, "free", stencils.Opts(4), nodes)
    T = taylor.n_terms(2, 4)
    for _, info in rows.values():
        A = info["A"]
        n_int = info["n_int"]
        for r in A[:n_int]:
            assert (np.abs(r[:T]).sum() == 0) != (np.abs(r[T:]).sum() == 0)
        assert all(np.abs(r[:T]).sum() > 0 and np.abs(r[T:]).sum() > 0 for r in A[n_int:])


# ---------------------------------------------------------------------------
# spatial convergence under grid refinement
# ---------------------------------------------------------------------------
def _flat_refinement_errors(M, bc, hs):
    """Max |L_mod f - lap f| at IB rows and at interior rows for a field that
    satisfies every imposed condition on the off-grid plane z = z0:
    free  f = sin(k (z - z0)) cos(m x)  (f, lap f, lap^2 f, ... vanish there),
    rigid f = cos(k (z - z0)) cos(m x)  (every normal derivative of odd order vanishes).
    Rows within M/2 of the other array edges (zero halo) are left out."""
    from oracle import operators
    out = []
    for h in hs:
        n = int(round(1.0 / h)) + 1
        z0 = 0.3037
        geom = stencils.Geometry(inputs.flat_surface_sdf((n, n), h, z0), h, M)
        L, rows = operators.laplacian_matrix(geom, bc, stencils.Opts(M))
        X, Z = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
        k, m = 2 * np.pi * 1.3, 2 * np.pi * 0.9
        f = (np.sin(k * (Z - z0)) if bc == "free" else np.cos(k * (Z - z0))) * np.cos(m * X)
        f = np.where(geom.mask, f, 0.0)
        err = np.abs((L @ f.ravel()).reshape(f.shape) + (k * k + m * m) * f)
        H = M // 2
        inner = geom.mask.copy()
        inner[:, :H] = inner[:, n - H:] = inner[n - H:, :] = False
        ib = np.zeros_like(inner)
        for (i, j) in rows:
            if H <= i < n - H:
                ib[j, i] = True
        inner &= ~ib
        out.append((err[ib].max(), err[inner].max()))
    return out


@pytest.mark.parametrize("bc", ["free", "rigid"])
@pytest.mark.parametrize("M", [4, 8])
def test_spatial_convergence_flat_offgrid(bc, M):
    """Interior rows converge at the stencil order M.  Modified rows converge
    at the order of the extrapolation: a basis of order 4 leaves an O(h^5)
    error in the extrapolated values, O(h^3) after the 1/h^2 of the second
    derivative.  The surface sits at a different fraction of a cell on each
    grid, so the modified rows are checked over two refinements together."""
    e = _flat_refinement_errors(M, bc, (1 / 24, 1 / 48, 1 / 96))
    for a, b in zip(e, e[1:]):
        order = np.log2(a[1] / b[1])
        assert M - 0.5 < order < M + 0.5, order
    assert np.log2(e[0][0] / e[2][0]) / 2 > 2.5, e
