"""Support regions, constrained fits and modified stencils (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper sections followed, in the paper's order:
1. Hyperspherical support of radius r around the expansion point, starting at
   r = (M+1)/2 ("Constructing Finite-Difference Approximations", support
   figure paragraph).
2. Interior points in the support, minus those with a boundary point inside
   their 2 eta-sided box; boundary points in the support carry one row per
   boundary condition (Eq. of the BC dot product; general boundary linear
   system).
3. rank(A) must equal the number of basis terms; otherwise enlarge the support,
   and as a last resort lower the basis order (rank paragraph; order-reduction
   paragraph; 3D first-order example).
4. delta = A^+ [f(X); g] with the Moore-Penrose pseudoinverse; exterior values
   f~(X_e) = B A^+ [f(X); g]; with g = 0 the forcing columns drop out
   ("Reconciliation with the Interior Numerical Discretization"; example
   geometry).
5. The interior stencil with exterior values replaced by the extrapolants gives
   the modified operator (modified-stencil equation).  For the Laplacian all
   axes share the expansion point, so the per-axis modified operators are
   summed into one row (the Laplacian is the sum of per-dimension second
   derivative operators, 2nd-order application section).
6. Multiple fields: block rows, coupled by BC rows that span several fields
   (multi-field section; particle-velocity free surface; appendix).

A modified row is returned as the *correction* to the standard stencil:
    L_mod f(x0) = sum_{interior axial} w_k f(x0 + k e_a) + sum_j c_j f(X_j)
with c = ((A^+)^T u)[interior rows], u = sum_e w_e a(x_e - x0).  The first sum
is the standard stencil with exterior values set to zero, which is what the
propagators apply everywhere.

Readings of the paper used here (the paper is silent or ambiguous):
* support membership |x - x0|_2 <= r is decided exactly (positions are
  half-integers in grid units, so 4|x - x0|^2 and 4 r^2 are integers);
* boundary points are in the support if |x_b - x0|^2 <= r^2 + 1e-9;
* r grows by 0.5 up to r0 + 3; then the basis order drops by 2 (down to 2);
* rank test: sigma_min > rank_tol * sigma_max of A (SVD), and A has at least
  as many rows as columns.  The paper asks for rank(A) equal to the number of
  basis terms and gives no tolerance; the default is set per boundary
  condition from the measured growth per step of the schemes
  (``oracle.stability``): 1e-3 for the free surface (order-8 basis on the
  seeded sinusoid: 1.05 at 1e-10, 1.0013 at 1e-3; 512 x 512 x 384 Gaussian
  hills: 1.0002 at 1e-3, 1.041 at 1e-2) and 1e-2 for the rigid surface
  (hills: 1.076 at 1e-3, 1.00002 at 1e-2; sinusoid with eta 0.25: 1.00064 at
  1e-3, 1.00011 at 1e-2);
* expansion point: the stencil centre (2nd-order form); the node receiving the
  derivative (staggered form);
* eta of the pressure fits: 0.5 for the free surface, as the paper sets it
  (2D example-geometry paragraph), and 0.25 for the rigid surface, for which
  the paper gives no value (rigid, rank tolerance 1e-2, seeded sinusoid:
  growth per step 1.0026 at eta 0.5, 1.00011 at 0.25; at rank tolerance 1e-3
  on a 34 x 34 x 30 hills crop: 1.10 at 0.5, 1.0004 at 0.25, 1.17 at 0.75);
* basis order of the extrapolants (``Opts.basis``): min(M, 4) by default.
  The paper asks for a basis of the interior order for consistent error (3D
  expansion paragraph of "Constructing Finite-Difference Approximations") and
  allows a reduced basis order where footprints would grow too large
  (order-reduction paragraph).  This reading takes the reduction at M > 4:
  the whole-field error then converges at order 4 (the paper's own examples
  are order 4 throughout), the 3D order-8 footprint stays at 81 points
  instead of ~380 (165 unknowns), and the measured growth per step of the
  order-8 schemes is no better with the full basis on the method's
  workloads (batched 2D shots: 1.083 with either basis, the surface meeting
  the zero-Dirichlet array edge; staggered sinusoid: 1.0013 vs 1.0009).
  ``Opts(M, ib_order=M)`` selects the full basis.
"""
import math
import itertools

import numpy as np

from . import taylor
from .geometry import BoundaryPoints, in_array, logical_shape, value


class RankError(RuntimeError):
    """A node could not be constrained at the largest radius and lowest order."""


class Opts:
    def __init__(self, M, eta_p=None, eta_v=0.0, radius=0.0, growth=3.0,
                 min_order=2, rank_tol=None, ib_order=0, extrap="nd"):
        self.M = int(M)
        # basis order of the extrapolants (<= M); 0 selects min(M, 4) (see basis)
        self.ib_order = int(ib_order)
        # pressure cut-off; None selects the default of eta_pressure(bc)
        self.eta_p = None if eta_p is None else float(eta_p)
        self.eta_v = float(eta_v)
        self.radius = float(radius)
        self.growth = float(growth)
        self.min_order = int(min_order)
        # rank tolerance; None selects the default of for_bc
        self.rank_tol = None if rank_tol is None else float(rank_tol)
        # "nd": N-dimensional basis over a hyperspherical support (the paper's
        # method); "1d": per-axis 1D extrapolation (laplacian_rows_1d)
        if extrap not in ("nd", "1d"):
            raise ValueError("extrap must be 'nd' or '1d'")
        self.extrap = extrap

    def for_bc(self, bc):
        """These options with the boundary-condition defaults filled in: rank
        tolerance 1e-3 (free) or 1e-2 (rigid); eta_p as eta_pressure(bc)."""
        out = Opts(self.M, eta_p=self.eta_pressure(bc), eta_v=self.eta_v, radius=self.radius,
                   growth=self.growth, min_order=self.min_order,
                   rank_tol=self.rank_tol if self.rank_tol is not None else (1e-3 if bc == "free" else 1e-2),
                   ib_order=self.ib_order, extrap=self.extrap)
        return out

    def eta_pressure(self, bc):
        """eta of the pressure fits: eta_p if set, else 0.5 for the free surface
        (the paper's value) and 0.25 for the rigid surface (the paper gives none;
        see the module notes)."""
        if self.eta_p is not None:
            return self.eta_p
        return 0.5 if bc == "free" else 0.25

    def basis(self, d):
        """Basis order of the extrapolants (d dimensions): ib_order if set, else min(M, 4)."""
        if self.ib_order:
            return self.ib_order
        return min(self.M, 4)


class Field:
    """One unknown field of the fit: node j sits at j + shift (grid units)."""

    def __init__(self, mask, shift, eta):
        self.mask = mask
        self.shift = np.asarray(shift, dtype=np.float64)
        self.eta = float(eta)


_SUPPORT_CACHE = {}


def _support_offsets(frac, r):
    """Offsets o (integer tuples) with |o - frac|_2 <= r, exact in quarter units,
    sorted by distance then array order; frac in {-1/2, 0, 1/2}^d."""
    key = (frac, r)
    hit = _SUPPORT_CACHE.get(key)
    if hit is not None:
        return hit
    d = len(frac)
    four_r2 = int(math.floor(4.0 * r * r + 1e-9))
    R = int(math.ceil(r)) + 1
    out = []
    for off in itertools.product(range(-R, R + 1), repeat=d):
        q = sum(int(round(2.0 * (o - f))) ** 2 for o, f in zip(off, frac))
        if q <= four_r2:
            out.append((q, tuple(reversed(off)), off))
    out.sort()
    res = [o for _, _, o in out]
    _SUPPORT_CACHE[key] = res
    return res


def support_nodes(xi0, shift, r, lshape):
    """In-array nodes j of a field with |j + shift - xi0|_2 <= r, sorted by
    distance, then by array-order index."""
    base = [int(round(x - s)) for x, s in zip(xi0, shift)]
    frac = tuple(float(x - s - b) for x, s, b in zip(xi0, shift, base))
    out = []
    for off in _support_offsets(frac, float(r)):
        j = tuple(b + o for b, o in zip(base, off))
        if in_array(j, lshape):
            out.append(j)
    return out


def fit(xi0, fields, bps, bc_rows_fn, E, opts, lshape):
    """Constrained extrapolation fit at expansion point xi0.

    fields     : list of Field
    bc_rows_fn : order -> BC template (``taylor.bc_templates_*``): rows of
                 per-field (normal axis, operator) terms
    E          : list of (field index, exterior position, standard weight)
    Returns (support, c, info): support = [(field, node)], c = correction
    weights of the modified operator on those nodes.
    """
    xi0 = np.asarray(xi0, dtype=np.float64)
    d = len(xi0)
    nf = len(fields)
    P0 = opts.basis(d)
    for Mp in range(P0, opts.min_order - 1, -2):
        idx = taylor.multi_indices(d, Mp)
        T = len(idx)
        if opts.radius > 0 and Mp == P0:
            r0 = opts.radius
        else:
            r0 = (Mp + 1) / 2.0
        for g in range(int(round(opts.growth / 0.5)) + 1):
            r = r0 + 0.5 * g
            sup = []
            for f, F in enumerate(fields):
                for j in support_nodes(xi0, F.shift, r, lshape):
                    if not value(F.mask, j):
                        continue
                    pos = np.array(j, dtype=np.float64) + F.shift
                    if bps.eta_excluded(pos, F.eta):
                        continue
                    sup.append((f, j, pos))
            blist = bps.within(xi0, r)
            rows = []
            for f in range(nf):
                P = [pos - xi0 for ff, _, pos in sup if ff == f]
                if P:
                    blk = np.zeros((len(P), nf * T))
                    blk[:, f * T:(f + 1) * T] = taylor.basis_rows(np.array(P), idx)
                    rows.extend(blk)
            if blist:
                rows.extend(taylor.template_rows(bc_rows_fn(Mp), bps.xb[blist] - xi0,
                                                 bps.normal[blist], idx, nf))
            if len(rows) < nf * T:
                continue
            A = np.array(rows)
            sv = np.linalg.svd(A, compute_uv=False)
            if not sv[-1] > opts.rank_tol * sv[0]:
                continue
            u = np.zeros(nf * T)
            for f, xe, w in E:
                u[f * T:(f + 1) * T] += w * taylor.basis_row(np.asarray(xe, dtype=np.float64) - xi0, idx)
            y = np.linalg.pinv(A).T @ u
            info = dict(radius=r, order=Mp, n_bp=len(blist), n_rows=A.shape[0],
                        n_int=len(sup), cond=float(sv[0] / sv[-1]), A=A, u=u, y=y,
                        support=[(f, j) for f, j, _ in sup])
            return [(f, j) for f, j, _ in sup], y[:len(sup)], info
    raise RankError("node at %s unconstrained" % (tuple(xi0),))


# ---------------------------------------------------------------------------
# 2nd-order form: merged modified Laplacian
# ---------------------------------------------------------------------------
def _shifted(mask, axis_arr, k):
    """out[i] = mask[i + k] along array axis (False outside the array)."""
    out = np.zeros_like(mask)
    n = mask.shape[axis_arr]
    src = [slice(None)] * mask.ndim
    dst = [slice(None)] * mask.ndim
    if k > 0:
        src[axis_arr] = slice(k, n)
        dst[axis_arr] = slice(0, n - k)
    else:
        src[axis_arr] = slice(0, n + k)
        dst[axis_arr] = slice(-k, n)
    out[tuple(dst)] = mask[tuple(src)]
    return out


def laplacian_ib_nodes(mask, M):
    """Interior nodes whose +-M/2 axial stencil reaches an in-array exterior node
    (logical tuples, array order)."""
    ext = ~mask
    hit = np.zeros_like(mask)
    d = mask.ndim
    for a in range(d):
        ax = d - 1 - a
        for k in list(range(-(M // 2), 0)) + list(range(1, M // 2 + 1)):
            hit |= _shifted(ext, ax, k)
    return [tuple(int(v) for v in reversed(i)) for i in np.argwhere(mask & hit)]


def scalar_bc_fn(bc, d):
    return lambda Mp: taylor.bc_templates_scalar(bc, d, Mp)


def vector_bc_fn(bc, d):
    return lambda Mp: taylor.bc_templates_vector(bc, d, Mp)


class Geometry:
    """Discretised SDF with its interior masks and boundary points."""

    def __init__(self, sdf, h, M):
        self.sdf = np.asarray(sdf, dtype=np.float64)
        self.h = float(h)
        self.M = int(M)
        self.sdf_g = self.sdf / self.h
        self.mask = self.sdf_g > 0.0
        self.lshape = logical_shape(self.sdf)
        self.d = len(self.lshape)
        self.bps = BoundaryPoints(self.sdf, self.h, self.M)

    def vmask(self, a):
        """Interior mask of the staggered v_a nodes (j + e_a/2): the mean of the
        SDF at the two neighbouring nodes is > 0 (own value at the array end)."""
        ax = self.d - 1 - a
        s = self.sdf_g
        n = s.shape[ax]
        nb = np.array(s, copy=True)
        sl_dst = [slice(None)] * s.ndim
        sl_src = [slice(None)] * s.ndim
        sl_dst[ax] = slice(0, n - 1)
        sl_src[ax] = slice(1, n)
        nb[tuple(sl_dst)] = s[tuple(sl_src)]
        return 0.5 * (s + nb) > 0.0


def laplacian_rows(geom, bc, opts, nodes=None):
    """Modified-Laplacian corrections at IB nodes (grid units; divide by h^2).

    Returns dict node -> (dict offset -> weight, info).
    """
    opts = opts.for_bc(bc)
    if opts.extrap == "1d":
        return laplacian_rows_1d(geom, bc, opts, nodes)
    M = opts.M
    w2 = [float(x) for x in taylor.central_second(M)]
    H = M // 2
    fields = [Field(geom.mask, np.zeros(geom.d), opts.eta_pressure(bc))]
    bcfn = scalar_bc_fn(bc, geom.d)
    if nodes is None:
        nodes = laplacian_ib_nodes(geom.mask, M)
    out = {}
    for node in nodes:
        E = []
        for a in range(geom.d):
            for k in list(range(-H, 0)) + list(range(1, H + 1)):
                nb = list(node)
                nb[a] += k
                if in_array(nb, geom.lshape) and not value(geom.mask, nb):
                    E.append((0, np.array(nb, dtype=np.float64), w2[k + H]))
        if not E:
            continue
        sup, c, info = fit(np.array(node, dtype=np.float64), fields, geom.bps, bcfn, E, opts, geom.lshape)
        wts = {}
        for (f, j), cj in zip(sup, c):
            off = tuple(jj - nn for jj, nn in zip(j, node))
            wts[off] = wts.get(off, 0.0) + float(cj)
        out[node] = (wts, info)
    return out


def extrapolation_1d(u_int, u_b, u_e, P, bc):
    """Weights e (one per interior point) of the 1D extrapolant of order P at u_e:
    f~(u_e) = sum_i e_i f(u_i).  Rows: the Taylor basis u^m / m! (m <= P) at the
    interior points u_int, and its derivatives of the free-surface conditions
    p = 0, p'' = 0, .. (orders 0, 2, .. <= P) at u_b with right-hand side zero
    ("Reduction to 1D"); solved with the pseudoinverse (the inverse: the system
    is square)."""
    if bc != "free":
        raise ValueError("the 1D reduction is stated for the free surface")
    m = np.arange(P + 1)
    fact = np.array([math.factorial(int(k)) for k in m], dtype=np.float64)
    rows = [np.asarray(u, dtype=np.float64) ** m / fact for u in u_int]
    for j in range(0, P + 1, 2):
        r = np.zeros(P + 1)
        for k in range(j, P + 1):
            r[k] = u_b ** (k - j) / math.factorial(k - j)
        rows.append(r)
    A = np.array(rows)
    phi_e = np.asarray(u_e, dtype=np.float64) ** m / fact
    return (phi_e @ np.linalg.pinv(A))[:len(u_int)]


def laplacian_rows_1d(geom, bc, opts, nodes=None):
    """Modified-Laplacian corrections from per-axis 1D extrapolation, the variant
    the paper relates to Mulder's scheme ("Reduction to 1D").  For each axis and
    each side of an IB row's axial stencil that reaches in-array exterior nodes:
    the boundary is where the SDF, interpolated linearly between the last
    interior node and the first exterior node on that side, crosses zero (a
    reading: the paper places 1D boundary points on the grid line without
    saying how); the interior points are the P/2 nodes on the line, moving away
    from the boundary, at more than eta from it, for a square system with the
    P/2 + 1 conditions of order <= P; P = M, lowered by 2 while the line holds
    too few such nodes.  Every exterior node of that side takes the
    extrapolated value.  Corrections are summed over axes and sides.  Free
    surface only: the paper states the reduction for p = 0, p'' = 0, ...
    info: radius 0, order = the lowest P used."""
    if bc != "free":
        raise ValueError("the 1D reduction is stated for the free surface")
    M = opts.M
    H = M // 2
    w2 = [float(x) for x in taylor.central_second(M)]
    eta = opts.eta_pressure(bc)
    sdf = geom.sdf_g
    if nodes is None:
        nodes = laplacian_ib_nodes(geom.mask, M)
    out = {}
    for node in nodes:
        wts = {}
        pmin = M
        for a in range(geom.d):
            for sg in (1, -1):
                ext = []
                for k in range(1, H + 1):
                    nb = list(node)
                    nb[a] += sg * k
                    if in_array(nb, geom.lshape) and not value(geom.mask, nb):
                        ext.append(k)
                if not ext:
                    continue
                kb = ext[0]
                n_in = list(node)
                n_in[a] += sg * (kb - 1)
                n_ex = list(node)
                n_ex[a] += sg * kb
                s1, s2 = value(sdf, n_in), value(sdf, n_ex)
                u_b = (kb - 1) + s1 / (s1 - s2)
                cand = []
                u = kb - 1
                while True:
                    nb = list(node)
                    nb[a] += sg * u
                    if not in_array(nb, geom.lshape) or not value(geom.mask, nb):
                        break
                    if u_b - u > eta:
                        cand.append(u)
                    u -= 1
                    if len(cand) > M:
                        break
                P = M
                while P > 0 and len(cand) < P // 2:
                    P -= 2
                need = P // 2
                pmin = min(pmin, P)
                if need == 0:
                    continue            # order 0: the extrapolant is zero
                pts = cand[:need]
                for k in ext:
                    e = extrapolation_1d(pts, u_b, k, P, bc)
                    for ui, ei in zip(pts, e):
                        off = [0] * geom.d
                        off[a] = sg * ui
                        off = tuple(off)
                        wts[off] = wts.get(off, 0.0) + w2[H + k] * float(ei)
        out[node] = (wts, dict(radius=0.0, order=pmin, n_bp=0, cond=1.0))
    return out


# ---------------------------------------------------------------------------
# 1st-order staggered form
# ---------------------------------------------------------------------------
def gradient_ib_nodes(geom, a, M):
    """Interior v_a nodes j whose forward-staggered d/dx_a stencil
    (p at j + k e_a, k = -M/2+1 .. M/2) reaches an in-array exterior p node."""
    vm = geom.vmask(a)
    ext = ~geom.mask
    ax = geom.d - 1 - a
    hit = np.zeros_like(vm)
    for k in range(-(M // 2) + 1, M // 2 + 1):
        hit |= _shifted(ext, ax, k)
    return [tuple(int(v) for v in reversed(i)) for i in np.argwhere(vm & hit)]


def divergence_ib_nodes(geom, M):
    """Interior p nodes whose backward-staggered divergence stencils
    (v_a at j + k e_a, k = -M/2 .. M/2-1) reach an in-array exterior v node."""
    hit = np.zeros_like(geom.mask)
    for a in range(geom.d):
        ext = ~geom.vmask(a)
        ax = geom.d - 1 - a
        for k in range(-(M // 2), M // 2):
            hit |= _shifted(ext, ax, k)
    return [tuple(int(v) for v in reversed(i)) for i in np.argwhere(geom.mask & hit)]


def gradient_rows(geom, a, bc, opts, nodes=None):
    """Corrections of the modified d/dx_a (grid units; divide by h) at v_a nodes.

    Expansion point: the v_a node position j + e_a/2; fit on the pressure
    field with the pressure BC hierarchy and eta_p.
    Returns dict node j -> (dict p-offset -> weight, info).
    """
    opts = opts.for_bc(bc)
    M = opts.M
    c = [float(x) for x in taylor.staggered_first(M)]      # at offsets -(M-1)/2..(M-1)/2
    fields = [Field(geom.mask, np.zeros(geom.d), opts.eta_pressure(bc))]
    bcfn = scalar_bc_fn(bc, geom.d)
    if nodes is None:
        nodes = gradient_ib_nodes(geom, a, M)
    ea = np.zeros(geom.d)
    ea[a] = 0.5
    out = {}
    for node in nodes:
        E = []
        for k in range(-(M // 2) + 1, M // 2 + 1):
            nb = list(node)
            nb[a] += k
            if in_array(nb, geom.lshape) and not value(geom.mask, nb):
                E.append((0, np.array(nb, dtype=np.float64), c[k + M // 2 - 1]))
        if not E:
            continue
        xi0 = np.array(node, dtype=np.float64) + ea
        sup, cc, info = fit(xi0, fields, geom.bps, bcfn, E, opts, geom.lshape)
        wts = {}
        for (f, j), cj in zip(sup, cc):
            off = tuple(jj - nn for jj, nn in zip(j, node))
            wts[off] = wts.get(off, 0.0) + float(cj)
        out[node] = (wts, info)
    return out


def divergence_rows(geom, bc, opts, nodes=None):
    """Corrections of the modified divergence (grid units; divide by h) at p nodes.

    Expansion point: the p node; coupled fit on all velocity components with
    the velocity BC hierarchy and eta_v.
    Returns dict node -> (dict (component, v-offset) -> weight, info).
    """
    opts = opts.for_bc(bc)
    M = opts.M
    d = geom.d
    c = [float(x) for x in taylor.staggered_first(M)]
    fields = []
    for a in range(d):
        sh = np.zeros(d)
        sh[a] = 0.5
        fields.append(Field(geom.vmask(a), sh, opts.eta_v))
    vmasks = [F.mask for F in fields]
    bcfn = vector_bc_fn(bc, d)
    if nodes is None:
        nodes = divergence_ib_nodes(geom, M)
    out = {}
    for node in nodes:
        E = []
        for a in range(d):
            for k in range(-(M // 2), M // 2):
                nb = list(node)
                nb[a] += k
                if in_array(nb, geom.lshape) and not value(vmasks[a], nb):
                    pos = np.array(nb, dtype=np.float64)
                    pos[a] += 0.5
                    E.append((a, pos, c[k + M // 2]))
        if not E:
            continue
        sup, cc, info = fit(np.array(node, dtype=np.float64), fields, geom.bps, bcfn, E, opts, geom.lshape)
        wts = {}
        for (f, j), cj in zip(sup, cc):
            off = (f,) + tuple(jj - nn for jj, nn in zip(j, node))
            wts[off] = wts.get(off, 0.0) + float(cj)
        out[node] = (wts, info)
    return out
