"""Geometry on the FD grid: interior mask, boundary points, eta cut-off (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Conventions (shared with the inputs, not with the CUDA code):
* arrays are stored with the slowest axis first, i.e. 2D ``[nz][nx]`` and 3D
  ``[nz][ny][nx]``; logical axis 0 is x (the last array axis) and logical axis
  d-1 is z (depth, the first array axis);
* positions xi are in grid units, logical order (x, [y,] z), node (i_x, .., i_z)
  sits at xi = (i_x, .., i_z);
* the signed-distance function s is positive in the physical domain; a node with
  s <= 0 is exterior.

Paper: the topography is an SDF discretised on the FD grid (Examples, 2D free
surface).  Boundary points are where the boundary normal through a grid point
meets the surface, kept if they lie inside the point-centred unit
hyperrectangle; interior points with a boundary point inside their
2 eta-sided box are left out of the fit (boundary-point paragraph of
"Approximating Boundary Conditions").
"""
import itertools
import math

import numpy as np

from . import taylor


def logical_shape(sdf):
    return tuple(reversed(sdf.shape))


def value(arr, node):
    """arr at logical node index (i_x, .., i_z)."""
    return arr[tuple(reversed(node))]


def in_array(node, lshape):
    return all(0 <= i < n for i, n in zip(node, lshape))


def interior_mask(sdf):
    """True where s > 0 (a node exactly on the surface is exterior)."""
    return sdf > 0.0


def sdf_gradient(sdf_g, node, M):
    """Gradient of the discretised SDF (grid units) at a node.

    Along each axis: the widest even-order central first-derivative stencil,
    of order at most M, that fits inside the array; a one-sided first
    difference at the array edge.
    """
    lshape = logical_shape(sdf_g)
    d = len(lshape)
    g = np.zeros(d)
    for a in range(d):
        i, n = node[a], lshape[a]
        q = min(M, 2 * min(i, n - 1 - i))
        q -= q % 2
        def at(k):
            nn = list(node)
            nn[a] = i + k
            return value(sdf_g, nn)
        if q >= 2:
            w = taylor.central_first(q)
            acc = 0.0
            for kk in range(1, q // 2 + 1):
                acc += float(w[q // 2 + kk]) * (at(kk) - at(-kk))
            g[a] = acc
        elif i == 0:
            g[a] = at(1) - at(0)
        else:
            g[a] = at(0) - at(-1)
    return g


class BoundaryPoints:
    """Boundary points x_b, one at most per grid node (its owner).

    Attributes: owners (list of logical node tuples), xb (n, d) grid units,
    normal (n, d) unit outward-into-domain normals (grad s / |grad s|),
    and ``by_owner`` dict owner -> index.
    """

    def __init__(self, sdf, h, M):
        sdf_g = np.asarray(sdf, dtype=np.float64) / h
        lshape = logical_shape(sdf_g)
        d = len(lshape)
        lim = math.sqrt(d) / 2.0
        owners, xb, nrm = [], [], []
        cand = np.argwhere(np.abs(sdf_g) <= lim)          # array-order indices
        for idx in cand:
            node = tuple(int(v) for v in reversed(idx))
            s = value(sdf_g, node)
            g = sdf_gradient(sdf_g, node, M)
            gn = math.sqrt(float(np.dot(g, g)))
            if gn == 0.0:
                continue
            n = g / gn
            off = -s * n
            if np.max(np.abs(off)) <= 0.5:
                owners.append(node)
                xb.append(np.array(node, dtype=np.float64) + off)
                nrm.append(n)
        # deterministic order: by linear (array-order) index
        order = sorted(range(len(owners)), key=lambda j: tuple(reversed(owners[j])))
        self.owners = [owners[j] for j in order]
        self.xb = np.array([xb[j] for j in order]).reshape(-1, d)
        self.normal = np.array([nrm[j] for j in order]).reshape(-1, d)
        self.by_owner = {o: j for j, o in enumerate(self.owners)}
        self.d = d
        self.lshape = lshape

    def near(self, xi, dist_inf):
        """Indices of boundary points whose owner is within `dist_inf`+0.5 of xi
        in the infinity norm (a superset of points within dist_inf of xi)."""
        reach = int(math.floor(dist_inf + 0.5)) + 1
        base = [int(math.floor(x)) for x in xi]
        out = []
        for off in itertools.product(range(-reach, reach + 2), repeat=self.d):
            o = tuple(b + k for b, k in zip(base, off))
            j = self.by_owner.get(o)
            if j is not None:
                out.append(j)
        return sorted(set(out))

    def eta_excluded(self, xi, eta):
        """True if a boundary point lies strictly inside the box |x - xi|_inf < eta."""
        if eta <= 0.0:
            return False
        for j in self.near(xi, eta):
            if np.max(np.abs(self.xb[j] - np.asarray(xi))) < eta:
                return True
        return False

    def within(self, xi, r):
        """Boundary points with |x_b - xi|_2 <= r (absolute slack 1e-9)."""
        out = []
        for j in self.near(xi, r):
            dv = self.xb[j] - np.asarray(xi)
            if float(np.dot(dv, dv)) <= r * r + 1e-9:
                out.append(j)
        return out
