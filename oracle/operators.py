"""Modified operators assembled as sparse matrices (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Rows are the standard interior stencils with exterior columns removed (the
exterior field is identically zero), plus the immersed-boundary corrections of
``stencils``.  Rows and columns of exterior nodes are empty.  Node numbering is
the array-order flat index.

Paper: modified operators replace the interior stencils near the boundary
("Reconciliation with the Interior Numerical Discretization"); the Laplacian
is the sum of per-axis second derivatives (2nd-order application section); the
first-order form uses backward-staggered base stencils (1st-order section).
"""
import numpy as np
import scipy.sparse as sp

from . import taylor
from . import stencils


def _strides(shape):
    st = [1] * len(shape)
    for i in range(len(shape) - 2, -1, -1):
        st[i] = st[i + 1] * shape[i + 1]
    return st


def _axial_pairs(shape, row_mask, col_mask, a, k):
    """(row, col) flat index pairs with col = row + k e_a (logical axis a),
    both in the array, row in row_mask and col in col_mask."""
    d = len(shape)
    ax = d - 1 - a
    n = shape[ax]
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    sl_r = [slice(None)] * d
    sl_c = [slice(None)] * d
    if k >= 0:
        sl_r[ax] = slice(0, n - k)
        sl_c[ax] = slice(k, n)
    else:
        sl_r[ax] = slice(-k, n)
        sl_c[ax] = slice(0, n + k)
    r = idx[tuple(sl_r)]
    c = idx[tuple(sl_c)]
    ok = row_mask[tuple(sl_r)] & col_mask[tuple(sl_c)]
    return r[ok], c[ok]


def _flat(node, shape):
    st = _strides(shape)
    return sum(i * s for i, s in zip(reversed(node), st))


def laplacian_matrix(geom, bc, opts, ib_rows=None):
    """Modified Laplacian (1/h^2 units) restricted to interior nodes."""
    shape = geom.sdf.shape
    N = int(np.prod(shape))
    M = opts.M
    H = M // 2
    w2 = [float(x) for x in taylor.central_second(M)]
    rows, cols, vals = [], [], []
    for a in range(geom.d):
        for k in range(-H, H + 1):
            if k == 0 and a > 0:
                continue
            wk = w2[k + H] * (geom.d if k == 0 else 1)
            r, c = _axial_pairs(shape, geom.mask, geom.mask, a, k)
            rows.append(r)
            cols.append(c)
            vals.append(np.full(r.shape, wk))
    if ib_rows is None:
        ib_rows = stencils.laplacian_rows(geom, bc, opts)
    for node, (wts, _) in ib_rows.items():
        i = _flat(node, shape)
        for off, w in wts.items():
            j = _flat(tuple(n + o for n, o in zip(node, off)), shape)
            rows.append(np.array([i]))
            cols.append(np.array([j]))
            vals.append(np.array([w]))
    L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    L.sum_duplicates()
    return L / (geom.h * geom.h), ib_rows


def staggered_matrices(geom, bc, opts, grad_rows=None, div_rows=None):
    """Modified forward-staggered gradients G_a (v_a rows, p columns) and the
    modified backward-staggered divergence D (p rows, [v_0 .. v_{d-1}] columns),
    in 1/h units, restricted to interior nodes of each field."""
    shape = geom.sdf.shape
    N = int(np.prod(shape))
    M = opts.M
    H = M // 2
    c = [float(x) for x in taylor.staggered_first(M)]
    vm = [geom.vmask(a) for a in range(geom.d)]
    if grad_rows is None:
        grad_rows = [stencils.gradient_rows(geom, a, bc, opts) for a in range(geom.d)]
    if div_rows is None:
        div_rows = stencils.divergence_rows(geom, bc, opts)
    G = []
    for a in range(geom.d):
        rows, cols, vals = [], [], []
        for k in range(-H + 1, H + 1):          # p at j + k e_a, offset k - 1/2
            r, cc = _axial_pairs(shape, vm[a], geom.mask, a, k)
            rows.append(r)
            cols.append(cc)
            vals.append(np.full(r.shape, c[k + H - 1]))
        for node, (wts, _) in grad_rows[a].items():
            i = _flat(node, shape)
            for off, w in wts.items():
                rows.append(np.array([i]))
                cols.append(np.array([_flat(tuple(n + o for n, o in zip(node, off)), shape)]))
                vals.append(np.array([w]))
        Ga = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(N, N)).tocsr()
        Ga.sum_duplicates()
        G.append(Ga / geom.h)
    rows, cols, vals = [], [], []
    for a in range(geom.d):
        for k in range(-H, H):                  # v_a at j + k e_a, offset k + 1/2
            r, cc = _axial_pairs(shape, geom.mask, vm[a], a, k)
            rows.append(r)
            cols.append(cc + a * N)
            vals.append(np.full(r.shape, c[k + H]))
    for node, (wts, _) in div_rows.items():
        i = _flat(node, shape)
        for off, w in wts.items():
            comp, o = off[0], off[1:]
            rows.append(np.array([i]))
            cols.append(np.array([comp * N + _flat(tuple(n + q for n, q in zip(node, o)), shape)]))
            vals.append(np.array([w]))
    D = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, geom.d * N)).tocsr()
    D.sum_duplicates()
    return G, D / geom.h, grad_rows, div_rows
