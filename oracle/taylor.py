"""Truncated Taylor basis, derivative operators and 1D stencil weights (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper sections followed:
* "Constructing Finite-Difference Approximations": the 1D Taylor system
  A delta = f(x) whose inverse gives stencil weights for every derivative order
  (printed M=2 example), the N-D basis truncated at total degree M, and the
  grid-scaled derivative vector (unknowns Delta x^k d^k f, i.e. grid units).
* "Approximating Boundary Conditions": a linear BC operator applied to the
  basis gives one row of A (Eq. for the BC dot product).
* Free-surface constraints (2nd-order form): p = 0, lap p = 0, lap^2 p = 0, ...
  with conditions of order above M discarded.
* Velocity free surface (1st-order form): div v = 0, lap div v = 0, ...
"""
from fractions import Fraction
import functools
import itertools
import math

import numpy as np


# ---------------------------------------------------------------------------
# multi-indices of the truncated basis
# ---------------------------------------------------------------------------
def multi_indices(d, M):
    """Exponent tuples k (k[0] = x power, ...) with sum(k) <= M.

    Ordered by total degree, then lexicographically with the x power
    descending: (1, x, y, x^2/2, xy, y^2/2, ...) as in the paper's a-vector.
    """
    out = []
    for deg in range(M + 1):
        ks = [k for k in itertools.product(range(deg + 1), repeat=d) if sum(k) == deg]
        ks.sort(reverse=True)
        out.extend(ks)
    return out


def n_terms(d, M):
    """Number of basis terms: M+1, (M+1)(M+2)/2, (M+1)(M+2)(M+3)/6."""
    return len(multi_indices(d, M))


# ---------------------------------------------------------------------------
# constant-coefficient differential operators  {alpha: coefficient}
# ---------------------------------------------------------------------------
def op_identity(d):
    return {(0,) * d: 1.0}


def op_partial(d, axis):
    a = [0] * d
    a[axis] = 1
    return {tuple(a): 1.0}


def op_mul(p, q):
    """Composition of two constant-coefficient operators (alphas add)."""
    out = {}
    for a, ca in p.items():
        for b, cb in q.items():
            key = tuple(x + y for x, y in zip(a, b))
            out[key] = out.get(key, 0.0) + ca * cb
    return out


def op_add(p, q, cq=1.0):
    out = dict(p)
    for b, cb in q.items():
        out[b] = out.get(b, 0.0) + cq * cb
    return out


def op_scale(p, c):
    return {a: c * v for a, v in p.items()}


def op_laplacian(d):
    out = {}
    for i in range(d):
        a = [0] * d
        a[i] = 2
        out[tuple(a)] = 1.0
    return out


def op_power(p, k, d):
    out = op_identity(d)
    for _ in range(k):
        out = op_mul(out, p)
    return out


def op_order(p):
    return max(sum(a) for a in p)


# ---------------------------------------------------------------------------
# rows of A
# ---------------------------------------------------------------------------
def _deriv_monomial(xi, k, alpha):
    """d^alpha of prod_i xi_i^k_i / k_i!  evaluated at xi."""
    v = 1.0
    for x, ki, ai in zip(xi, k, alpha):
        if ki < ai:
            return 0.0
        e = ki - ai
        v *= x ** e / math.factorial(e)
    return v


def basis_row(xi, idx):
    """Taylor row a(xi) = (prod xi_i^k_i / k_i!)_k  (paper's a-vector)."""
    return basis_rows(np.asarray(xi, dtype=np.float64)[None, :], idx)[0]


def op_row(op, xi, idx):
    """Row of the BC dot product: (sum_alpha c_alpha d^alpha a)(xi)."""
    return op_rows(op, np.asarray(xi, dtype=np.float64)[None, :], idx)[0]


def basis_row_scalar(xi, idx):
    """Element-by-element form of ``basis_row`` (kept as its definition)."""
    return np.array([_deriv_monomial(xi, k, (0,) * len(xi)) for k in idx], dtype=np.float64)


def op_row_scalar(op, xi, idx):
    """Element-by-element form of ``op_row`` (kept as its definition)."""
    row = np.zeros(len(idx), dtype=np.float64)
    for alpha, c in op.items():
        for j, k in enumerate(idx):
            row[j] += c * _deriv_monomial(xi, k, alpha)
    return row


def _power_table(XI, M):
    """P[n, a, e] = XI[n, a]^e / e!  for e = 0..M."""
    n, d = XI.shape
    P = np.ones((n, d, M + 1))
    for e in range(1, M + 1):
        P[:, :, e] = P[:, :, e - 1] * XI / e
    return P


def basis_rows(XI, idx):
    """basis_row for many points at once: (n, T)."""
    return op_rows({(0,) * XI.shape[1]: 1.0}, XI, idx)


def op_rows(op, XI, idx):
    """op_row for many points at once: (n, T)."""
    XI = np.asarray(XI, dtype=np.float64)
    K = np.array(idx, dtype=np.int64)                # (T, d)
    Mx = int(K.max()) if K.size else 0
    P = _power_table(XI, Mx)
    n, d = XI.shape
    out = np.zeros((n, len(idx)))
    for alpha, c in op.items():
        E = K - np.array(alpha, dtype=np.int64)[None, :]
        ok = np.all(E >= 0, axis=1)
        Ec = np.clip(E, 0, None)
        v = np.ones((n, len(idx)))
        for a in range(d):
            v = v * P[:, a, Ec[:, a]]
        out += c * v * ok[None, :]
    return out


# ---------------------------------------------------------------------------
# boundary-condition hierarchies
# ---------------------------------------------------------------------------
def bc_rows_scalar(bc, d, M, normal):
    """Operators imposed on a scalar field (pressure) at one boundary point.

    free : lap^k p = 0 for 2k <= M (p = 0, lap p = 0, lap^2 p = 0, ...).
    rigid: n . grad lap^k p = 0 for 2k+1 <= M (zero normal particle velocity
           and its time derivatives through the wave equation).
    Returns a list of operators (one per row).
    """
    L = op_laplacian(d)
    rows = []
    if bc == "free":
        k = 0
        while 2 * k <= M:
            rows.append(op_power(L, k, d))
            k += 1
    elif bc == "rigid":
        k = 0
        while 2 * k + 1 <= M:
            nd = {}
            for a in range(d):
                nd = op_add(nd, op_partial(d, a), float(normal[a]))
            rows.append(op_mul(nd, op_power(L, k, d)))
            k += 1
    else:
        raise ValueError(bc)
    return rows


def bc_rows_vector(bc, d, M, normal):
    """Coupled rows on the particle-velocity components (v_0 .. v_{d-1}).

    Each row is a list of d operators, one per component block.
    free : lap^k div v = 0 for 2k+1 <= M.
    rigid: n . v = 0, and n . grad lap^k div v = 0 for 2k+2 <= M (zero normal
           velocity and its time derivatives), plus lap^k curl v = 0 for
           2k+1 <= M: the acoustic velocity of the first-order system is
           irrotational (v_t = grad p / rho with constant rho), which fixes the
           tangential extrapolation.  Reading: the paper gives no velocity
           conditions for a rigid surface; without the curl rows the staggered
           rigid scheme grows exponentially on a sinusoidal surface.
    """
    L = op_laplacian(d)
    rows = []
    if bc == "free":
        k = 0
        while 2 * k + 1 <= M:
            Lk = op_power(L, k, d)
            rows.append([op_mul(op_partial(d, a), Lk) for a in range(d)])
            k += 1
    elif bc == "rigid":
        rows.append([op_scale(op_identity(d), float(normal[a])) for a in range(d)])
        k = 0
        while 2 * k + 2 <= M:
            Lk = op_power(L, k, d)
            nd = {}
            for b in range(d):
                nd = op_add(nd, op_partial(d, b), float(normal[b]))
            rows.append([op_mul(op_mul(nd, op_partial(d, a)), Lk) for a in range(d)])
            k += 1
        k = 0
        while 2 * k + 1 <= M:
            Lk = op_power(L, k, d)
            for (i, j) in _curl_pairs(d):
                row = [{} for _ in range(d)]
                row[j] = op_mul(op_partial(d, i), Lk)
                row[i] = op_scale(op_mul(op_partial(d, j), Lk), -1.0)
                rows.append(row)
            k += 1
    else:
        raise ValueError(bc)
    return rows


def _curl_pairs(d):
    """Index pairs (i, j) of the curl components d_i v_j - d_j v_i."""
    return [(0, 1)] if d == 2 else [(1, 2), (2, 0), (0, 1)]


# ---------------------------------------------------------------------------
# 1D stencils from the Taylor system (exact rationals)
# ---------------------------------------------------------------------------
def _exact_inverse(A):
    n = len(A)
    M = [list(r) + [Fraction(int(i == j)) for j in range(n)] for i, r in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        pv = M[c][c]
        M[c] = [x / pv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [row[n:] for row in M]


def taylor_stencil(offsets, deriv):
    """Weights of the `deriv`-th derivative (times h^deriv) at 0 from f at `offsets`.

    Builds the square Taylor system A delta = f with A[j][m] = o_j^m / m!
    and returns row `deriv` of A^{-1} as exact Fractions.
    """
    offs = [Fraction(o) for o in offsets]
    n = len(offs)
    A = [[o ** m / math.factorial(m) for m in range(n)] for o in offs]
    return _exact_inverse(A)[deriv]


@functools.lru_cache(maxsize=None)
def central_second(M):
    """Order-M central 2nd-derivative weights at offsets -M/2..M/2."""
    return taylor_stencil(range(-M // 2, M // 2 + 1), 2)


@functools.lru_cache(maxsize=None)
def central_first(M):
    """Order-M central 1st-derivative weights at offsets -M/2..M/2."""
    return taylor_stencil(range(-M // 2, M // 2 + 1), 1)


@functools.lru_cache(maxsize=None)
def staggered_first(M):
    """Order-M staggered 1st-derivative weights at offsets -(M-1)/2 .. (M-1)/2."""
    offs = [Fraction(2 * j - M + 1, 2) for j in range(M)]
    return taylor_stencil(offs, 1)


# Templates: the same hierarchies with the normal factored out, so a row for
# many boundary points can be evaluated at once.  A template is a list of rows;
# a row is a list (one per field) of lists of terms (axis, operator); a term
# contributes normal[axis] * op (or op when axis is None).
def bc_templates_scalar(bc, d, M):
    L = op_laplacian(d)
    rows = []
    if bc == "free":
        k = 0
        while 2 * k <= M:
            rows.append([[(None, op_power(L, k, d))]])
            k += 1
    elif bc == "rigid":
        k = 0
        while 2 * k + 1 <= M:
            Lk = op_power(L, k, d)
            rows.append([[(a, op_mul(op_partial(d, a), Lk)) for a in range(d)]])
            k += 1
    else:
        raise ValueError(bc)
    return rows


def bc_templates_vector(bc, d, M):
    L = op_laplacian(d)
    rows = []
    if bc == "free":
        k = 0
        while 2 * k + 1 <= M:
            Lk = op_power(L, k, d)
            rows.append([[(None, op_mul(op_partial(d, a), Lk))] for a in range(d)])
            k += 1
    elif bc == "rigid":
        rows.append([[(a, op_identity(d))] for a in range(d)])
        k = 0
        while 2 * k + 2 <= M:
            Lk = op_power(L, k, d)
            rows.append([[(b, op_mul(op_mul(op_partial(d, b), op_partial(d, a)), Lk)) for b in range(d)]
                         for a in range(d)])
            k += 1
        k = 0
        while 2 * k + 1 <= M:
            Lk = op_power(L, k, d)
            for (i, j) in _curl_pairs(d):
                row = [[] for _ in range(d)]
                row[j].append((None, op_mul(op_partial(d, i), Lk)))
                row[i].append((None, op_scale(op_mul(op_partial(d, j), Lk), -1.0)))
                rows.append(row)
            k += 1
    else:
        raise ValueError(bc)
    return rows


def template_rows(template, XB, NRM, idx, nf):
    """Evaluate a BC template at boundary points XB (n, d) with normals NRM:
    returns (n * len(template), nf * T), rows grouped by boundary point."""
    T = len(idx)
    n = XB.shape[0]
    out = np.zeros((n, len(template), nf * T))
    for r, row in enumerate(template):
        for f, terms in enumerate(row):
            for axis, op in terms:
                v = op_rows(op, XB, idx)
                if axis is not None:
                    v = v * NRM[:, axis:axis + 1]
                out[:, r, f * T:(f + 1) * T] += v
    return out.reshape(n * len(template), nf * T)
