"""Pins of the oracle's basis, BC rows and 1D stencils against the paper and
against independent textbook constructions (no GPU)."""
from fractions import Fraction
import os

import numpy as np
import pytest
import sympy

from oracle import taylor

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line)
    return out


def test_printed_m2_inverse():
    """The paper prints the inverse of the M=2 grid-unit Taylor system."""
    rows = [[Fraction(x) for x in r.split()] for r in _read_rows("taylor_m2_inverse.txt")]
    for k in range(3):
        assert taylor.taylor_stencil([-1, 0, 1], k) == rows[k]


def fornberg(z, x, m):
    """Fornberg's recursion (Math. Comp. 1988) for weights of derivatives 0..m
    at z from nodes x, in exact arithmetic.  Independent of the Taylor inverse."""
    n = len(x) - 1
    c = [[Fraction(0)] * (m + 1) for _ in range(n + 1)]
    c1 = Fraction(1)
    c4 = x[0] - z
    c[0][0] = Fraction(1)
    for i in range(1, n + 1):
        mn = min(i, m)
        c2 = Fraction(1)
        c5 = c4
        c4 = x[i] - z
        for j in range(i):
            c3 = x[i] - x[j]
            c2 = c2 * c3
            if j == i - 1:
                for k in range(mn, 0, -1):
                    c[i][k] = c1 * (k * c[i - 1][k - 1] - c5 * c[i - 1][k]) / c2
                c[i][0] = -c1 * c5 * c[i - 1][0] / c2
            for k in range(mn, 0, -1):
                c[j][k] = (c4 * c[j][k] - k * c[j][k - 1]) / c3
            c[j][0] = c4 * c[j][0] / c3
        c1 = c2
    return c


@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_central_second_vs_fornberg(M):
    x = [Fraction(k) for k in range(-M // 2, M // 2 + 1)]
    c = fornberg(Fraction(0), x, 2)
    assert taylor.central_second(M) == [c[j][2] for j in range(len(x))]
    assert taylor.central_first(M) == [c[j][1] for j in range(len(x))]


@pytest.mark.parametrize("M", [2, 4, 6, 8])
def test_staggered_first_vs_fornberg(M):
    x = [Fraction(2 * j - M + 1, 2) for j in range(M)]
    c = fornberg(Fraction(0), x, 1)
    assert taylor.staggered_first(M) == [c[j][1] for j in range(len(x))]


def test_textbook_values():
    assert taylor.central_second(4) == [Fraction(-1, 12), Fraction(4, 3), Fraction(-5, 2),
                                        Fraction(4, 3), Fraction(-1, 12)]
    assert taylor.staggered_first(4) == [Fraction(1, 24), Fraction(-9, 8), Fraction(9, 8),
                                         Fraction(-1, 24)]


@pytest.mark.parametrize("M", [2, 4, 8])
def test_stencil_exactness(M):
    """Order-M second derivative is exact on x^k, k <= M+1 (symmetry adds one)."""
    w = taylor.central_second(M)
    offs = range(-M // 2, M // 2 + 1)
    for k in range(M + 2):
        got = sum(wj * Fraction(o) ** k for wj, o in zip(w, offs))
        want = Fraction(k * (k - 1)) * (0 ** (k - 2) if k >= 2 else 0)
        assert got == want


def test_term_counts():
    """(M+1)(M+2)/2 in 2D and (M+1)(M+2)(M+3)/6 in 3D (rank paragraph)."""
    for M in (2, 4, 6, 8):
        assert taylor.n_terms(1, M) == M + 1
        assert taylor.n_terms(2, M) == (M + 1) * (M + 2) // 2
        assert taylor.n_terms(3, M) == (M + 1) * (M + 2) * (M + 3) // 6
    assert [taylor.n_terms(2, 4), taylor.n_terms(2, 8), taylor.n_terms(3, 4), taylor.n_terms(3, 8)] \
        == [15, 45, 35, 165]


def test_printed_bc_rows_2d_order4():
    idx = taylor.multi_indices(2, 4)
    ops = taylor.bc_rows_scalar("free", 2, 4, None)
    assert len(ops) == 3
    rng = np.random.default_rng(7)
    for _ in range(5):
        X, Y = rng.uniform(-2.5, 2.5, 2)
        for line, op in zip(_read_rows("bc_rows_2d_order4.txt"), ops):
            name, expr = line.split("|")
            want = np.array(eval("[" + expr + "]", {"X": X, "Y": Y}), dtype=float)
            got = taylor.op_row(op, (X, Y), idx)
            np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_printed_velocity_row():
    idx = taylor.multi_indices(2, 2)
    rows = taylor.bc_rows_vector("free", 2, 2, None)
    assert len(rows) == 1        # lap div v is order 3 > 2 and is discarded
    expr = _read_rows("velocity_row_2d_order2.txt")[0]
    for X, Y in [(0.3, -0.45), (-1.2, 0.8)]:
        want = np.array(eval("[" + expr + "]", {"X": X, "Y": Y}), dtype=float)
        got = np.concatenate([taylor.op_row(op, (X, Y), idx) for op in rows[0]])
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d,M", [(2, 4), (2, 8), (3, 4)])
@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_bc_rows_vs_sympy(d, M, bc):
    """Rows equal the BC operator applied to the Taylor polynomial, derived
    independently by sympy differentiation of sum_k delta_k (x-x0)^k / k!."""
    syms = sympy.symbols("x0:%d" % d)
    idx = taylor.multi_indices(d, M)
    dl = sympy.symbols("c0:%d" % len(idx))
    poly = sum(c * sympy.prod([s ** k / sympy.factorial(k) for s, k in zip(syms, kk)])
               for c, kk in zip(dl, idx))
    rng = np.random.default_rng(d * 10 + M)
    nrm = rng.normal(size=d)
    nrm /= np.linalg.norm(nrm)
    xb = rng.uniform(-2, 2, d)
    lap = lambda f: sum(sympy.diff(f, s, 2) for s in syms)
    exprs = []
    if bc == "free":
        f = poly
        k = 0
        while 2 * k <= M:
            exprs.append(f)
            f = lap(f)
            k += 1
    else:
        f = poly
        k = 0
        while 2 * k + 1 <= M:
            exprs.append(sum(float(n) * sympy.diff(f, s) for n, s in zip(nrm, syms)))
            f = lap(f)
            k += 1
    ops = taylor.bc_rows_scalar(bc, d, M, nrm)
    assert len(ops) == len(exprs)
    sub = dict(zip(syms, xb))
    for e, op in zip(exprs, ops):
        e = sympy.expand(e)
        want = np.array([float(e.coeff(c).subs(sub)) for c in dl])
        got = taylor.op_row(op, xb, idx)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_vector_bc_rows_vs_sympy(bc):
    d, M = 2, 4
    syms = sympy.symbols("x0:%d" % d)
    idx = taylor.multi_indices(d, M)
    T = len(idx)
    cs = [sympy.symbols("a%d_0:%d" % (a, T)) for a in range(d)]
    v = [sum(c * sympy.prod([s ** k / sympy.factorial(k) for s, k in zip(syms, kk)])
             for c, kk in zip(cs[a], idx)) for a in range(d)]
    div = sum(sympy.diff(v[a], syms[a]) for a in range(d))
    lap = lambda f: sum(sympy.diff(f, s, 2) for s in syms)
    nrm = np.array([0.6, 0.8])
    xb = np.array([0.4, -1.3])
    exprs = []
    if bc == "free":
        f = div
        k = 0
        while 2 * k + 1 <= M:
            exprs.append(f)
            f = lap(f)
            k += 1
    else:
        exprs.append(sum(float(n) * vv for n, vv in zip(nrm, v)))
        f = div
        k = 0
        while 2 * k + 2 <= M:
            exprs.append(sum(float(n) * sympy.diff(f, s) for n, s in zip(nrm, syms)))
            f = lap(f)
            k += 1
        f = sympy.diff(v[1], syms[0]) - sympy.diff(v[0], syms[1])      # 2D curl
        k = 0
        while 2 * k + 1 <= M:
            exprs.append(f)
            f = lap(f)
            k += 1
    rows = taylor.bc_rows_vector(bc, d, M, nrm)
    assert len(rows) == len(exprs)
    sub = dict(zip(syms, xb))
    for e, row in zip(exprs, rows):
        e = sympy.expand(e)
        want = np.array([float(e.coeff(c).subs(sub)) for a in range(d) for c in cs[a]])
        got = np.concatenate([taylor.op_row(op, xb, idx) for op in row])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_vectorised_rows_match_definition():
    rng = np.random.default_rng(3)
    for d, M in [(2, 8), (3, 8)]:
        idx = taylor.multi_indices(d, M)
        xi = rng.normal(size=d) * 3
        np.testing.assert_allclose(taylor.basis_row(xi, idx), taylor.basis_row_scalar(xi, idx),
                                   rtol=1e-13)
        for op in taylor.bc_rows_scalar("rigid", d, M, rng.normal(size=d)):
            b = taylor.op_row_scalar(op, xi, idx)
            np.testing.assert_allclose(taylor.op_row(op, xi, idx), b, rtol=1e-12,
                                       atol=1e-12 * np.abs(b).max())
