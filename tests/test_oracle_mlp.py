"""Pins of the oracle's learned-stencil pieces (no GPU): bfloat16 rounding,
the network gradient, the Adam step, the feature layout and the exactness
acceptance test."""
import math

import numpy as np
import pytest

from oracle import mlp, stencils, taylor
from paper_2309_03600_gb300 import inputs


def circle_sdf(nx, nz, cx, cz, R):
    x = np.arange(nx)[None, :] - cx
    z = np.arange(nz)[:, None] - cz
    return np.sqrt(x * x + z * z) - R


# ---------------------------------------------------------------------------
# bfloat16
# ---------------------------------------------------------------------------
def test_bf16_known_values():
    # bfloat16 keeps 8 significant bits: pi -> 0x4049 = 3.140625, 1/3 -> 0x3EAB
    assert mlp.bf16(math.pi) == 3.140625
    assert mlp.bf16(1.0 / 3.0) == 0.333984375
    # halfway cases round to the even neighbour
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3.0 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(-(1.0 + 3.0 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    # representable values are fixed points; with 8 significant bits the
    # relative rounding error is at most half a unit in the last place, 2^-8
    x = np.random.default_rng(0).normal(size=10000) * 10.0 ** np.random.default_rng(1).integers(-20, 20, 10000)
    r = mlp.bf16(x)
    np.testing.assert_array_equal(mlp.bf16(r), r)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -8


# ---------------------------------------------------------------------------
# network gradient and Adam
# ---------------------------------------------------------------------------
def _tiny(seed=0):
    sizes = mlp.layer_sizes(5, 4, 2, 3)
    n = sum(a * b + a for a, b in sizes)
    rng = np.random.default_rng(seed)
    return sizes, rng.normal(size=n) * 0.7, rng.normal(size=(6, 5)), rng.normal(size=(6, 3))


def test_gradient_matches_finite_differences():
    sizes, p, X, T = _tiny()
    g, _ = mlp.backward(p, sizes, X, T, emulate=False)
    eps = 1e-6
    num = np.zeros_like(p)
    for i in range(p.size):
        d = np.zeros_like(p)
        d[i] = eps
        fp = mlp.mse(mlp.forward(p + d, sizes, X, False)[0], T)
        fm = mlp.mse(mlp.forward(p - d, sizes, X, False)[0], T)
        num[i] = (fp - fm) / (2 * eps)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_emulated_gradient_equals_exact_on_representable_values():
    """When every weight, input and intermediate is already a bfloat16 value the
    emulation changes nothing except the rounding of the back-propagated
    signal; with a zero-residual target at the output only the output layer
    gradient is affected and it must vanish."""
    sizes, p, X, _ = _tiny(3)
    Y, _ = mlp.forward(p, sizes, X, emulate=True)
    g, loss = mlp.backward(p, sizes, X, Y, emulate=True)
    assert loss == 0.0
    assert np.all(g == 0.0)


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(4)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = mlp.adam(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(new, p - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    p = np.array([3.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for t in range(1, 3001):
        p, m, v = mlp.adam(p, 2.0 * p, m, v, t, lr=1e-2)
    assert np.max(np.abs(p)) < 1e-2


# ---------------------------------------------------------------------------
# layout
# ---------------------------------------------------------------------------
def test_ball_counts():
    # lattice points in balls: 2D r=2.5 -> 21, r=4 -> 49; 3D r=2.5 -> 81, r=4 -> 257
    assert len(mlp.ball(2, 2.5)) == 21
    assert len(mlp.ball(2, 4.0)) == 49
    assert len(mlp.ball(3, 2.5)) == 81
    assert len(mlp.ball(3, 4.0)) == 257
    b = mlp.ball(3, 4.0)
    assert b[0] == (0, 0, 0)
    assert all(sum(x * x for x in b[i]) <= sum(x * x for x in b[i + 1]) for i in range(len(b) - 1))


def test_features_of_flat_surface_are_linear_in_depth():
    h, z0 = 10.0, 83.0
    sdf = inputs.flat_surface_sdf((30, 20), h, z0)     # s = z - z0 (domain below)
    off = mlp.ball(2, 4.0)
    node = (12, 11)
    f = mlp.feature_vector(sdf, h, node, "rigid", 8, off)
    expect = [((node[1] + o[1]) * h - z0) / h for o in off]
    np.testing.assert_allclose(f[:len(off)], expect, atol=1e-12)
    assert list(f[len(off):]) == [0.0, 1.0, 1.0]
    # offsets leaving the array take the nearest in-array node
    f = mlp.feature_vector(sdf, h, (0, 0), "free", 4, off)
    i = off.index((-3, -2))
    assert f[i] == (0.0 - z0) / h


# ---------------------------------------------------------------------------
# exactness acceptance test
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def circle_rows():
    sdf = circle_sdf(44, 44, 21.3, 22.6, 11.7)
    geom = stencils.Geometry(sdf, 1.0, 8)
    nodes = stencils.laplacian_ib_nodes(geom.mask, 8)[::5]
    out = {}
    for bc in ("free", "rigid"):
        out[bc] = stencils.laplacian_rows(geom, bc, stencils.Opts(8), nodes)
    return out


@pytest.mark.parametrize("bc", ["free", "rigid"])
def test_plain_rows_pass_and_perturbed_rows_fail(circle_rows, bc):
    rng = np.random.default_rng(5)
    n_checked = 0
    for node, (wts, info) in circle_rows[bc].items():
        A, u, y, ni = info["A"], info["u"], info["y"], info["n_int"]
        assert mlp.exactness_residual(A, ni, u, y[:ni]) < 1e-9
        N = mlp.bc_null_space(A, ni)
        if N.shape[1] == 0:
            continue
        e = rng.normal(size=ni) * 1e-2 * np.abs(y[:ni]).max()
        rho = mlp.exactness_residual(A, ni, u, y[:ni] + e)
        # the residual of a perturbation is that of the perturbation alone
        expect = np.linalg.norm(N.T @ (A[:ni].T @ e)) / np.linalg.norm(u)
        assert abs(rho - expect) <= 1e-9 + 1e-9 * expect
        assert rho > 1e-6
        n_checked += 1
    assert n_checked > 5


def test_residual_is_polynomial_exactness(circle_rows):
    """Brute force: for random BC-satisfying polynomials q = a . delta, the
    residual of a perturbed row bounds |sum_j c_j q(X_j) - sum_e w_e q(x_e)|."""
    rng = np.random.default_rng(6)
    w2 = [float(x) for x in taylor.central_second(8)]
    for node, (wts, info) in list(circle_rows["free"].items())[:10]:
        A, u, y, ni = info["A"], info["u"], info["y"], info["n_int"]
        N = mlp.bc_null_space(A, ni)
        if N.shape[1] == 0:
            continue
        idx = taylor.multi_indices(2, info["order"])
        c = y[:ni] + rng.normal(size=ni) * 1e-3
        rho = mlp.exactness_residual(A, ni, u, c)
        sup = [np.array(j, dtype=float) for _, j in info["support"]]
        x0 = np.array(node, dtype=float)
        for _ in range(5):
            alpha = N @ rng.normal(size=N.shape[1])
            alpha /= np.linalg.norm(alpha)
            lhs = sum(cj * float(taylor.basis_row(xj - x0, idx) @ alpha) for cj, xj in zip(c, sup))
            # u . alpha is the standard stencil applied to q at the exterior points
            rhs = float(u @ alpha)
            assert abs(lhs - rhs) <= rho * np.linalg.norm(u) * (1 + 1e-9) + 1e-12


def test_prediction_on_support_and_targets(circle_rows):
    off = mlp.ball(2, 2.5)
    for node, (wts, info) in list(circle_rows["free"].items())[:20]:
        t = mlp.target_vector(wts, off)
        if info["radius"] > 2.5:
            continue
        assert t is not None
        sup_off = [tuple(jj - nn for jj, nn in zip(j, node)) for _, j in info["support"]]
        c = mlp.prediction_on_support(t, off, sup_off)
        np.testing.assert_allclose(c, info["y"][:info["n_int"]], atol=1e-15)
