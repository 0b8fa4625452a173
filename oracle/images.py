"""Method-of-images analytic solutions for a flat surface (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

For p_tt = c^2 lap p + w(t) delta(x - x_s) in free space the solution is the
convolution of w with the Green's function
    2D: G(r, t) = H(t - r/c) / (2 pi c sqrt(c^2 t^2 - r^2))
    3D: G(r, t) = delta(t - r/c) / (4 pi c^2 r)
A flat free surface (p = 0) reflects with coefficient -1 and a rigid surface
(zero normal particle velocity, dp/dn = 0) with +1, so in the half space the
solution is the direct field minus (free) or plus (rigid) the field of the
mirrored source (reflection polarity paragraph of the 2nd-order section and
the rigid-surface example).

2D quadrature: p(r, t) = int_{r/c}^{t} w(t - tau) G(r, tau) dtau; with
tau = r/c + s^2 the inverse square-root singularity cancels:
    p = int_0^{sqrt(t - r/c)} w(t - r/c - s^2) / (pi c sqrt(c (2 r + c s^2))) ds
evaluated by composite Gauss-Legendre quadrature.
"""
import math

import numpy as np


def _gauss_legendre(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def free_space_2d(w_of_t, r, t, c, panels=64, order=16):
    """Direct 2D field at distances r (array) and times t (array, same shape)."""
    r = np.asarray(r, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros(np.broadcast(r, t).shape)
    rr, tt = np.broadcast_arrays(r, t)
    smax = np.sqrt(np.clip(tt - rr / c, 0.0, None))
    xg, wg = _gauss_legendre(order)
    for p in range(panels):
        a = smax * p / panels
        b = smax * (p + 1) / panels
        half = 0.5 * (b - a)
        mid = 0.5 * (a + b)
        for xk, wk in zip(xg, wg):
            s = mid + half * xk
            f = w_of_t(tt - rr / c - s * s) / (math.pi * c * np.sqrt(c * (2.0 * rr + c * s * s)))
            out += wk * half * f
    return out


def free_space_3d(w_of_t, r, t, c):
    r = np.asarray(r, dtype=np.float64)
    return w_of_t(np.asarray(t) - r / c) / (4.0 * math.pi * c * c * r)


def flat_surface_traces(w_of_t, src, rec, times, c, z0, bc, ndim):
    """Traces [nrec][ntimes] for a flat surface z = z0 (domain z > z0).

    src, rec: coordinates in metres, logical order (x, [y,] z)."""
    src = np.asarray(src, dtype=np.float64)
    rec = np.asarray(rec, dtype=np.float64)
    img = src.copy()
    img[-1] = 2.0 * z0 - src[-1]
    sign = -1.0 if bc == "free" else 1.0
    r1 = np.linalg.norm(rec - src[None, :], axis=1)[:, None]
    r2 = np.linalg.norm(rec - img[None, :], axis=1)[:, None]
    T = np.asarray(times, dtype=np.float64)[None, :]
    if ndim == 2:
        return free_space_2d(w_of_t, r1, T, c) + sign * free_space_2d(w_of_t, r2, T, c)
    return free_space_3d(w_of_t, r1, T, c) + sign * free_space_3d(w_of_t, r2, T, c)


def ricker_fn(f0, t0=None):
    if t0 is None:
        t0 = 1.5 / f0

    def w(t):
        a = (math.pi * f0 * (np.asarray(t) - t0)) ** 2
        return (1.0 - 2.0 * a) * np.exp(-a)
    return w


def ricker_derivative_fn(f0, t0=None, shift=0.0):
    """d/dt of the Ricker wavelet, delayed by `shift`."""
    if t0 is None:
        t0 = 1.5 / f0

    def dw(t):
        tau = np.asarray(t) - t0 - shift
        a = (math.pi * f0) ** 2
        return (-6.0 * a * tau + 4.0 * a * a * tau ** 3) * np.exp(-a * tau * tau)
    return dw


def mirror_point(src, point_on_plane, normal):
    """Mirror image of `src` across the plane through `point_on_plane` with
    unit `normal`."""
    src = np.asarray(src, dtype=np.float64)
    n = np.asarray(normal, dtype=np.float64)
    dist = np.dot(src - np.asarray(point_on_plane, dtype=np.float64), n)
    return src - 2.0 * dist * n


def plane_traces(w_of_t, src, rec, times, c, point_on_plane, normal, bc, ndim):
    """Traces for an arbitrary plane (image across the plane)."""
    img = mirror_point(src, point_on_plane, normal)
    sign = -1.0 if bc == "free" else 1.0
    r1 = np.linalg.norm(np.asarray(rec) - np.asarray(src)[None, :], axis=1)[:, None]
    r2 = np.linalg.norm(np.asarray(rec) - img[None, :], axis=1)[:, None]
    T = np.asarray(times, dtype=np.float64)[None, :]
    f = free_space_2d if ndim == 2 else free_space_3d
    return f(w_of_t, r1, T, c) + sign * f(w_of_t, r2, T, c)
