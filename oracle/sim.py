"""Whole-simulation helpers built from the oracle pieces (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.
"""
import numpy as np

from . import operators, propagate, stencils


class Leapfrog:
    """Second-order form on one geometry: modified Laplacian, K, S, R."""

    def __init__(self, sdf, vel, h, M, bc, dt, src, rec, opts=None, damp=None):
        """damp: None or (width in nodes, eta_max in 1/s) of the absorbing layer."""
        self.opts = opts or stencils.Opts(M)
        self.geom = stencils.Geometry(sdf, h, M)
        self.L, self.rows = operators.laplacian_matrix(self.geom, bc, self.opts)
        self.a = (propagate.damping_coefficient(self.geom.sdf.shape, damp[0], damp[1], dt) * self.geom.mask.ravel()
                  if damp is not None else None)
        self.vel = np.asarray(vel, dtype=np.float64)
        self.dt = dt
        self.h = h
        shape = self.geom.sdf.shape
        d = self.geom.d
        self.K = propagate.leapfrog_coefficient(self.vel, dt, self.geom.mask)
        self.S = (propagate.multilinear_matrix(src, h, shape, self.geom.mask).toarray().sum(0)
                  * dt * dt / h ** d)
        self.R = propagate.multilinear_matrix(rec, h, shape, self.geom.mask)

    def forward(self, wavelet, nt, keep_history=False):
        return propagate.forward_leapfrog(self.L, self.K, self.S, wavelet, self.R, nt, keep_history, self.a)

    def with_velocity(self, vel):
        out = object.__new__(Leapfrog)
        out.__dict__.update(self.__dict__)
        out.vel = np.asarray(vel, dtype=np.float64)
        out.K = propagate.leapfrog_coefficient(out.vel, self.dt, self.geom.mask)
        return out

    def adjoint(self, residual, hist):
        return propagate.adjoint_leapfrog(self.L, self.K, self.vel.reshape(-1), self.dt, self.R,
                                          residual, self.S, hist, self.a)


class Staggered:
    """First-order staggered form on one geometry."""

    def __init__(self, sdf, vel, rho, h, M, bc, dt, src, rec, opts=None):
        self.opts = opts or stencils.Opts(M)
        self.geom = stencils.Geometry(sdf, h, M)
        self.G, self.D, self.grad_rows, self.div_rows = operators.staggered_matrices(
            self.geom, bc, self.opts)
        self.bv, self.kp = propagate.staggered_coefficients(self.geom, vel, rho, dt)
        shape = self.geom.sdf.shape
        d = self.geom.d
        self.S = (propagate.multilinear_matrix(src, h, shape, self.geom.mask).toarray().sum(0)
                  * dt / h ** d)
        self.R = propagate.multilinear_matrix(rec, h, shape, self.geom.mask)

    def forward(self, wavelet, nt):
        return propagate.forward_staggered(self.G, self.D, self.bv, self.kp, self.S, wavelet,
                                           self.R, nt)
