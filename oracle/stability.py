"""Stability of the explicit schemes with the modified operators (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The paper's time stepping (2nd-order application section) is the leapfrog
recursion p^{n+1} = 2 p^n - p^{n-1} + A p^n with A = diag(K) L_mod and
K = dt^2 c^2 (0 at exterior nodes).  One step maps (p^n, p^{n-1}) to
(p^{n+1}, p^n) by the companion matrix [[2I + A, -I], [I, 0]].  For an
eigenvalue mu of A the companion matrix has the two eigenvalues lambda with
    lambda^2 - (2 + mu) lambda + 1 = 0,
and |lambda| <= 1 for both iff mu is real and -4 <= mu <= 0.  The modified
operator is not symmetric, so mu can be complex or positive near the surface:
the scheme then grows like rho^n with rho = max |lambda| > 1.  The paper gives
no stability analysis; this module measures rho two ways:

* ``leapfrog_mu`` / ``growth_from_mu``: the eigenvalues of A (dense, small
  problems) and the largest |lambda| they give;
* ``leapfrog_growth``: power iteration on the companion map (source-free time
  stepping from a seeded random state, renormalised), the same estimate the
  library's stability check makes on the GPU.

``staggered_growth`` does the power iteration for the first-order staggered
scheme (1st-order section): (v, p) -> (v + bv G p, p + kp D v_new).
"""
import numpy as np


def leapfrog_matrix(L, K):
    """A = diag(K) L restricted to the interior nodes (K != 0): dense array and
    the indices it keeps."""
    keep = np.flatnonzero(np.asarray(K) != 0.0)
    A = (L.tocsr()[keep][:, keep]).toarray() * np.asarray(K)[keep][:, None]
    return A, keep


def leapfrog_mu(L, K):
    """Eigenvalues mu of diag(K) L on the interior nodes (dense; small problems)."""
    A, _ = leapfrog_matrix(L, K)
    return np.linalg.eigvals(A)


def lambda_of_mu(mu):
    """Both roots of lambda^2 - (2 + mu) lambda + 1 = 0 for each mu (complex)."""
    mu = np.asarray(mu, dtype=np.complex128)
    b = 2.0 + mu
    s = np.sqrt(b * b - 4.0)
    return (b + s) / 2.0, (b - s) / 2.0


def growth_from_mu(mu):
    """Per-step growth factor rho = max |lambda| over the spectrum of A."""
    l1, l2 = lambda_of_mu(mu)
    return float(max(np.abs(l1).max(), np.abs(l2).max()))


def leapfrog_growth(L, K, nsteps=2000, seed=0, renorm=50, a=None):
    """Power iteration on the leapfrog companion map.  Starts from a seeded
    random p^0 = p^{-1} on interior nodes, steps source-free, renormalises every
    `renorm` steps, and returns (rho estimate, log-norm history).  For a
    stable scheme the estimate tends to 1; an unstable mode with |lambda| = rho
    dominates once rho^n outgrows the initial transient.  a: absorbing-layer
    coefficient per node (``propagate.damping_coefficient``) or None."""
    K = np.asarray(K, dtype=np.float64)
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(K.shape[0]) * (K != 0.0)
    pm = p.copy()
    logn = np.zeros(nsteps + 1)
    scale = 0.0
    logn[0] = np.log(np.sqrt(np.dot(p, p) + np.dot(pm, pm)))
    for n in range(1, nsteps + 1):
        if a is None:
            pn = 2.0 * p - pm + K * (L @ p)
        else:
            pn = (2.0 * p - (1.0 - a) * pm + K * (L @ p)) / (1.0 + a)
        pm, p = p, pn
        nrm = np.sqrt(np.dot(p, p) + np.dot(pm, pm))
        logn[n] = scale + np.log(nrm)
        if n % renorm == 0:
            scale += np.log(nrm)
            p /= nrm
            pm /= nrm
    return float(np.exp((logn[nsteps] - logn[nsteps // 2]) / (nsteps - nsteps // 2))), logn


def staggered_growth(G, D, bv, kp, nsteps=2000, seed=0, renorm=50):
    """Power iteration on the staggered map (v, p) -> (v', p') with
    v'_a = v_a + bv_a (G_a p), p' = p + kp (D v').  Returns (rho estimate, log-norm history)."""
    rng = np.random.default_rng(seed)
    d = len(G)
    kp = np.asarray(kp, dtype=np.float64)
    p = rng.standard_normal(kp.shape[0]) * (kp != 0.0)
    v = [rng.standard_normal(kp.shape[0]) * (np.asarray(bv[a]) != 0.0) for a in range(d)]
    logn = np.zeros(nsteps + 1)
    scale = 0.0

    def norm():
        return np.sqrt(np.dot(p, p) + sum(np.dot(x, x) for x in v))

    logn[0] = np.log(norm())
    for n in range(1, nsteps + 1):
        for a in range(d):
            v[a] = v[a] + bv[a] * (G[a] @ p)
        p = p + kp * (D @ np.concatenate(v))
        nrm = norm()
        logn[n] = scale + np.log(nrm)
        if n % renorm == 0:
            scale += np.log(nrm)
            p = p / nrm
            v = [x / nrm for x in v]
    return float(np.exp((logn[nsteps] - logn[nsteps // 2]) / (nsteps - nsteps // 2))), logn
