"""Time stepping, sources, receivers and the discrete adjoint (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Second-order form (2nd-order application section):
    p^{n+1} = 2 p^n - p^{n-1} + dt^2 c^2 (L p^n) + dt^2 f^n
with p^0 = p^{-1} = 0, exterior nodes held at zero and zero values beyond the
array (zero Dirichlet edges, Examples section).

First-order form, paper's signs (1st-order section), backward-staggered:
    v_a^{n+1/2} = v_a^{n-1/2} + dt (1/rho) (G_a p^n)
    p^{n+1}     = p^n + dt rho c^2 (D v^{n+1/2}) + dt f^n

Readings (the paper is silent): the source is w(t) delta(x - x_s) with the
delta spread multilinearly to the 2^d nodes of its cell (1/h^d scaling),
exterior nodes dropped; wavelet sample n is used in the step that produces
p^{n+1}; receivers record trace[r][n] = multilinear interpolation of p^{n+1};
1/rho at a staggered node is the mean of 1/rho at its two neighbours.

Absorbing layer (the paper's examples use zero Dirichlet edges and note that a
damping boundary of choice combines with the method, Examples section):
p_tt + eta p_t = c^2 lap p + f with eta = eta_max min(1, d^2 / W^2), d the
node distance into a layer of W nodes along the side edges and the bottom,
centred in time:
    (p^{n+1} - 2 p^n + p^{n-1}) + a (p^{n+1} - p^{n-1}) = dt^2 c^2 L p^n + dt^2 f^n,
    a = eta dt / 2.

Adjoint: the exact transpose of the discrete leapfrog map (Lagrangian of the
recursion above with J = 1/2 sum |trace - d|^2):
    mu^m = 2 mu^{m+1} - mu^{m+2} + L^T (K mu^{m+1}) + R^T res^{m-1},  m = nt..1
    dJ/dc(x) = sum_n mu^{n+1}(x) 2 c(x) dt^2 (L p^n)(x)
    dJ/dw[n] = (S mu^{n+1}) dt^2 / h^d
with K = dt^2 c^2 on interior nodes and 0 elsewhere.  With the absorbing layer,
with B = 1 / (1 + a) and C = (1 - a) / (1 + a) (diagonal):
    mu^m = (2 I + K L)^T (B mu^{m+1}) - C mu^{m+2} + R^T res^{m-1}
    dJ/dc(x) = sum_n mu^{n+1}(x) B(x) 2 c(x) dt^2 (L p^n)(x)
    dJ/dw[n] = (B S mu^{n+1}) dt^2 / h^d
"""
import math

import numpy as np
import scipy.sparse as sp


def multilinear_matrix(points_m, h, shape, mask):
    """Rows: multilinear interpolation weights of each point (metres) to the
    2^d nodes of its cell; nodes outside the array or exterior are dropped."""
    d = len(shape)
    lshape = tuple(reversed(shape))
    N = int(np.prod(shape))
    rows, cols, vals = [], [], []
    st = [1] * d
    for i in range(d - 2, -1, -1):
        st[i] = st[i + 1] * shape[i + 1]
    lst = list(reversed(st))                 # stride of logical axis a
    for r, pt in enumerate(np.asarray(points_m, dtype=np.float64)):
        xi = pt / h
        base = [int(math.floor(x)) for x in xi]
        fr = [x - b for x, b in zip(xi, base)]
        for corner in range(1 << d):
            w = 1.0
            node = []
            for a in range(d):
                bit = (corner >> a) & 1
                node.append(base[a] + bit)
                w *= fr[a] if bit else (1.0 - fr[a])
            if w == 0.0:
                continue
            if not all(0 <= node[a] < lshape[a] for a in range(d)):
                continue
            flat = sum(node[a] * lst[a] for a in range(d))
            if not mask.reshape(-1)[flat]:
                continue
            rows.append(r)
            cols.append(flat)
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(points_m), N))


def damping_coefficient(shape, width, eta_max, dt):
    """a = eta dt / 2 per node (flattened, array order): eta = eta_max min(1,
    d^2 / W^2), d^2 the summed squares of the node's distances into the layer
    from the first and last index of each horizontal axis and from the last
    index of the depth axis (axis 0)."""
    d2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        i = np.arange(n, dtype=np.float64)
        if ax == 0:
            dist = np.maximum(i - (n - 1 - width), 0.0)
        else:
            dist = np.maximum(np.maximum(width - i, i - (n - 1 - width)), 0.0)
        sh = [1] * len(shape)
        sh[ax] = n
        d2 = d2 + (dist ** 2).reshape(sh)
    return (0.5 * eta_max * dt * np.minimum(d2 / float(width) ** 2, 1.0)).reshape(-1)


def leapfrog_coefficient(vel, dt, mask):
    """K = dt^2 c^2 on interior nodes, 0 on exterior nodes."""
    return np.where(mask, (dt * np.asarray(vel, dtype=np.float64)) ** 2, 0.0).reshape(-1)


def forward_leapfrog(L, K, S, wavelet, R, nt, keep_history=False, a=None):
    """Second-order leapfrog.  S: source vector (dt^2/h^d times multilinear
    weights, summed over sources); a: absorbing-layer coefficient per node or
    None.  Returns traces [nrec][nt] (and p^0..p^nt)."""
    N = L.shape[0]
    p = np.zeros(N)
    pm = np.zeros(N)
    traces = np.zeros((R.shape[0], nt))
    hist = [p.copy()] if keep_history else None
    for n in range(nt):
        if a is None:
            pn = 2.0 * p - pm + K * (L @ p) + S * wavelet[n]
        else:
            pn = (2.0 * p - (1.0 - a) * pm + K * (L @ p) + S * wavelet[n]) / (1.0 + a)
        traces[:, n] = R @ pn
        pm, p = p, pn
        if keep_history:
            hist.append(p.copy())
    return (traces, hist) if keep_history else traces


def adjoint_leapfrog(L, K, vel_flat, dt, R, residual, S, hist, a=None):
    """Exact discrete adjoint.  hist = [p^0, .., p^nt]; a as in forward_leapfrog.
    Returns (dJ/dc over nodes, dJ/dw over steps)."""
    N = L.shape[0]
    nt = residual.shape[1]
    LT = L.T.tocsr()
    B = np.ones(N) if a is None else 1.0 / (1.0 + a)
    C = np.ones(N) if a is None else (1.0 - a) / (1.0 + a)
    mu1 = np.zeros(N)        # mu^{m+1}
    mu2 = np.zeros(N)        # mu^{m+2}
    grad = np.zeros(N)
    gw = np.zeros(nt)
    c2dt2 = np.where(K != 0.0, 2.0 * vel_flat * dt * dt, 0.0)
    for m in range(nt, 0, -1):
        bmu = B * mu1
        mu = 2.0 * bmu - C * mu2 + LT @ (K * bmu) + R.T @ residual[:, m - 1]
        n = m - 1
        grad += mu * B * c2dt2 * (L @ hist[n])
        gw[n] = S @ (B * mu)
        mu2, mu1 = mu1, mu
    return grad, gw


def forward_staggered(G, D, bv, kp, S, wavelet, R, nt):
    """First-order staggered scheme.  bv[a] = dt/rho at v_a nodes (0 outside),
    kp = dt rho c^2 at p nodes (0 outside), S = dt/h^d times source weights."""
    N = kp.shape[0]
    d = len(G)
    p = np.zeros(N)
    v = [np.zeros(N) for _ in range(d)]
    traces = np.zeros((R.shape[0], nt))
    for n in range(nt):
        for a in range(d):
            v[a] = v[a] + bv[a] * (G[a] @ p)
        p = p + kp * (D @ np.concatenate(v)) + S * wavelet[n]
        traces[:, n] = R @ p
    return traces


def staggered_coefficients(geom, vel, rho, dt):
    """bv[a] = dt * mean(1/rho) at v_a nodes (interior v_a only); kp = dt rho c^2."""
    rho = np.asarray(rho, dtype=np.float64)
    vel = np.asarray(vel, dtype=np.float64)
    kp = np.where(geom.mask, dt * rho * vel * vel, 0.0).reshape(-1)
    bv = []
    inv = 1.0 / rho
    for a in range(geom.d):
        ax = geom.d - 1 - a
        n = inv.shape[ax]
        nb = inv.copy()
        sd = [slice(None)] * inv.ndim
        ss = [slice(None)] * inv.ndim
        sd[ax] = slice(0, n - 1)
        ss[ax] = slice(1, n)
        nb[tuple(sd)] = inv[tuple(ss)]
        bv.append(np.where(geom.vmask(a), dt * 0.5 * (inv + nb), 0.0).reshape(-1))
    return bv, kp
