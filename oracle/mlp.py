"""Learned modified-stencil predictor (oracle): features, the network, its
training step and the exactness acceptance test.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The paper constructs every modified stencil by a least-squares fit; it has no
learned component.  What is restated here is the plain definition of a small
multilayer perceptron that predicts a modified Laplacian row from the signed
distance around the row's node, of its mean-squared-error gradient, of one Adam
step, and of the test that decides whether a predicted row is kept.  That test
is the exactness property the paper's construction guarantees (section
"Reconciliation with the Interior Numerical Discretization"): for every
polynomial of the extrapolation basis that satisfies each imposed boundary
condition at each boundary point of the support, the modified row applied to
the polynomial's values at the interior support nodes reproduces the standard
stencil applied to the polynomial on the full lattice.  In matrix form, with
A = [A_I; A_B] the fit matrix (interior rows first, boundary-condition rows
after) and u = sum_e w_e a(x_e - x0), a correction c is exact iff
N^T (A_I^T c - u) = 0 for N a basis of the null space of A_B.  The plain fit's
c = ((A^+)^T u)[interior rows] satisfies it because A^T (A^+)^T u = u.

Reduced-precision points (where the library rounds to bfloat16) are emulated
with ``bf16`` so that the two sides round at the same places; everything else
is FP64.
"""
import numpy as np

from . import taylor
from .stencils import _support_offsets
from .geometry import logical_shape


# ---------------------------------------------------------------------------
# bfloat16 rounding (round to nearest, ties to even) on float32 values
# ---------------------------------------------------------------------------
def bf16(x):
    """Round to the nearest bfloat16 (ties to even), as float64.  The input is
    first rounded to float32 (the library rounds float32 values)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


# ---------------------------------------------------------------------------
# layout of inputs and outputs
# ---------------------------------------------------------------------------
def ball(d, r):
    """Lattice offsets o with |o|_2 <= r, in support order (distance, then
    array order), as tuples (x, y[, z])."""
    return list(_support_offsets(tuple([0.0] * d), float(r)))


def feature_vector(sdf, h, node, bc, M, in_off):
    """SDF/h at node + o for o in ``in_off`` (nearest in-array node where the
    offset leaves the array), then [free, rigid, M / 8]."""
    s = np.asarray(sdf, dtype=np.float64)
    ls = logical_shape(s)
    d = len(ls)
    out = []
    for o in in_off:
        q = [min(max(node[a] + o[a], 0), ls[a] - 1) for a in range(d)]
        out.append(s[tuple(reversed(q))] / h)
    out += [1.0 if bc == "free" else 0.0, 1.0 if bc == "rigid" else 0.0, M / 8.0]
    return np.array(out)


def target_vector(wts, out_off):
    """Correction weights of one row on the output footprint, or None when the
    row has entries outside it."""
    index = {tuple(o): i for i, o in enumerate(out_off)}
    t = np.zeros(len(out_off))
    for off, w in wts.items():
        i = index.get(tuple(off))
        if i is None:
            return None
        t[i] += w
    return t


# ---------------------------------------------------------------------------
# the network: Linear -> ReLU (hidden layers) -> Linear
# ---------------------------------------------------------------------------
def layer_sizes(n_in, n_hidden, n_layers, n_out):
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unflatten(params, sizes):
    """Flat parameter vector -> [(W [n_out][n_in], b [n_out])] in layer order."""
    out, p = [], 0
    for no, ni in sizes:
        W = params[p:p + no * ni].reshape(no, ni)
        p += no * ni
        b = params[p:p + no]
        p += no
        out.append((W, b))
    assert p == params.size
    return out


def forward(params, sizes, X, emulate=True):
    """Returns (Y, acts): acts[l] is the input of layer l as the library keeps
    it (bfloat16 when ``emulate``)."""
    q = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unflatten(np.asarray(params, dtype=np.float64), sizes)
    h = q(X)
    acts = []
    for l, (W, b) in enumerate(layers):
        acts.append(h)
        z = h @ q(W).T + b
        if l + 1 < len(layers):
            h = q(np.maximum(z, 0.0))
        else:
            h = z
    return h, acts


def mse(Y, T):
    """Mean over rows and outputs of (Y - T)^2."""
    return float(np.mean((Y - T) ** 2))


def backward(params, sizes, X, T, emulate=True):
    """Gradient of ``mse`` w.r.t. the flat parameter vector (same layout).
    With ``emulate`` the output gradient and the hidden-layer gradients are
    rounded to bfloat16 before they enter a product, as in the library."""
    q = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unflatten(np.asarray(params, dtype=np.float64), sizes)
    Y, acts = forward(params, sizes, X, emulate)
    n, k = T.shape
    g = 2.0 * (Y - T) / (n * k)               # d loss / d Y
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gq = q(g)
        dW = gq.T @ acts[l]
        db = g.sum(axis=0)
        grads[l] = (dW, db)
        if l > 0:
            g = (gq @ q(W)) * (acts[l] > 0.0)
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return flat, mse(Y, T)


def adam(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1) at step number t >= 1.
    Returns (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------------------------------------------------------------------
# exactness of a predicted row
# ---------------------------------------------------------------------------
def bc_null_space(A, n_int, tol=1e-10):
    """Orthonormal basis of the null space of the BC block A[n_int:] (SVD,
    singular values <= tol * largest count as zero)."""
    C = A[n_int:]
    T = A.shape[1]
    if C.shape[0] == 0:
        return np.eye(T)
    _, s, Vt = np.linalg.svd(C)
    rank = int((s > tol * s[0]).sum()) if s.size and s[0] > 0 else 0
    return Vt[rank:].T


def exactness_residual(A, n_int, u, c, tol=1e-10):
    """|N^T (A_I^T c - u)| / |u|: zero for an exact row (see module doc)."""
    N = bc_null_space(A, n_int, tol)
    r = N.T @ (A[:n_int].T @ np.asarray(c, dtype=np.float64) - u)
    nu = float(np.linalg.norm(u))
    return float(np.linalg.norm(r)) / (nu if nu > 0 else 1.0)


def prediction_on_support(pred, out_off, support_offsets):
    """Predicted correction at each interior support node (None if a node lies
    outside the output footprint)."""
    index = {tuple(o): i for i, o in enumerate(out_off)}
    out = []
    for o in support_offsets:
        i = index.get(tuple(o))
        if i is None:
            return None
        out.append(pred[i])
    return np.array(out)
