"""Seeded synthetic inputs: topography SDFs, velocity models, wavelets, geometry.

This module holds no arithmetic of the immersed-boundary method itself.  It
only builds inputs (signed-distance fields of synthetic surfaces, velocity
models, Ricker wavelets, source/receiver coordinates) and is shared by the
tests, the oracle checks and the benchmark.

Conventions: arrays are stored slowest axis first (2D ``[nz][nx]``, 3D
``[nz][ny][nx]``), node (i_x, .., i_z) sits at (i_x h, .., i_z h), z is depth
(positive down) and the SDF is positive in the physical domain (below the
surface).  Coordinates are in metres, logical order (x, [y,] z).
"""
import math

import numpy as np
import torch


# ---------------------------------------------------------------------------
# wavelets and time stepping
# ---------------------------------------------------------------------------
def ricker(f0, dt, nt, t0=None, dtype=np.float64):
    """Ricker wavelet (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0,
    sampled at t = n dt, n = 0..nt-1; t0 defaults to 1.5 / f0."""
    if t0 is None:
        t0 = 1.5 / f0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(dtype)


def dt_from_courant(courant, h, vmax):
    """dt = C h / c_max."""
    return courant * h / vmax


# ---------------------------------------------------------------------------
# signed distance fields
# ---------------------------------------------------------------------------
def _grid(shape_xyz, h, dtype=torch.float64, device="cpu"):
    axes = [torch.arange(n, dtype=dtype, device=device) * h for n in shape_xyz]
    return axes


def flat_surface_sdf(shape_xyz, h, z0):
    """SDF of the plane z = z0 (domain below): s = z - z0."""
    d = len(shape_xyz)
    z = np.arange(shape_xyz[-1], dtype=np.float64) * h - z0
    shp = tuple(reversed(shape_xyz))
    view = [1] * d
    view[0] = shape_xyz[-1]
    return np.broadcast_to(z.reshape(view), shp).copy()


def tilted_plane_sdf(shape_xyz, h, point, angle_deg):
    """SDF of the line (2D) through `point` (metres) whose normal into the
    domain is (sin a, cos a), a = angle from the vertical."""
    assert len(shape_xyz) == 2
    a = math.radians(angle_deg)
    nx, nz = math.sin(a), math.cos(a)
    x = np.arange(shape_xyz[0], dtype=np.float64) * h - point[0]
    z = np.arange(shape_xyz[1], dtype=np.float64) * h - point[1]
    return z[:, None] * nz + x[None, :] * nx


def heightfield_sdf_2d(nx, nz, h, zs, dzs, band=12, newton=8, device="cpu"):
    """Euclidean SDF of the curve z = zs(x) (domain below).

    zs, dzs: callables on float64 torch tensors (metres).  Within `band` grid
    steps (vertically) of the curve the distance is found by a dense search
    over x' followed by Newton steps on |x - x'|^2 + (z - zs(x'))^2; outside the
    band the vertical offset z - zs(x) is used (correct sign, larger
    magnitude), which no near-surface computation reads.
    """
    x = torch.arange(nx, dtype=torch.float64, device=device) * h
    z = torch.arange(nz, dtype=torch.float64, device=device) * h
    Z, X = torch.meshgrid(z, x, indexing="ij")
    vert = Z - zs(X)
    sdf = vert.clone()
    sel = vert.abs() <= band * h
    xs, zsel = X[sel], Z[sel]
    # dense search
    offs = torch.linspace(-band * h, band * h, 8 * band + 1, dtype=torch.float64, device=device)
    best = None
    bestx = None
    for o in offs:
        xp = xs + o
        dd = (xs - xp) ** 2 + (zsel - zs(xp)) ** 2
        if best is None:
            best, bestx = dd, xp.clone()
        else:
            m = dd < best
            best = torch.where(m, dd, best)
            bestx = torch.where(m, xp, bestx)
    xp = bestx
    for _ in range(newton):
        f = zs(xp)
        g = dzs(xp)
        eps = 1e-3
        g2 = (dzs(xp + eps) - dzs(xp - eps)) / (2 * eps)
        grad = -(xs - xp) - (zsel - f) * g
        hess = 1.0 + g * g - (zsel - f) * g2
        xp = xp - grad / torch.clamp(hess, min=0.1)
    dist = torch.sqrt((xs - xp) ** 2 + (zsel - zs(xp)) ** 2)
    sdf[sel] = torch.sign(vert[sel]) * dist
    return sdf.cpu().numpy()


def sinusoid_sdf(nx, nz, h, z0=200.0, amp=60.0, wavelength=1500.0, device="cpu"):
    """Free surface z_s(x) = z0 + amp sin(2 pi x / wavelength)."""
    k = 2 * math.pi / wavelength
    zs = lambda x: z0 + amp * torch.sin(k * x)
    dzs = lambda x: amp * k * torch.cos(k * x)
    return heightfield_sdf_2d(nx, nz, h, zs, dzs, device=device)


def hills_params(n_hills, seed, extent_x, extent_y, hmin=50.0, hmax=400.0,
                 smin=300.0, smax=1500.0):
    rng = np.random.default_rng(seed)
    return dict(hgt=rng.uniform(hmin, hmax, n_hills), sig=rng.uniform(smin, smax, n_hills),
                cx=rng.uniform(0, extent_x, n_hills), cy=rng.uniform(0, extent_y, n_hills))


def hills_surface(params, datum=1000.0, zmin=100.0):
    """z_s(x, y) = max(datum - sum h_i exp(-|x - c_i|^2 / (2 s_i^2)), zmin) and
    its first and second derivatives (torch callables)."""
    P = {k: torch.as_tensor(v, dtype=torch.float64) for k, v in params.items()}

    def parts(x, y):
        dev = x.device
        hgt, sig, cx, cy = (P[k].to(dev) for k in ("hgt", "sig", "cx", "cy"))
        z = torch.zeros_like(x)
        zx = torch.zeros_like(x)
        zy = torch.zeros_like(x)
        zxx = torch.zeros_like(x)
        zyy = torch.zeros_like(x)
        zxy = torch.zeros_like(x)
        for i in range(hgt.numel()):
            dx = x - cx[i]
            dy = y - cy[i]
            s2 = sig[i] * sig[i]
            g = hgt[i] * torch.exp(-(dx * dx + dy * dy) / (2 * s2))
            z = z + g
            zx = zx - g * dx / s2
            zy = zy - g * dy / s2
            zxx = zxx + g * (dx * dx / s2 - 1) / s2
            zyy = zyy + g * (dy * dy / s2 - 1) / s2
            zxy = zxy + g * dx * dy / (s2 * s2)
        surf = datum - z
        clamp = surf < zmin
        surf = torch.where(clamp, torch.full_like(surf, zmin), surf)
        zero = torch.zeros_like(x)
        return (surf, torch.where(clamp, zero, -zx), torch.where(clamp, zero, -zy),
                torch.where(clamp, zero, -zxx), torch.where(clamp, zero, -zyy),
                torch.where(clamp, zero, -zxy))

    return parts


def heightfield_sdf_3d(nx, ny, nz, h, parts, band=12, newton=10, device="cpu",
                       chunk=1 << 22):
    """Euclidean SDF of the surface z = z_s(x, y) (domain below), by damped
    Newton steps on the closest-point problem inside a vertical band of `band`
    grid steps; the vertical offset elsewhere."""
    x = torch.arange(nx, dtype=torch.float64, device=device) * h
    y = torch.arange(ny, dtype=torch.float64, device=device) * h
    Y, X = torch.meshgrid(y, x, indexing="ij")
    zsurf = parts(X, Y)[0]                                     # [ny][nx]
    z = torch.arange(nz, dtype=torch.float64, device=device) * h
    sdf = (z[:, None, None] - zsurf[None, :, :]).clone()      # [nz][ny][nx]
    sel = sdf.abs() <= band * h
    idx = torch.nonzero(sel.reshape(-1)).squeeze(1)
    flat = sdf.reshape(-1)
    for c0 in range(0, idx.numel(), chunk):
        ii = idx[c0:c0 + chunk]
        iz = ii // (ny * nx)
        iy = (ii // nx) % ny
        ix = ii % nx
        px, py, pz = ix.double() * h, iy.double() * h, iz.double() * h
        qx, qy = px.clone(), py.clone()
        for _ in range(newton):
            f, fx, fy, fxx, fyy, fxy = parts(qx, qy)
            r = pz - f
            gx = -(px - qx) - r * fx
            gy = -(py - qy) - r * fy
            hxx = 1 + fx * fx - r * fxx
            hyy = 1 + fy * fy - r * fyy
            hxy = fx * fy - r * fxy
            det = hxx * hyy - hxy * hxy
            ok = (det > 1e-6) & (hxx > 0)
            sx = torch.where(ok, (hyy * gx - hxy * gy) / torch.where(ok, det, torch.ones_like(det)), gx)
            sy = torch.where(ok, (hxx * gy - hxy * gx) / torch.where(ok, det, torch.ones_like(det)), gy)
            qx = qx - sx
            qy = qy - sy
        f = parts(qx, qy)[0]
        dist = torch.sqrt((px - qx) ** 2 + (py - qy) ** 2 + (pz - f) ** 2)
        vert = flat[ii]
        dist = torch.minimum(dist, vert.abs())
        flat[ii] = torch.sign(vert) * dist
    return sdf.cpu().numpy(), zsurf.cpu().numpy()


# ---------------------------------------------------------------------------
# velocity models
# ---------------------------------------------------------------------------
def layered_velocity(shape_xyz, h, depths, values):
    """Velocity by depth: values[k] between depths[k-1] and depths[k]."""
    z = np.arange(shape_xyz[-1], dtype=np.float64) * h
    v1 = np.full_like(z, values[0])
    for dep, val in zip(depths, values[1:]):
        v1[z >= dep] = val
    d = len(shape_xyz)
    view = [1] * d
    view[0] = shape_xyz[-1]
    return np.broadcast_to(v1.reshape(view), tuple(reversed(shape_xyz))).copy()


def smooth_random_velocity_3d(nx, ny, nz, h, zsurf, seed, vmin=1500.0, vmax=4000.0,
                              sigma=500.0, n_modes=64, device="cpu"):
    """Smooth random field (random Fourier modes with a Gaussian spectrum of
    correlation length `sigma`) blended with depth below the surface and mapped
    to [vmin, vmax]."""
    rng = np.random.default_rng(seed)
    kv = rng.normal(0.0, 1.0 / sigma, size=(n_modes, 3))
    ph = rng.uniform(0, 2 * math.pi, n_modes)
    x = torch.arange(nx, dtype=torch.float64, device=device) * h
    y = torch.arange(ny, dtype=torch.float64, device=device) * h
    out = torch.empty((nz, ny, nx), dtype=torch.float32, device=device)
    Y, X = torch.meshgrid(y, x, indexing="ij")
    zs = torch.as_tensor(zsurf, dtype=torch.float64, device=device)
    depth_span = nz * h
    for iz in range(nz):
        z = iz * h
        f = torch.zeros_like(X)
        for m in range(n_modes):
            f = f + torch.cos(kv[m, 0] * X + kv[m, 1] * Y + kv[m, 2] * z + ph[m])
        f = f / math.sqrt(n_modes / 2.0)                 # ~unit variance
        f01 = 0.5 + 0.25 * torch.clamp(f, -2.0, 2.0)     # in [0, 1]
        dep = torch.clamp((z - zs) / depth_span, 0.0, 1.0)
        t = torch.clamp(0.5 * f01 + 0.5 * dep, 0.0, 1.0)
        out[iz] = (vmin + (vmax - vmin) * t).float()
    return out.cpu().numpy()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload_flat2d(nx=201, nz=201, h=10.0, c=1500.0, M=4, courant=0.4, nt=500,
                    z0_cells=40.3, f0=10.0, src_cells=(100.0, 80.0),
                    rec_x_cells=(50, 150), rec_z_cells=45, bc="free"):
    """2D second-order, constant velocity, flat off-grid surface at z = 40.3 h,
    10 Hz Ricker at (100 h, 80 h), 101 receivers on row z = 45 h."""
    sdf = flat_surface_sdf((nx, nz), h, z0_cells * h)
    vel = np.full((nz, nx), c, dtype=np.float64)
    dt = dt_from_courant(courant, h, c)
    src = np.array([[src_cells[0] * h, src_cells[1] * h]])
    rx = np.arange(rec_x_cells[0], rec_x_cells[1] + 1, dtype=np.float64) * h
    rec = np.stack([rx, np.full_like(rx, rec_z_cells * h)], axis=1)
    return dict(name="flat2d", ndim=2, shape=(nx, nz), h=h, M=M, sdf=sdf, vel=vel, dt=dt, nt=nt,
                src=src, rec=rec, wavelet=ricker(f0, dt, nt), bc=bc, z0=z0_cells * h, c=c, f0=f0)


def workload_sinusoid_staggered(nx=1001, nz=1001, h=5.0, M=8, nt=3000, courant=0.4,
                                seed=2, f0=12.0, bc="free", rho=1000.0, device="cpu"):
    """2D first-order staggered: z_s(x) = 200 + 60 sin(2 pi x / 1500) m, four
    layers 1500/2200/2800/3500 m/s at seeded sorted depths in [500, 4500] m,
    12 Hz Ricker at (2500, 600) m, 500 receivers 10 m below the surface."""
    rng = np.random.default_rng(seed)
    hi = min(4500.0, (nz - 1) * h)
    depths = np.sort(rng.uniform(min(500.0, 0.5 * hi), hi, 3))
    vals = [1500.0, 2200.0, 2800.0, 3500.0]
    sdf = sinusoid_sdf(nx, nz, h, device=device)
    vel = layered_velocity((nx, nz), h, depths, vals).astype(np.float32)
    dt = dt_from_courant(courant, h, max(vals))
    Lx = (nx - 1) * h
    src = np.array([[min(2500.0, 0.5 * Lx), min(600.0, 0.6 * (nz - 1) * h)]])
    rx = np.linspace(0.05 * Lx, 0.95 * Lx, 500 if nx >= 500 else nx // 2)
    rz = 200.0 + 60.0 * np.sin(2 * math.pi * rx / 1500.0) + 10.0
    rec = np.stack([rx, rz], axis=1)
    return dict(name="sinusoid_staggered", ndim=2, shape=(nx, nz), h=h, M=M, sdf=sdf, vel=vel,
                rho=np.full((nz, nx), rho, dtype=np.float32), dt=dt, nt=nt, src=src, rec=rec,
                wavelet=ricker(f0, dt, nt), bc=bc, depths=depths)


def workload_hills3d(nx=512, ny=512, nz=384, h=10.0, M=8, nt=2000, courant=0.45, seed=3,
                     n_hills=12, f0=10.0, bc="free", rec_stride=2, device="cpu", hmax=400.0):
    """3D second-order: z_s = 1000 m - sum of seeded Gaussian hills (heights
    50-400 m, widths 300-1500 m), clamped at 100 m; smooth random velocity in
    [1500, 4000] m/s increasing with depth; 10 Hz source 500 m below the
    surface at the centre; receivers every `rec_stride` nodes 2 h below it."""
    Lx, Ly = (nx - 1) * h, (ny - 1) * h
    prm = hills_params(n_hills, seed, Lx, Ly, hmax=hmax)
    parts = hills_surface(prm)
    sdf, zsurf = heightfield_sdf_3d(nx, ny, nz, h, parts, device=device)
    vel = smooth_random_velocity_3d(nx, ny, nz, h, zsurf, seed, device=device)
    dt = dt_from_courant(courant, h, 4000.0)
    cx, cy = 0.5 * Lx, 0.5 * Ly
    icx, icy = int(round(cx / h)), int(round(cy / h))
    src = np.array([[cx, cy, min(zsurf[icy, icx] + 500.0, (nz - 2) * h)]])
    rxs = np.arange(0, nx, rec_stride)
    rys = np.arange(0, ny, rec_stride)
    RY, RX = np.meshgrid(rys, rxs, indexing="ij")
    rz = zsurf[RY, RX] + 2 * h
    rec = np.stack([RX.ravel() * h, RY.ravel() * h, rz.ravel()], axis=1)
    return dict(name="hills3d", ndim=3, shape=(nx, ny, nz), h=h, M=M, sdf=sdf, vel=vel, dt=dt,
                nt=nt, src=src, rec=rec, wavelet=ricker(f0, dt, nt), bc=bc, zsurf=zsurf)


def damping_eta(cmax, width, h, reflection):
    """Peak coefficient (1/s) of a quadratic absorbing layer of `width` nodes
    for a nominal reflection coefficient: 1.5 cmax ln(1 / R) / (W h)."""
    return 1.5 * cmax * math.log(1.0 / reflection) / (width * h)


def workload_shot2d(shot, h=10.0, M=8, nt=2000, courant=0.4, f0=10.0, bc="free",
                    side=(400, 1200), device="cpu"):
    """One shot of the batched set: sides uniform in [400, 1200] (seed 4 + shot),
    surface a + b sin(2 pi x / lam) + Gaussian bump, 3-5 layers below it; an
    absorbing layer of 20 nodes on the sides and the bottom (nominal
    reflection 1e-8) in `damp`."""
    rng = np.random.default_rng(4 + shot)
    nx = int(rng.integers(side[0], side[1] + 1))
    nz = int(rng.integers(side[0], side[1] + 1))
    Lx, Lz = (nx - 1) * h, (nz - 1) * h
    a = rng.uniform(0.08, 0.15) * Lz
    b = rng.uniform(10.0, 60.0)
    lam = rng.uniform(800.0, 2500.0)
    bh = rng.uniform(20.0, 80.0)
    bc_x = rng.uniform(0.2, 0.8) * Lx
    bs = rng.uniform(150.0, 400.0)
    k = 2 * math.pi / lam
    zs = lambda x: a + b * torch.sin(k * x) - bh * torch.exp(-(x - bc_x) ** 2 / (2 * bs * bs))
    dzs = lambda x: (b * k * torch.cos(k * x)
                     + bh * (x - bc_x) / (bs * bs) * torch.exp(-(x - bc_x) ** 2 / (2 * bs * bs)))
    sdf = heightfield_sdf_2d(nx, nz, h, zs, dzs, device=device)
    nl = int(rng.integers(3, 6))
    depths = np.sort(rng.uniform(a + b + 200.0, Lz, nl - 1))
    vals = np.sort(rng.uniform(1500.0, 4000.0, nl))
    vel = layered_velocity((nx, nz), h, depths, vals).astype(np.float32)
    dt = dt_from_courant(courant, h, 4000.0)
    src = np.array([[rng.uniform(0.3, 0.7) * Lx, a + b + 300.0]])
    rx = np.arange(5, nx - 5, 4, dtype=np.float64) * h
    xt = torch.as_tensor(rx)
    rz = zs(xt).numpy() + 2 * h
    rec = np.stack([rx, rz], axis=1)
    return dict(name="shot2d_%d" % shot, ndim=2, shape=(nx, nz), h=h, M=M, sdf=sdf, vel=vel,
                dt=dt, nt=nt, src=src, rec=rec, wavelet=ricker(f0, dt, nt), bc=bc,
                damp=(20, damping_eta(4000.0, 20, h, 1e-8)))


# ---------------------------------------------------------------------------
# learned-stencil network: seeded initial parameters and training topographies
# ---------------------------------------------------------------------------
def mlp_init(n_in, n_hidden, n_layers, n_out, seed):
    """Flat FP32 parameter vector (W_0, b_0, W_1, b_1, ...), W_l [n_out][n_in]
    uniform in +-sqrt(6 / fan_in) (He initialisation), biases zero."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    parts = []
    for i in range(len(dims) - 1):
        a = math.sqrt(6.0 / dims[i])
        parts.append(rng.uniform(-a, a, size=dims[i + 1] * dims[i]))
        parts.append(np.zeros(dims[i + 1]))
    return np.concatenate(parts).astype(np.float32)


def random_hills_sdf(nx, ny, nz, h, seed, n_hills=12, device="cpu"):
    """SDF of a seeded sum of Gaussian hills on a datum at ~55% depth, with
    heights and widths scaled to the grid (training topographies)."""
    rng = np.random.default_rng(seed + 7919)
    depth = (nz - 1) * h
    prm = hills_params(n_hills, seed, (nx - 1) * h, (ny - 1) * h, hmin=0.05 * depth, hmax=0.3 * depth,
                       smin=3.0 * h, smax=0.2 * min(nx, ny) * h)
    datum = float(rng.uniform(0.5, 0.6)) * depth
    parts = hills_surface(prm, datum=datum, zmin=0.15 * depth)
    sdf, _ = heightfield_sdf_3d(nx, ny, nz, h, parts, device=device)
    return sdf


def workload_learned3d(nx=768, ny=768, nz=384, h=10.0, M=8, nt=1500, seed=5, device="cpu"):
    """3D second-order on a sum of 60 seeded Gaussian hills (heights 50-250 m,
    widths 300-1500 m) on a 1 km datum, free surface, order 8, 1500 steps;
    receivers every third node 2 h below the surface."""
    w = workload_hills3d(nx=nx, ny=ny, nz=nz, h=h, M=M, nt=nt, seed=seed, n_hills=60, hmax=250.0,
                         rec_stride=3, device=device)
    w["name"] = "learned3d"
    return w


def training_hills_sdf(seed, nx=256, ny=256, nz=160, h=10.0, device="cpu"):
    """Training topography for the learned stencils: the same hill statistics
    as ``workload_learned3d`` (7 hills on a 256 x 256 patch), seeded."""
    Lx, Ly = (nx - 1) * h, (ny - 1) * h
    prm = hills_params(7, seed, Lx, Ly, hmax=250.0)
    parts = hills_surface(prm, datum=0.6 * (nz - 1) * h, zmin=0.2 * (nz - 1) * h)
    sdf, _ = heightfield_sdf_3d(nx, ny, nz, h, parts, device=device)
    return sdf
