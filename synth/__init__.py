"""Seeded synthetic inputs shaped like the paper's downscaling workloads.

This module is shared by the CUDA path's tests and benchmark and by the
CPU oracle's tests.  It holds none of the method's arithmetic: it only
builds a terrain-following node grid (x_i, y_j, z_s(x_i, y_j) + zeta_k)
and a first-guess wind u0 at the nodes.  Everything is float64 numpy.

Layout of every nodal array: ``[k][j][i]`` with i fastest, shape
``(nz+1, ny+1, nx+1)``; the wind is ``[3][k][j][i]`` (u, v, w).

Recipes (the paper has no dataset; these follow its target domain of
3000 x 3000 x 15 cells at 30 m, Sec. 1, and the grid it describes in
Sec. 2-3: terrain following, stretched vertically away from the ground):

* layer thicknesses 5 * 1.2**k m (k = 0 at the ground), zeta_0 = 0;
* log-law wind U(z) = U_ref ln(max(z, z0)/z0) / ln(10/z0), z the height
  above ground, z0 = 0.1 m, U_ref the speed at 10 m;
* meteorological direction theta (the direction the wind comes from):
  u = -U sin(theta), v = -U cos(theta), w = 0;
* Gaussian hills H exp(-r^2 / (2 sigma^2)), evaluated within 5 sigma of
  the center (zero beyond; the truncation is part of the recipe).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Z0 = 0.1          # roughness length [m]
DX = 30.0         # horizontal spacing [m]


def layer_thicknesses(nz: int, h0: float = 5.0, ratio: float = 1.2) -> np.ndarray:
    """Thickness of each of the nz layers, ground first."""
    return h0 * ratio ** np.arange(nz, dtype=np.float64)


def zeta_levels(nz: int, h0: float = 5.0, ratio: float = 1.2) -> np.ndarray:
    """Heights above ground of the nz+1 node layers."""
    return np.concatenate([[0.0], np.cumsum(layer_thicknesses(nz, h0, ratio))])


def add_hill(zs: np.ndarray, x: np.ndarray, y: np.ndarray, xc: float, yc: float,
             height: float, sigma: float) -> None:
    """Add one Gaussian hill to the terrain array zs[j][i] in place."""
    r = 5.0 * sigma
    i0 = max(0, int(math.floor((xc - r - x[0]) / (x[1] - x[0]))))
    i1 = min(len(x), int(math.ceil((xc + r - x[0]) / (x[1] - x[0]))) + 1)
    j0 = max(0, int(math.floor((yc - r - y[0]) / (y[1] - y[0]))))
    j1 = min(len(y), int(math.ceil((yc + r - y[0]) / (y[1] - y[0]))) + 1)
    if i0 >= i1 or j0 >= j1:
        return
    dx2 = (x[i0:i1] - xc) ** 2
    dy2 = (y[j0:j1] - yc) ** 2
    d2 = dy2[:, None] + dx2[None, :]
    g = height * np.exp(-d2 / (2.0 * sigma * sigma))
    g[d2 > r * r] = 0.0
    zs[j0:j1, i0:i1] += g


def log_law(zag: np.ndarray, u_ref: float, z0: float = Z0) -> np.ndarray:
    return u_ref * np.log(np.maximum(zag, z0) / z0) / math.log(10.0 / z0)


@dataclass
class Case:
    """One synthetic downscaling problem."""
    name: str
    nx: int
    ny: int
    nz: int
    a: tuple
    X: np.ndarray
    Y: np.ndarray
    Z: np.ndarray
    u0: np.ndarray
    h1: float
    h3: np.ndarray            # layer thicknesses above flat ground (planning hint)
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_free(self) -> int:
        return (self.nx - 1) * (self.ny - 1) * self.nz


def node_grid(nx: int, ny: int, nz: int, zs: np.ndarray, dx: float = DX,
              h0: float = 5.0, ratio: float = 1.2):
    """Shift-form terrain-following grid: X=x_i, Y=y_j, Z=z_s(x_i,y_j)+zeta_k."""
    x = dx * np.arange(nx + 1, dtype=np.float64)
    y = dx * np.arange(ny + 1, dtype=np.float64)
    zeta = zeta_levels(nz, h0, ratio)
    shape = (nz + 1, ny + 1, nx + 1)
    X = np.broadcast_to(x[None, None, :], shape).copy()
    Y = np.broadcast_to(y[None, :, None], shape).copy()
    Z = zs[None, :, :] + zeta[:, None, None]
    return X, Y, np.ascontiguousarray(Z), zeta


def log_wind(nx, ny, nz, zeta, u_ref, theta_deg, noise, rng):
    shape = (nz + 1, ny + 1, nx + 1)
    U = log_law(zeta, u_ref)[:, None, None]
    th = math.radians(theta_deg)
    u0 = np.zeros((3,) + shape)
    u0[0] = -U * math.sin(th)
    u0[1] = -U * math.cos(th)
    if noise > 0:
        u0 += rng.normal(0.0, noise, size=u0.shape)
    return u0


def single_hill(nx=64, ny=64, nz=8, seed=0, a=(1.0, 1.0, 1.0), height=150.0,
                sigma=400.0, u_ref=8.0, theta=270.0, noise=0.2, dx=DX) -> Case:
    """One centered Gaussian hill with a log-law wind plus iid noise at the
    nodes; at the defaults this is the 64 x 64 x 8 cell, 65 x 65 x 9 node
    problem with a 150 m hill, sigma 400 m, 8 m/s from 270 deg, noise 0.2."""
    rng = np.random.default_rng(seed)
    x = dx * np.arange(nx + 1)
    y = dx * np.arange(ny + 1)
    zs = np.zeros((ny + 1, nx + 1))
    add_hill(zs, x, y, 0.5 * x[-1], 0.5 * y[-1], height, sigma)
    X, Y, Z, zeta = node_grid(nx, ny, nz, zs, dx)
    u0 = log_wind(nx, ny, nz, zeta, u_ref, theta, noise, rng)
    return Case(f"hill{nx}x{ny}x{nz}", nx, ny, nz, tuple(a), X, Y, Z, u0, dx,
                layer_thicknesses(nz))


def random_hills(nx=512, ny=512, nz=16, seed=0, a=(1.0, 1.0, 1.0), n_hills=40,
                 hmin=50.0, hmax=500.0, smin=200.0, smax=1500.0, u_ref=10.0,
                 noise=0.5, dx=DX) -> Case:
    """Sum of seeded random Gaussian hills, log-law wind from a random
    direction plus iid noise: at the defaults the 512 x 512 x 16 cell case."""
    rng = np.random.default_rng(seed)
    x = dx * np.arange(nx + 1)
    y = dx * np.arange(ny + 1)
    zs = np.zeros((ny + 1, nx + 1))
    for _ in range(n_hills):
        h = rng.uniform(hmin, hmax)
        s = rng.uniform(smin, smax)
        xc = rng.uniform(0.0, x[-1])
        yc = rng.uniform(0.0, y[-1])
        add_hill(zs, x, y, xc, yc, h, s)
    theta = rng.uniform(0.0, 360.0)
    X, Y, Z, zeta = node_grid(nx, ny, nz, zs, dx)
    u0 = log_wind(nx, ny, nz, zeta, u_ref, theta, noise, rng)
    return Case(f"hills{nx}x{ny}x{nz}", nx, ny, nz, tuple(a), X, Y, Z, u0, dx,
                layer_thicknesses(nz), {"theta": theta})


def _bilinear_matrix(n_fine: int, n_coarse: int) -> np.ndarray:
    """Dense (n_fine, n_coarse) bilinear weights from a coarse lattice that
    spans the same extent as the fine one."""
    t = np.linspace(0.0, n_coarse - 1.0, n_fine)
    i0 = np.minimum(np.floor(t).astype(np.int64), n_coarse - 2)
    w = t - i0
    W = np.zeros((n_fine, n_coarse))
    W[np.arange(n_fine), i0] = 1.0 - w
    W[np.arange(n_fine), i0 + 1] = w
    return W


def ridge_terrain(nx, ny, rng, dx=DX, n_hills=400, zmax=1200.0):
    x = dx * np.arange(nx + 1)
    y = dx * np.arange(ny + 1)
    zs = np.zeros((ny + 1, nx + 1))
    for _ in range(n_hills):
        h = rng.uniform(50.0, 500.0)
        s = rng.uniform(200.0, 1500.0)
        add_hill(zs, x, y, rng.uniform(0, x[-1]), rng.uniform(0, y[-1]), h, s)
    # Gaussian ridge band through the center, sigma 1 km (about 2 km wide).
    ang = rng.uniform(0.0, math.pi)
    xc, yc = 0.5 * x[-1], 0.5 * y[-1]
    nxr, nyr = -math.sin(ang), math.cos(ang)
    for j0 in range(0, ny + 1, 512):
        j1 = min(ny + 1, j0 + 512)
        d = (x[None, :] - xc) * nxr + (y[j0:j1, None] - yc) * nyr
        zs[j0:j1] += 800.0 * np.exp(-d * d / (2.0 * 1000.0 ** 2))
    zs *= zmax / zs.max()
    return zs


def full_domain(nx=3000, ny=3000, nz=15, seed=0, a=(1.0, 1.0, 1.0), dx=DX,
                coarse=100) -> Case:
    """Ridge-and-hills terrain (400 hills + a ridge band, max 1200 m) with u0
    bilinearly interpolated per node layer from a coarse 100 x 100 x nz wind
    whose layer means rise linearly from 5 to 15 m/s along a seeded
    direction, plus N(0, 2) on u and v; w = 0.  At the defaults this is the
    3000 x 3000 x 15 cell, 90 km square domain."""
    rng = np.random.default_rng(seed)
    zs = ridge_terrain(nx, ny, rng, dx)
    X, Y, Z, zeta = node_grid(nx, ny, nz, zs, dx)
    del X, Y
    theta = rng.uniform(0.0, 360.0)
    th = math.radians(theta)
    means = np.linspace(5.0, 15.0, nz)
    cu = -means[:, None, None] * math.sin(th) + rng.normal(0.0, 2.0, (nz, coarse, coarse))
    cv = -means[:, None, None] * math.cos(th) + rng.normal(0.0, 2.0, (nz, coarse, coarse))
    Wy = _bilinear_matrix(ny + 1, coarse)
    Wx = _bilinear_matrix(nx + 1, coarse)
    shape = (nz + 1, ny + 1, nx + 1)
    u0 = np.zeros((3,) + shape)
    for k in range(nz + 1):
        kc = min(k, nz - 1)
        u0[0, k] = Wy @ cu[kc] @ Wx.T
        u0[1, k] = Wy @ cv[kc] @ Wx.T
    x = dx * np.arange(nx + 1, dtype=np.float64)
    y = dx * np.arange(ny + 1, dtype=np.float64)
    X = np.broadcast_to(x[None, None, :], shape).copy()
    Y = np.broadcast_to(y[None, :, None], shape).copy()
    return Case(f"domain{nx}x{ny}x{nz}", nx, ny, nz, tuple(a), X, Y, Z, u0, dx,
                layer_thicknesses(nz), {"theta": theta})


def full_domain_window(i0, j0, w, h, nx=3000, ny=3000, nz=15, seed=0, a=(1.0, 1.0, 1.0),
                       dx=DX, coarse=100) -> Case:
    """Cells [i0, i0+w) x [j0, j0+h) of full_domain(nx, ny, nz, seed): the
    same terrain, wind and node positions, cut out as a w x h x nz problem
    (its lateral faces become fixed boundaries)."""
    rng = np.random.default_rng(seed)
    zs = ridge_terrain(nx, ny, rng, dx)
    theta = rng.uniform(0.0, 360.0)
    th = math.radians(theta)
    means = np.linspace(5.0, 15.0, nz)
    cu = -means[:, None, None] * math.sin(th) + rng.normal(0.0, 2.0, (nz, coarse, coarse))
    cv = -means[:, None, None] * math.cos(th) + rng.normal(0.0, 2.0, (nz, coarse, coarse))
    Wy = _bilinear_matrix(ny + 1, coarse)[j0:j0 + h + 1]
    Wx = _bilinear_matrix(nx + 1, coarse)[i0:i0 + w + 1]
    zeta = zeta_levels(nz)
    shape = (nz + 1, h + 1, w + 1)
    Z = zs[None, j0:j0 + h + 1, i0:i0 + w + 1] + zeta[:, None, None]
    x = dx * np.arange(i0, i0 + w + 1, dtype=np.float64)
    y = dx * np.arange(j0, j0 + h + 1, dtype=np.float64)
    X = np.broadcast_to(x[None, None, :], shape).copy()
    Y = np.broadcast_to(y[None, :, None], shape).copy()
    u0 = np.zeros((3,) + shape)
    for k in range(nz + 1):
        kc = min(k, nz - 1)
        u0[0, k] = Wy @ cu[kc] @ Wx.T
        u0[1, k] = Wy @ cv[kc] @ Wx.T
    return Case(f"window{w}x{h}x{nz}@{i0},{j0}", w, h, nz, tuple(a), X, Y,
                np.ascontiguousarray(Z), u0, dx, layer_thicknesses(nz), {"theta": theta})


def batch_domains(n=96, seed=0, nmin=48, nmax=384, zmin=8, zmax=20, a3_choices=(1.0, 4.0, 10.0),
                  dx=DX):
    """n independent domains of uneven sizes: horizontal cells uniform in
    [nmin, nmax] per axis, vertical cells uniform in [zmin, zmax], a3 drawn
    from a3_choices (a1 = a2 = 1); each with a few random hills (H ~ U[50,150]
    m, sigma ~ U[200,600] m, one per 100 x 100 cells, at least one) and a
    log-law wind of 8 m/s from a random direction plus N(0, 0.2) per node."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n):
        nx = int(rng.integers(nmin, nmax + 1))
        ny = int(rng.integers(nmin, nmax + 1))
        nz = int(rng.integers(zmin, zmax + 1))
        a3 = float(a3_choices[int(rng.integers(0, len(a3_choices)))])
        x = dx * np.arange(nx + 1)
        y = dx * np.arange(ny + 1)
        zs = np.zeros((ny + 1, nx + 1))
        for _ in range(max(1, (nx * ny) // 10000)):
            add_hill(zs, x, y, rng.uniform(0, x[-1]), rng.uniform(0, y[-1]),
                     rng.uniform(50.0, 150.0), rng.uniform(200.0, 600.0))
        X, Y, Z, zeta = node_grid(nx, ny, nz, zs, dx)
        u0 = log_wind(nx, ny, nz, zeta, 8.0, rng.uniform(0.0, 360.0), 0.2, rng)
        out.append(Case(f"dom{d}_{nx}x{ny}x{nz}_a{a3:g}", nx, ny, nz, (1.0, 1.0, a3), X, Y, Z, u0,
                        dx, layer_thicknesses(nz)))
    return out


def perturb_wind(u0: np.ndarray, seed: int, rel: float = 0.02) -> np.ndarray:
    """The next time step's first guess: u0 * (1 + rel * xi), xi ~ N(0, 1)."""
    rng = np.random.default_rng(seed + 1000003)
    return u0 * (1.0 + rel * rng.standard_normal(u0.shape))


def flat_box(nx, ny, nz, dx=DX, dz=None, a=(1.0, 1.0, 1.0), u0=None, stretch=1.0) -> Case:
    """Flat ground, box elements: X=x_i, Y=y_j, Z=zeta_k (used by pins)."""
    zs = np.zeros((ny + 1, nx + 1))
    h0 = dz if dz is not None else 5.0
    X, Y, Z, zeta = node_grid(nx, ny, nz, zs, dx, h0, stretch)
    if u0 is None:
        u0 = np.zeros((3, nz + 1, ny + 1, nx + 1))
    return Case(f"box{nx}x{ny}x{nz}", nx, ny, nz, tuple(a), X, Y, Z, u0, dx,
                layer_thicknesses(nz, h0, stretch))


def jittered(nx, ny, nz, seed=0, amp=0.2, dx=DX, a=(1.0, 1.0, 1.0)) -> Case:
    """A general (non shift-form) hexahedral grid: every node of a stretched
    box grid moved by a seeded random offset of up to amp times the local
    spacing in each direction, with random nodal wind.  Elements stay
    convex for amp < 0.25."""
    rng = np.random.default_rng(seed)
    zs = np.zeros((ny + 1, nx + 1))
    X, Y, Z, zeta = node_grid(nx, ny, nz, zs, dx)
    dz = np.diff(zeta)
    dzn = np.minimum(np.concatenate([dz, dz[-1:]]), np.concatenate([dz[:1], dz]))
    X = X + amp * dx * rng.uniform(-1, 1, X.shape)
    Y = Y + amp * dx * rng.uniform(-1, 1, Y.shape)
    Z = Z + amp * dzn[:, None, None] * rng.uniform(-1, 1, Z.shape)
    u0 = rng.normal(0.0, 1.0, (3, nz + 1, ny + 1, nx + 1))
    return Case(f"jit{nx}x{ny}x{nz}", nx, ny, nz, tuple(a), X, Y, Z, u0, dx,
                layer_thicknesses(nz))
