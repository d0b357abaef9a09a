"""CPU ORACLE -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product: it shares no code with the
CUDA path.  Inputs come from the seeded generators in ``synth``.

It computes, plainly and in FP64, the discrete problem of the paper
(Mandel et al., arXiv:2101.08453):

* ``assemble_K`` / ``assemble_f``: the global stiffness matrix and load
  vector of Eq. 5 by the element loop in ``fe_oracle.c`` (2x2x2 Gauss on
  isoparametric trilinear hexahedra, Sec. 2);
* boundary conditions of Eq. 4: lambda = 0 on the top and lateral faces,
  natural (no condition) on the terrain surface Gamma; the free nodes are
  1 <= i <= nx-1, 1 <= j <= ny-1, 0 <= k <= nz-1 (Dirichlet wins on edges);
* ``solve``: K_FF lambda_F = f_F by sparse LU (SuperLU) or by conjugate
  gradients to a 1e-14 true relative residual;
* ``recover``: u = u0 + A^{-1} grad lambda, Eq. 3;
* ``kkt_dense``: the constrained least-squares problem of Eq. 1 in its
  discrete form, min 1/2 (u-u0)^T M (u-u0) subject to B_F u = 0, solved as
  one dense saddle-point system (tiny grids only);
* the multigrid cycle of Sec. 3 step by step: ``plan_levels`` (adaptive
  semicoarsening rule), ``prolongation`` (trilinear index-space weights
  over 2x2x2 agglomerations), ``galerkin`` (K_c = P^T K P, Eq. 7),
  ``gs_sweep`` (vertical Gauss-Seidel in 4 column groups), ``vcycle``.

Every function says which passage it follows.  "parity unpinned": none;
each function is pinned by the tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.POINTER(ctypes.c_int64)
        c_int = ctypes.c_int
        L.oracle_element_stiffness.argtypes = [d, d, d]
        L.oracle_element_rhs.argtypes = [d, d, c_int, d]
        L.oracle_assemble_coo.argtypes = [c_int] * 3 + [d] * 4 + [i64, i64, d]
        L.oracle_assemble_rhs.argtypes = [c_int] * 3 + [d] * 4 + [c_int, d]
        L.oracle_assemble_rhs_par.argtypes = [c_int] * 3 + [d] * 4 + [c_int, d]
        L.oracle_stencil_row.argtypes = [c_int] * 3 + [d] * 4 + [c_int] * 3 + [d]
        L.oracle_apply_K.argtypes = [c_int] * 3 + [d] * 6
        L.oracle_recover.argtypes = [c_int] * 3 + [d] * 6 + [c_int, d]
        L.oracle_weak_div.argtypes = [c_int] * 3 + [d] * 5
        L.oracle_gs_sweep.argtypes = [c_int] * 3 + [i64, i64, d, d, d, c_int]
        L.oracle_gauss_detj.argtypes = [c_int] * 3 + [d] * 4
        L.oracle_interp_gauss.argtypes = [c_int] * 3 + [d, d]
        L.oracle_assemble_rhs_centers.argtypes = [c_int] * 3 + [d] * 4 + [c_int, d]
        for name in ("oracle_element_stiffness", "oracle_element_rhs", "oracle_assemble_coo",
                     "oracle_assemble_rhs", "oracle_assemble_rhs_par", "oracle_stencil_row",
                     "oracle_apply_K", "oracle_recover", "oracle_weak_div",
                     "oracle_gauss_detj", "oracle_interp_gauss", "oracle_assemble_rhs_centers"):
            getattr(L, name).restype = c_int
        L.oracle_gs_sweep.restype = None
        _lib = L
    return _lib


def _p(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class GeometryError(RuntimeError):
    """An element with a non-positive Jacobian determinant."""


def _check(rc):
    if rc == -2:
        raise GeometryError("element with detJ <= 0")
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")


# --------------------------------------------------------------------------
# element level (Sec. 2)

def element_stiffness(xe, a):
    """8x8 element matrix of the left side of Eq. 5 (2x2x2 Gauss)."""
    xe = _f64(xe).reshape(8, 3)
    a = _f64(a)
    Ke = np.zeros((8, 8))
    _check(lib().oracle_element_stiffness(_p(xe), _p(a), _p(Ke)))
    return Ke


def element_rhs(xe, ue, quad=0):
    """Element load of the right side of Eq. 5; quad 0 = 2x2x2, 1 = center."""
    xe = _f64(xe).reshape(8, 3)
    ue = _f64(ue).reshape(8, 3)
    fe = np.zeros(8)
    _check(lib().oracle_element_rhs(_p(xe), _p(ue), quad, _p(fe)))
    return fe


# --------------------------------------------------------------------------
# global assembly and boundary conditions (Sec. 2, Eq. 4-5)

def n_nodes(nx, ny, nz):
    return (nx + 1) * (ny + 1) * (nz + 1)


def free_mask(Nx, Ny, Nz):
    """Free nodes of a grid of Nx x Ny x Nz nodes (Eq. 4: lambda = 0 on the
    top and the lateral faces; the bottom is the terrain surface Gamma)."""
    m = np.zeros((Nz, Ny, Nx), dtype=bool)
    m[: Nz - 1, 1: Ny - 1, 1: Nx - 1] = True
    return m.ravel()


def case_free_mask(c):
    return free_mask(c.nx + 1, c.ny + 1, c.nz + 1)


def assemble_K(c, a=None):
    """Full global stiffness (all nodes, no boundary condition), CSR."""
    a = _f64(c.a if a is None else a)
    NE = c.nx * c.ny * c.nz
    rows = np.empty(64 * NE, dtype=np.int64)
    cols = np.empty(64 * NE, dtype=np.int64)
    vals = np.empty(64 * NE)
    _check(lib().oracle_assemble_coo(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)),
                                     _p(_f64(c.Z)), _p(a), _p(rows, ctypes.c_int64),
                                     _p(cols, ctypes.c_int64), _p(vals)))
    N = c.n_nodes
    K = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()
    K.sum_duplicates()
    return K


def assemble_f(c, u0=None, quad=0, parallel=False):
    """Full global load vector f = -int grad mu . u0 (all nodes)."""
    u0 = _f64(c.u0 if u0 is None else u0)
    f = np.zeros(c.n_nodes)
    fn = lib().oracle_assemble_rhs_par if parallel else lib().oracle_assemble_rhs
    _check(fn(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)), _p(_f64(c.Z)), _p(u0), quad,
              _p(f)))
    return f


def assemble_f_centers(c, uc, quad=0):
    """Load vector for a wind given at the element centers, uc (3, nz, ny, nx):
    constant over each element (the paper's wind representation, Sec. 2)."""
    f = np.zeros(c.n_nodes)
    _check(lib().oracle_assemble_rhs_centers(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)),
                                             _p(_f64(c.Z)), _p(_f64(uc)), quad, _p(f)))
    return f


def recover_centers(c, lam, uc, a=None):
    """u = uc + A^{-1} grad lambda at the element centers (Eq. 3), wind given there."""
    return recover(c, lam, u0=np.zeros((3,) + c.u0.shape[1:]), where=0, a=a) + uc


def stencil_row(c, i, j, k, a=None):
    """27 coefficients of row (i, j, k) of the full K, s = (di+1)+3(dj+1)+9(dk+1)."""
    a = _f64(c.a if a is None else a)
    row = np.zeros(27)
    _check(lib().oracle_stencil_row(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)),
                                    _p(_f64(c.Z)), _p(a), i, j, k, _p(row)))
    return row


def apply_K(c, x, a=None):
    """y = K x with the full K, element by element (no matrix stored)."""
    a = _f64(c.a if a is None else a)
    x = _f64(x).ravel()
    y = np.zeros(c.n_nodes)
    _check(lib().oracle_apply_K(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)),
                                _p(_f64(c.Z)), _p(a), _p(x), _p(y)))
    return y


def restrict_free(K, free):
    """K_FF embedded in the full index space: rows and columns of fixed nodes zeroed."""
    D = sp.diags(free.astype(np.float64))
    return (D @ K @ D).tocsr()


def residual_norms(c, lam, f=None, u0=None, quad=0):
    """(||f_F - K_FF lam_F||_2, ||f_F||_2) with K applied element by element.
    lam must be zero at fixed nodes."""
    free = case_free_mask(c)
    if f is None:
        f = assemble_f(c, u0=u0, quad=quad, parallel=True)
    lam = _f64(lam).ravel().copy()
    lam[~free] = 0.0
    r = f - apply_K(c, lam)
    return float(np.linalg.norm(r[free])), float(np.linalg.norm(f[free]))


def solve(c, u0=None, quad=0, method="direct", K=None, f=None, tol=1e-14, maxiter=200000):
    """lambda (all nodes, 0 at fixed nodes) solving K_FF lambda_F = f_F."""
    free = case_free_mask(c)
    if K is None:
        K = assemble_K(c)
    if f is None:
        f = assemble_f(c, u0=u0, quad=quad)
    Kff = K[free][:, free].tocsc()
    ff = f[free]
    lam = np.zeros(c.n_nodes)
    if method == "direct":
        lam[free] = spla.spsolve(Kff, ff)
    else:
        lam[free] = cg(Kff.tocsr(), ff, tol=tol, maxiter=maxiter)
    return lam


def cg(A, b, tol=1e-14, maxiter=200000, x0=None):
    """Jacobi-preconditioned conjugate gradients, restarted from the true
    residual until ||b - A x|| <= tol ||b||."""
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x
    it = 0
    while it < maxiter:
        r = b - A @ x
        if np.linalg.norm(r) <= tol * nb:
            break
        z = dinv * r
        p = z.copy()
        rz = r @ z
        for _ in range(2000):
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x += alpha * p
            r -= alpha * Ap
            it += 1
            if np.linalg.norm(r) <= 0.1 * tol * nb:
                break
            z = dinv * r
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
    return x


def recover(c, lam, u0=None, where=0, a=None):
    """u = u0 + A^{-1} grad lambda (Eq. 3) at element centers (where=0,
    shape (3, nz, ny, nx)) or at the 8 Gauss points (where=1,
    shape (3, 8, nz, ny, nx))."""
    a = _f64(c.a if a is None else a)
    u0 = _f64(c.u0 if u0 is None else u0)
    ng = 1 if where == 0 else 8
    u = np.zeros((3, ng, c.nz, c.ny, c.nx))
    _check(lib().oracle_recover(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)), _p(_f64(c.Z)),
                                _p(u0), _p(_f64(lam).ravel()), _p(a), where, _p(u)))
    return u[:, 0] if where == 0 else u


def weak_div(c, ug):
    """(B u)_m = sum_g detJ grad N_m(g) . u(g) at every node; ug (3, 8, nz, ny, nx)."""
    out = np.zeros(c.n_nodes)
    _check(lib().oracle_weak_div(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)), _p(_f64(c.Z)),
                                 _p(_f64(ug)), _p(out)))
    return out


def gauss_detj(c):
    out = np.zeros((8, c.nz, c.ny, c.nx))
    _check(lib().oracle_gauss_detj(c.nx, c.ny, c.nz, _p(_f64(c.X)), _p(_f64(c.Y)),
                                   _p(_f64(c.Z)), _p(out)))
    return out


def interp_gauss(c, u0=None):
    u0 = _f64(c.u0 if u0 is None else u0)
    out = np.zeros((3, 8, c.nz, c.ny, c.nx))
    _check(lib().oracle_interp_gauss(c.nx, c.ny, c.nz, _p(u0), _p(out)))
    return out


def kkt_dense(c, u0=None):
    """Brute-force minimization of the discrete form of Eq. 1:
    min 1/2 (u - u0)^T M (u - u0)  subject to  B_F u = 0,
    u at the Gauss points, M = blockdiag(detJ_g A), B the discrete weak
    divergence restricted to the free nodes.  Stationarity of the
    Lagrangian (Eq. 2) gives the dense system
        [[M, -B_F^T], [B_F, 0]] [u; lambda_F] = [M u0; 0].
    Returns (lambda on all nodes, u at the Gauss points).  Tiny grids only."""
    u0 = c.u0 if u0 is None else u0
    ne = c.nx * c.ny * c.nz
    nu = 3 * 8 * ne
    free = case_free_mask(c)
    # B column by column: apply the weak divergence to unit Gauss-point fields
    B = np.zeros((c.n_nodes, nu))
    e = np.zeros(nu)
    for q in range(nu):
        e[:] = 0.0
        e[q] = 1.0
        B[:, q] = weak_div(c, e.reshape(3, 8, c.nz, c.ny, c.nx))
    Bf = B[free]
    detj = gauss_detj(c).ravel()
    a2 = np.asarray(c.a, dtype=np.float64) ** 2
    Mdiag = np.concatenate([detj * a2[d] for d in range(3)])
    ug0 = interp_gauss(c, u0).ravel()
    nf = int(free.sum())
    S = np.zeros((nu + nf, nu + nf))
    S[:nu, :nu] = np.diag(Mdiag)
    S[:nu, nu:] = -Bf.T
    S[nu:, :nu] = Bf
    rhs = np.concatenate([Mdiag * ug0, np.zeros(nf)])
    sol = scipy.linalg.solve(S, rhs)
    lam = np.zeros(c.n_nodes)
    lam[free] = sol[nu:]
    return lam, sol[:nu].reshape(3, 8, c.nz, c.ny, c.nx)


# --------------------------------------------------------------------------
# multigrid (Sec. 3)

def plan_levels(nx, ny, nz, h1, h3, a, rule="paper", coarsest_max=1024, max_levels=40):
    """Grid hierarchy by the adaptive semicoarsening rule of Sec. 3.

    With ratio(h3) = h3 / (h1 a3) ("paper") or a3 h3 / (a1 h1) ("operator"):
    coarsen both horizontal directions by 2 when ratio(bottom layer) > 1/3;
    then, with h1 doubled if it was coarsened, go up from the ground and merge
    a layer with the one above it when ratio(layer) < 3, else keep it.
    A coarse direction keeps the even-index nodes plus the last node.
    Stop when the coarse problem has at most coarsest_max free nodes.  If the
    rule coarsens nothing while the level is still too large, coarsen
    horizontally anyway (or stop when that is impossible).

    Returns a list of dicts with cells (cx, cy, cz), node dims (Nx, Ny, Nz),
    and for every level but the last the transfer to the next one:
    hx, hy (horizontal coarsening flags) and kmap (coarse node k -> fine k).
    """
    a1, a3 = float(a[0]), float(a[2])

    def ratio(t, h):
        return t / (h * a3) if rule == "paper" else a3 * t / (a1 * h)

    levels = []
    cx, cy, cz, hh, layers = nx, ny, nz, float(h1), [float(t) for t in h3]
    while True:
        lev = dict(cx=cx, cy=cy, cz=cz, Nx=cx + 1, Ny=cy + 1, Nz=cz + 1,
                   n_free=(cx - 1) * (cy - 1) * cz)
        levels.append(lev)
        if lev["n_free"] <= coarsest_max or len(levels) >= max_levels:
            break
        horiz = ratio(layers[0], hh) > 1.0 / 3.0
        hx = horiz and cx >= 3
        hy = horiz and cy >= 3
        h_new = 2.0 * hh if (hx or hy) else hh
        kmap, new_layers, l = [0], [], 0
        while l < len(layers):
            if l + 1 < len(layers) and ratio(layers[l], h_new) < 3.0:
                new_layers.append(layers[l] + layers[l + 1])
                l += 2
            else:
                new_layers.append(layers[l])
                l += 1
            kmap.append(l)
        if not (hx or hy) and len(new_layers) == len(layers):
            hx, hy = cx >= 3, cy >= 3
            if not (hx or hy):
                break
            h_new = 2.0 * hh
        lev.update(hx=hx, hy=hy, kmap=kmap)
        cx = (cx + 1) // 2 if hx else cx
        cy = (cy + 1) // 2 if hy else cy
        cz = len(new_layers)
        hh, layers = h_new, new_layers
    return levels


def _p1d_horizontal(Nf, coarsen):
    """1-D prolongation for one horizontal direction (Sec. 3: the coarse
    nodes interpolate to the fine nodes of each pair of fine intervals with
    the weights of linear interpolation on a regular grid)."""
    if not coarsen:
        return sp.identity(Nf, format="csr")
    cmap = list(range(0, Nf - 1, 2)) + [Nf - 1]
    return _p1d_from_map(Nf, cmap)


def _p1d_from_map(Nf, cmap):
    Nc = len(cmap)
    P = sp.lil_matrix((Nf, Nc))
    pos = {f: I for I, f in enumerate(cmap)}
    for f in range(Nf):
        if f in pos:
            P[f, pos[f]] = 1.0
        else:
            I = max(I for I, g in enumerate(cmap) if g < f)
            assert cmap[I + 1] == f + 1 and cmap[I] == f - 1
            P[f, I] = 0.5
            P[f, I + 1] = 0.5
    return P.tocsr()


def prolongation(fine, coarse):
    """P (fine nodes x coarse nodes), node id (k*Ny + j)*Nx + i: the tensor
    product of the 1-D trilinear index-space weights (Sec. 3)."""
    Px = _p1d_horizontal(fine["Nx"], fine["hx"])
    Py = _p1d_horizontal(fine["Ny"], fine["hy"])
    Pz = _p1d_from_map(fine["Nz"], fine["kmap"])
    assert Px.shape[1] == coarse["Nx"] and Py.shape[1] == coarse["Ny"]
    assert Pz.shape[1] == coarse["Nz"]
    return sp.kron(Pz, sp.kron(Py, Px)).tocsr()


def galerkin(K, P):
    """K_c = P^T K P (Eq. 7, second row)."""
    return (P.T @ K @ P).tocsr()


def gs_sweep(K, f, x, dims, direction=0):
    """One smoothing sweep in place (see oracle_gs_sweep in fe_oracle.c)."""
    Nx, Ny, Nz = dims
    K = K.tocsr()
    K.sort_indices()
    indptr = np.ascontiguousarray(K.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(K.indices, dtype=np.int64)
    data = _f64(K.data)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    lib().oracle_gs_sweep(Nx, Ny, Nz, _p(indptr, ctypes.c_int64), _p(indices, ctypes.c_int64),
                          _p(data), _p(_f64(f)), _p(x), direction)
    return x


class Hierarchy:
    """The operators of every level: K_0 = K_FF (embedded), K_{l+1} = P^T K_l P
    with the fixed nodes' rows and columns dropped, and the coarsest free
    block factored by dense Cholesky (Sec. 3: a direct method on the coarsest
    grid)."""

    def __init__(self, c, rule="paper", coarsest_max=1024, K=None, a=None):
        a = c.a if a is None else a
        self.levels = plan_levels(c.nx, c.ny, c.nz, c.h1, c.h3, a, rule, coarsest_max)
        K = assemble_K(c, a) if K is None else K
        self.free = []
        self.K = []
        self.P = []
        for li, lev in enumerate(self.levels):
            free = free_mask(lev["Nx"], lev["Ny"], lev["Nz"])
            self.free.append(free)
            if li == 0:
                self.K.append(restrict_free(K, free))
            else:
                P = prolongation(self.levels[li - 1], lev)
                self.P.append(P)
                self.K.append(restrict_free(galerkin(self.K[-1], P), free))
        last = self.K[-1]
        fl = self.free[-1]
        Kc = last[fl][:, fl].toarray()
        self.coarse_chol = scipy.linalg.cho_factor(Kc, lower=True)

    def dims(self, li):
        lev = self.levels[li]
        return lev["Nx"], lev["Ny"], lev["Nz"]

    def coarse_solve(self, fc):
        x = np.zeros_like(fc)
        fl = self.free[-1]
        x[fl] = scipy.linalg.cho_solve(self.coarse_chol, fc[fl])
        return x

    def vcycle(self, li, f, x, nu1=2, nu2=2):
        """One V-cycle on level li (Sec. 3, Eq. 6-7): nu1 forward sweeps,
        f_c = P^T (f - K x), recursive coarse solve from zero, x += P x_c,
        nu2 reverse sweeps.  The coarsest level is solved directly."""
        if li == len(self.levels) - 1:
            return self.coarse_solve(f)
        K = self.K[li]
        d = self.dims(li)
        for _ in range(nu1):
            gs_sweep(K, f, x, d, 0)
        r = f - K @ x
        r[~self.free[li]] = 0.0
        P = self.P[li]
        fc = P.T @ r
        xc = self.vcycle(li + 1, fc, np.zeros(P.shape[1]), nu1, nu2)
        x += P @ xc
        for _ in range(nu2):
            gs_sweep(K, f, x, d, 1)
        return x

    def solve(self, f, x0=None, rtol=1e-8, max_cycles=100, nu1=2, nu2=2):
        """V-cycles until ||f_F - K_FF x_F|| <= rtol ||f_F||.  Returns x and
        the relative residual history (entry 0 before the first cycle)."""
        free = self.free[0]
        f = f.copy()
        f[~free] = 0.0
        x = np.zeros_like(f) if x0 is None else x0.copy()
        x[~free] = 0.0
        nf = np.linalg.norm(f)
        hist = [np.linalg.norm(f - self.K[0] @ x) / nf]
        for _ in range(max_cycles):
            if hist[-1] <= rtol:
                break
            x = self.vcycle(0, f, x, nu1, nu2)
            hist.append(np.linalg.norm(f - self.K[0] @ x) / nf)
        return x, hist


# --------------------------------------------------------------------------
# derivatives of the recovered wind (brute force, tiny grids)

def dense_wind_gradient(c, gu, a=None, h_loga=1e-6):
    """Gradient of l(u) with dl/du = gu (u at the element centers, Eq. 3 with
    lambda from Eq. 5), by dense linear algebra on matrices probed from the
    oracle's own maps with unit vectors:
        du/du0 = R_u0 + R_lam[:, F] K_FF^{-1} J_f[F, :],
    R_u0 = du/du0 at fixed lambda, R_lam = du/dlambda, J_f = df/du0.
    dl/dlog a_d by central differences (step h_loga) of l = gu . u(a) through
    the oracle's forward map.  Returns (dl/du0 shaped like u0, [3])."""
    a = np.asarray(c.a if a is None else a, dtype=np.float64)
    N = c.n_nodes
    free = case_free_mask(c)
    gu = np.asarray(gu, dtype=np.float64).ravel()
    zero_l = np.zeros(N)
    zero_u = np.zeros((3,) + c.u0.shape[1:])
    R_u0 = np.zeros((gu.size, 3 * N))
    J_f = np.zeros((N, 3 * N))
    e = np.zeros(3 * N)
    for q in range(3 * N):
        e[:] = 0.0
        e[q] = 1.0
        uq = e.reshape(c.u0.shape)
        R_u0[:, q] = recover(c, zero_l, u0=uq, a=a).ravel()
        J_f[:, q] = assemble_f(c, u0=uq)
    fidx = np.flatnonzero(free)
    R_l = np.zeros((gu.size, fidx.size))
    el = np.zeros(N)
    for col, q in enumerate(fidx):
        el[:] = 0.0
        el[q] = 1.0
        R_l[:, col] = recover(c, el, u0=zero_u, a=a).ravel()
    K = assemble_K(c, a).toarray()[np.ix_(free, free)]
    dudu0 = R_u0 + R_l @ np.linalg.solve(K, J_f[free])
    g_u0 = (dudu0.T @ gu).reshape(c.u0.shape)

    def loss(av):
        lam = solve(c, K=assemble_K(c, av))
        return float(gu @ recover(c, lam, a=av).ravel())

    g_loga = []
    for d in range(3):
        ap, am = a.copy(), a.copy()
        ap[d] *= np.exp(h_loga)
        am[d] *= np.exp(-h_loga)
        g_loga.append((loss(ap) - loss(am)) / (2.0 * h_loga))
    return g_u0, g_loga
