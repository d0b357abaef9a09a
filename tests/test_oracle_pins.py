"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each compares it with an
independent closed form, invariant, textbook value or brute-force problem
(Sec. 2 and Sec. 3 of the paper; Eq. 1-7)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def q1_1d(z):
    """1-D linear-element stiffness and mass matrices on nodes z (assembled)."""
    n = len(z)
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    G = np.zeros((n, n))   # G[i][j] = int phi_i' phi_j
    for e in range(n - 1):
        h = z[e + 1] - z[e]
        idx = [e, e + 1]
        K[np.ix_(idx, idx)] += np.array([[1, -1], [-1, 1]]) / h
        M[np.ix_(idx, idx)] += np.array([[2, 1], [1, 2]]) * h / 6.0
        G[np.ix_(idx, idx)] += np.array([[-1, -1], [1, 1]]) / 2.0
    return K, M, G


def box_case(nx, ny, nz, seed=0):
    rng = np.random.default_rng(seed)
    x = np.concatenate([[0], np.cumsum(rng.uniform(10, 40, nx))])
    y = np.concatenate([[0], np.cumsum(rng.uniform(10, 40, ny))])
    z = np.concatenate([[0], np.cumsum(rng.uniform(2, 20, nz))])
    shape = (nz + 1, ny + 1, nx + 1)
    X = np.broadcast_to(x[None, None, :], shape).copy()
    Y = np.broadcast_to(y[None, :, None], shape).copy()
    Z = np.broadcast_to(z[:, None, None], shape).copy()
    a = tuple(rng.uniform(0.5, 3.0, 3))
    u0 = rng.normal(size=(3,) + shape)
    c = synth.Case("box", nx, ny, nz, a, X, Y, Z, u0, 30.0, np.diff(z))
    return c, x, y, z


# ---------------------------------------------------------------- P1, P2, P3

def test_p1_box_element_kronecker():
    rng = np.random.default_rng(1)
    h = rng.uniform(1, 50, 3)
    a = rng.uniform(0.5, 4, 3)
    o = rng.uniform(-1e4, 1e4, 3)
    xe = np.array([[o[0] + (n & 1) * h[0], o[1] + ((n >> 1) & 1) * h[1],
                    o[2] + ((n >> 2) & 1) * h[2]] for n in range(8)])
    k = [np.array([[1, -1], [-1, 1]]) / hd for hd in h]
    m = [np.array([[2, 1], [1, 2]]) * hd / 6 for hd in h]
    # local node n = a + 2b + 4c: kron order (z, y, x)
    Kref = (np.kron(m[2], np.kron(m[1], k[0])) / a[0] ** 2
            + np.kron(m[2], np.kron(k[1], m[0])) / a[1] ** 2
            + np.kron(k[2], np.kron(m[1], m[0])) / a[2] ** 2)
    Ke = oracle.element_stiffness(xe, a)
    assert np.allclose(Ke, Kref, rtol=1e-13, atol=1e-13 * np.abs(Kref).max())


def test_p2_uniform_cube_stencil():
    g = json.load(open(os.path.join(GOLD, "stencil_q1_cube.json")))
    h = 7.0
    c = synth.flat_box(4, 4, 4, dx=h, dz=h, stretch=1.0)
    row = oracle.stencil_row(c, 2, 2, 2).reshape(3, 3, 3)  # [dk][dj][di]
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                nnz = abs(di) + abs(dj) + abs(dk)
                want = {0: g["center"], 1: g["face"], 2: g["edge"], 3: g["corner"]}[nnz] * h
                assert row[dk + 1, dj + 1, di + 1] == pytest.approx(want, abs=1e-12 * h)


def test_p3_global_kronecker_sum():
    c, x, y, z = box_case(5, 4, 3, seed=2)
    Kx, Mx, _ = q1_1d(x)
    Ky, My, _ = q1_1d(y)
    Kz, Mz, _ = q1_1d(z)
    a = np.asarray(c.a)
    Kref = (np.kron(Mz, np.kron(My, Kx)) / a[0] ** 2 + np.kron(Mz, np.kron(Ky, Mx)) / a[1] ** 2
            + np.kron(Kz, np.kron(My, Mx)) / a[2] ** 2)
    K = oracle.assemble_K(c).toarray()
    assert np.abs(K - Kref).max() <= 1e-12 * np.abs(Kref).max()


def test_rhs_box_kronecker():
    """f = -int grad mu . u0 with nodal trilinear u0 is integrated exactly by
    2x2x2 Gauss on box grids: f = -(Mz My Gx ux + Mz Gy Mx uy + Gz My Mx uz)."""
    c, x, y, z = box_case(4, 5, 3, seed=3)
    _, Mx, Gx = q1_1d(x)
    _, My, Gy = q1_1d(y)
    _, Mz, Gz = q1_1d(z)
    u = c.u0.reshape(3, -1)
    fref = -(np.kron(Mz, np.kron(My, Gx)) @ u[0] + np.kron(Mz, np.kron(Gy, Mx)) @ u[1]
             + np.kron(Gz, np.kron(My, Mx)) @ u[2])
    f = oracle.assemble_f(c)
    assert np.abs(f - fref).max() <= 1e-12 * np.abs(fref).max()


def test_rhs_vertical_wind_closed_form():
    """Constant vertical wind W over flat ground: by the divergence theorem
    f_i = -W int dphi_i/dz = W * (area of phi_i on the ground) at ground
    nodes and 0 at interior free nodes (the sign of Eq. 5's right side)."""
    W, h = 3.0, 20.0
    c = synth.flat_box(4, 5, 3, dx=h, dz=6.0, stretch=1.3)
    c.u0[2] = W
    f = oracle.assemble_f(c).reshape(c.nz + 1, c.ny + 1, c.nx + 1)
    assert np.allclose(f[0, 1:-1, 1:-1], W * h * h, rtol=1e-13)
    assert np.abs(f[1:-1, 1:-1, 1:-1]).max() <= 1e-12 * W * h * h
    # one-point center rule is exact for a constant wind on box elements
    fc = oracle.assemble_f(c, quad=1).reshape(f.shape)
    assert np.allclose(fc, f, rtol=1e-13, atol=1e-12 * W * h * h)


# ---------------------------------------------------------------- P4

@pytest.mark.parametrize("maker", [
    lambda: synth.single_hill(6, 5, 3, sigma=50.0, height=40.0),
    lambda: synth.jittered(5, 4, 3, seed=4),
])
def test_p4_symmetric_spd_zero_rowsum(maker):
    c = maker()
    K = oracle.assemble_K(c)
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-13 * np.abs(Kd).max()
    assert np.abs(Kd.sum(axis=1)).max() <= 1e-12 * np.abs(Kd).max()
    free = oracle.case_free_mask(c)
    Kff = Kd[np.ix_(free, free)]
    np.linalg.cholesky(Kff)
    assert np.linalg.eigvalsh(Kff).min() > 0


def test_patch_linear_lambda_deformed_grid():
    """Isoparametric Q1 reproduces linear functions: for lambda = g.x,
    (K lambda)_i = A^{-1} g . int grad phi_i = 0 at nodes off the boundary,
    and the recovered gradient is exactly g (Eq. 3)."""
    c = synth.jittered(5, 5, 4, seed=5, a=(1.0, 2.0, 0.5))
    g = np.array([0.3, -1.1, 2.0])
    lam = g[0] * c.X + g[1] * c.Y + g[2] * c.Z
    y = (oracle.assemble_K(c) @ lam.ravel()).reshape(lam.shape)
    assert np.abs(y[1:-1, 1:-1, 1:-1]).max() <= 1e-12 * np.abs(lam).max()
    for where in (0, 1):
        u = oracle.recover(c, lam, u0=np.zeros_like(c.u0), where=where)
        for d in range(3):
            assert np.allclose(u[d], g[d] / c.a[d] ** 2, rtol=1e-11, atol=1e-12)
    # a constant wind has zero load at interior nodes on any grid
    u0 = np.zeros_like(c.u0)
    u0[0], u0[1], u0[2] = 1.5, -0.5, 0.25
    f = oracle.assemble_f(c, u0=u0).reshape(lam.shape)
    assert np.abs(f[1:-1, 1:-1, 1:-1]).max() <= 1e-12


# ---------------------------------------------------------------- P5, P6, P7, P8, P9

def test_p5_uniform_horizontal_wind_flat_ground():
    c = synth.flat_box(6, 5, 4, stretch=1.2)
    c.u0[0], c.u0[1], c.u0[2] = 4.0, -2.5, 0.0
    f = oracle.assemble_f(c)
    free = oracle.case_free_mask(c)
    assert np.abs(f[free]).max() <= 1e-12 * 4.0 * 30 * 30
    lam = oracle.solve(c, f=f)
    assert np.abs(lam).max() <= 1e-10
    u = oracle.recover(c, lam)
    assert np.allclose(u[0], 4.0) and np.allclose(u[1], -2.5) and np.allclose(u[2], 0.0, atol=1e-12)


def test_p6_weak_divergence_vanishes():
    c = synth.single_hill(12, 10, 4, sigma=80.0, height=60.0, noise=0.5)
    lam = oracle.solve(c)
    ug = oracle.recover(c, lam, where=1)
    bu = oracle.weak_div(c, ug)
    bu0 = oracle.weak_div(c, oracle.interp_gauss(c))
    free = oracle.case_free_mask(c)
    assert np.linalg.norm(bu[free]) <= 1e-11 * np.linalg.norm(bu0[free])
    # and -B u0 is the load vector of Eq. 5
    assert np.allclose(-bu0, oracle.assemble_f(c), rtol=1e-12, atol=1e-12 * np.abs(bu0).max())


@pytest.mark.parametrize("dims,maker", [
    ((2, 2, 2), "hill"), ((3, 3, 2), "hill"), ((4, 3, 3), "hill"), ((3, 3, 3), "jit"),
])
def test_p7_dense_kkt_brute_force(dims, maker):
    nx, ny, nz = dims
    if maker == "hill":
        c = synth.single_hill(nx, ny, nz, sigma=30.0, height=25.0, noise=1.0, a=(1.0, 1.5, 3.0))
    else:
        c = synth.jittered(nx, ny, nz, seed=7, a=(2.0, 1.0, 0.7))
    lam_kkt, ug_kkt = oracle.kkt_dense(c)
    lam = oracle.solve(c)
    assert np.linalg.norm(lam - lam_kkt) <= 1e-10 * np.linalg.norm(lam_kkt)
    ug = oracle.recover(c, lam, where=1)
    assert np.linalg.norm(ug - ug_kkt) <= 1e-10 * np.linalg.norm(ug_kkt)


def test_p8_scaling_of_penalty_constants():
    c = synth.single_hill(8, 7, 4, sigma=60.0, height=50.0, a=(1.0, 1.0, 2.0))
    lam1 = oracle.solve(c)
    u1 = oracle.recover(c, lam1)
    s = 3.0
    K = oracle.assemble_K(c, a=tuple(s * np.asarray(c.a)))
    lam2 = oracle.solve(c, K=K)
    u2 = oracle.recover(c, lam2, a=tuple(s * np.asarray(c.a)))
    assert np.allclose(lam2, s * s * lam1, rtol=1e-10, atol=1e-12 * np.abs(lam2).max())
    assert np.allclose(u2, u1, rtol=1e-10, atol=1e-10)


def test_p9_manufactured_solution():
    c = synth.jittered(6, 5, 4, seed=9)
    rng = np.random.default_rng(9)
    free = oracle.case_free_mask(c)
    lam_star = np.where(free, rng.normal(size=c.n_nodes), 0.0)
    K = oracle.assemble_K(c)
    f = K @ lam_star
    for method in ("direct", "cg"):
        lam = oracle.solve(c, K=K, f=f, method=method)
        assert np.linalg.norm(lam - lam_star) <= 1e-9 * np.linalg.norm(lam_star)


def test_apply_K_matches_assembled():
    c = synth.jittered(7, 6, 5, seed=11)
    x = np.random.default_rng(3).normal(size=c.n_nodes)
    y1 = oracle.assemble_K(c) @ x
    y2 = oracle.apply_K(c, x)
    assert np.allclose(y1, y2, rtol=1e-12, atol=1e-12 * np.abs(y1).max())
    for (i, j, k) in [(0, 0, 0), (3, 2, 1), (7, 6, 5), (1, 5, 0)]:
        row = oracle.stencil_row(c, i, j, k)
        Kd = oracle.assemble_K(c)
        for s in range(27):
            di, dj, dk = s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1
            ii, jj, kk = i + di, j + dj, k + dk
            if 0 <= ii <= c.nx and 0 <= jj <= c.ny and 0 <= kk <= c.nz:
                r = (k * (c.ny + 1) + j) * (c.nx + 1) + i
                q = (kk * (c.ny + 1) + jj) * (c.nx + 1) + ii
                assert row[s] == pytest.approx(Kd[r, q], abs=1e-12 * abs(Kd[r, r]))
            else:
                assert row[s] == 0.0


def test_rhs_parallel_equals_serial():
    c = synth.single_hill(9, 8, 5, sigma=70.0, height=40.0)
    f1 = oracle.assemble_f(c)
    f2 = oracle.assemble_f(c, parallel=True)
    assert np.allclose(f1, f2, rtol=1e-13, atol=1e-13 * np.abs(f1).max())


# ---------------------------------------------------------------- multigrid pins

def test_plan_hill64_matches_hand_derivation():
    g = json.load(open(os.path.join(GOLD, "plan_hill64.json")))
    c = synth.single_hill()
    lv = oracle.plan_levels(c.nx, c.ny, c.nz, c.h1, c.h3, c.a, "paper", 1024)
    assert len(lv) == len(g["levels"])
    for got, want in zip(lv, g["levels"]):
        for key in want:
            assert got[key] == want[key], (key, got, want)


def _aniso64_levels(rule, a=None):
    g = json.load(open(os.path.join(GOLD, "plan_aniso64.json")))
    c = g["case"]
    h3 = [c["h3_first"] * c["h3_growth"] ** k for k in range(c["nz"])]
    a = c["a"] if a is None else a
    return g, oracle.plan_levels(c["nx"], c["ny"], c["nz"], c["h1"], h3, a, rule,
                                 c["coarsest_max"])


def _same_levels(got, want):
    return len(got) == len(want) and all(
        all(gl.get(key) == wl[key] for key in wl) for gl, wl in zip(got, want))


@pytest.mark.parametrize("rule", ["paper", "operator"])
def test_plan_aniso64_matches_hand_derivation(rule):
    """Both readings of the semicoarsening ratio of Sec. 3 against a
    hierarchy derived by hand where they disagree (a1 != 1, a3 = 10): the
    operator reading merges layers one by one above the ground."""
    g, lv = _aniso64_levels(rule)
    assert _same_levels(lv, g["levels_" + rule]), (lv, g["levels_" + rule])


@pytest.mark.parametrize("rule,mutated", [
    ("paper", (0.5, 1.0, 1.0)),        # a3 dropped
    ("paper", (10.0, 1.0, 0.5)),       # a1 and a3 swapped
    ("operator", (1.0, 1.0, 10.0)),    # a1 dropped
    ("operator", (0.5, 1.0, 1.0)),     # a3 dropped
    ("operator", (10.0, 1.0, 0.5)),    # a1 and a3 swapped
])
def test_plan_aniso64_detects_penalty_slips(rule, mutated):
    """The fixture fixes how a1 and a3 enter each ratio: planning with a
    penalty vector that a dropped or swapped constant would produce gives a
    different hierarchy, so such a slip in the planner cannot pass."""
    g, lv = _aniso64_levels(rule, mutated)
    assert not _same_levels(lv, g["levels_" + rule])


def test_p10_galerkin_nested_uniform_grid():
    """On a uniform box grid with full 2x coarsening the coarse space is the
    Q1 space of the 2h grid, so P^T K P is the 2h stiffness (Sec. 3)."""
    h = 10.0
    fine = synth.flat_box(8, 6, 4, dx=h, dz=h, stretch=1.0, a=(1.0, 1.3, 0.8))
    coarse = synth.flat_box(4, 3, 2, dx=2 * h, dz=2 * h, stretch=1.0, a=(1.0, 1.3, 0.8))
    lf = dict(Nx=9, Ny=7, Nz=5, hx=True, hy=True, kmap=[0, 2, 4])
    lc = dict(Nx=5, Ny=4, Nz=3)
    P = oracle.prolongation(lf, lc)
    Kc = oracle.galerkin(oracle.assemble_K(fine), P).toarray()
    Kc_ref = oracle.assemble_K(coarse).toarray()
    assert np.abs(Kc - Kc_ref).max() <= 1e-12 * np.abs(Kc_ref).max()


def test_prolongation_reproduces_index_linear():
    """P maps the coarse samples of a function linear in the grid indices to
    its fine samples (the trilinear weights of Sec. 3), including an odd
    cell count whose last coarse interval spans one fine cell."""
    lf = dict(Nx=8, Ny=6, Nz=6, hx=True, hy=False, kmap=[0, 2, 3, 5])
    cmap_x = [0, 2, 4, 6, 7]
    lc = dict(Nx=5, Ny=6, Nz=4)
    P = oracle.prolongation(lf, lc)
    k, j, i = np.meshgrid(np.arange(6), np.arange(6), np.arange(8), indexing="ij")
    fine = 0.7 * i - 1.3 * j + 2.1 * k + 0.4
    kk, jj, ii = np.meshgrid(np.array([0, 2, 3, 5]), np.arange(6), np.array(cmap_x), indexing="ij")
    coarse = 0.7 * ii - 1.3 * jj + 2.1 * kk + 0.4
    assert np.allclose(P @ coarse.ravel(), fine.ravel(), rtol=1e-14, atol=1e-13)
    assert np.allclose(P.sum(axis=1), 1.0)


def _gs_order(Nx, Ny, Nz, direction):
    order = []
    for gi in range(4):
        g = gi if direction == 0 else 3 - gi
        pi, pj = g & 1, g >> 1
        for j in range(1, Ny - 1):
            for i in range(1, Nx - 1):
                if (i & 1) != pi or (j & 1) != pj:
                    continue
                ks = range(Nz - 1) if direction == 0 else range(Nz - 2, -1, -1)
                for k in ks:
                    order.append((k * Ny + j) * Nx + i)
    return np.array(order)


@pytest.mark.parametrize("direction", [0, 1])
def test_gs_sweep_is_triangular_splitting(direction):
    """One sweep equals x <- (D + L)^{-1} (f - U x) with L, U the strict
    lower/upper parts of K_FF in the update order (the matrix form of
    Gauss-Seidel), solved here by a sparse triangular solve."""
    c = synth.single_hill(7, 6, 4, sigma=50.0, height=30.0)
    K = oracle.restrict_free(oracle.assemble_K(c), oracle.case_free_mask(c))
    dims = (c.nx + 1, c.ny + 1, c.nz + 1)
    rng = np.random.default_rng(direction)
    free = oracle.case_free_mask(c)
    x0 = np.where(free, rng.normal(size=c.n_nodes), 0.0)
    f = np.where(free, rng.normal(size=c.n_nodes), 0.0)
    x = oracle.gs_sweep(K, f, x0.copy(), dims, direction)
    order = _gs_order(*dims, direction)
    Kp = K[order][:, order].tocsr()
    low = sp.tril(Kp, k=0).tocsr()
    up = sp.triu(Kp, k=1).tocsr()
    xp = spla.spsolve_triangular(low, f[order] - up @ x0[order], lower=True)
    assert np.allclose(x[order], xp, rtol=1e-12, atol=1e-12 * np.abs(xp).max())
    assert np.all(x[~free] == 0.0)


def test_vcycle_converges_at_paper_rate():
    g = json.load(open(os.path.join(GOLD, "paper_rates.json")))
    c = synth.single_hill()
    H = oracle.Hierarchy(c)
    f = oracle.assemble_f(c)
    x, hist = H.solve(f, rtol=1e-10, max_cycles=60)
    rates = np.array(hist[1:]) / np.array(hist[:-1])
    assert hist[-1] <= 1e-10
    assert np.exp(np.mean(np.log(rates[2:]))) <= g["semicoarsening_rate_max"]
    lam = oracle.solve(c, f=f)
    assert np.linalg.norm(x - lam) <= 1e-8 * np.linalg.norm(lam)


def test_vcycle_is_symmetric_operator():
    """With reverse-order post-smoothing the V-cycle is a symmetric linear
    map of the right-hand side (from a zero start)."""
    c = synth.single_hill(10, 9, 4, sigma=60.0, height=30.0)
    H = oracle.Hierarchy(c, coarsest_max=20)
    assert len(H.levels) >= 2
    free = H.free[0]
    rng = np.random.default_rng(0)
    f1 = np.where(free, rng.normal(size=c.n_nodes), 0.0)
    f2 = np.where(free, rng.normal(size=c.n_nodes), 0.0)
    b1 = H.vcycle(0, f1, np.zeros_like(f1))
    b2 = H.vcycle(0, f2, np.zeros_like(f2))
    assert abs(f2 @ b1 - f1 @ b2) <= 1e-12 * abs(f2 @ b1)


def test_dense_wind_gradient_against_finite_differences():
    """The probed-Jacobian gradient agrees with central differences of the
    oracle's forward map, and the log-a derivatives sum to zero (a -> c a
    leaves u unchanged, Sec. 2 / P8)."""
    c = synth.single_hill(5, 4, 3, sigma=40.0, height=20.0, noise=0.5, a=(1.0, 1.3, 2.0))
    rng = np.random.default_rng(0)
    gu = rng.normal(size=(3, c.nz, c.ny, c.nx))
    g0, gl = oracle.dense_wind_gradient(c, gu)

    def loss(u0):
        lam = oracle.solve(c, u0=u0)
        return float(gu.ravel() @ oracle.recover(c, lam, u0=u0).ravel())

    for idx in [(0, 0, 0, 0), (1, 2, 2, 3), (2, 3, 4, 5), (0, 1, 3, 1)]:
        up, um = c.u0.copy(), c.u0.copy()
        up[idx] += 1e-6
        um[idx] -= 1e-6
        fd = (loss(up) - loss(um)) / 2e-6
        assert fd == pytest.approx(g0[idx], rel=1e-6, abs=1e-8)
    assert abs(sum(gl)) <= 1e-6 * max(abs(v) for v in gl)


def test_center_wind_load_vector():
    """A wind given at the element centers (Sec. 2's representation) that is
    constant gives the same load vector as the same constant at the nodes;
    a center wind that varies gives the nodal result of its mean per element
    for the one-point rule."""
    c = synth.jittered(5, 4, 3, seed=8)
    uc = np.zeros((3, c.nz, c.ny, c.nx))
    uc[0], uc[1], uc[2] = 1.5, -0.7, 0.3
    c.u0[0], c.u0[1], c.u0[2] = 1.5, -0.7, 0.3
    for quad in (0, 1):
        a = oracle.assemble_f_centers(c, uc, quad)
        b = oracle.assemble_f(c, quad=quad)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    rng = np.random.default_rng(2)
    u0 = rng.normal(size=c.u0.shape)
    mean = np.zeros_like(uc)
    for n in range(8):
        mean += u0[:, (n >> 2) & 1: c.nz + ((n >> 2) & 1), (n >> 1) & 1: c.ny + ((n >> 1) & 1),
                   n & 1: c.nx + (n & 1)] / 8.0
    a = oracle.assemble_f_centers(c, mean, 1)
    b = oracle.assemble_f(c, u0=u0, quad=1)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def _column_factors(c):
    """Horizontal factors of a shift-form grid, assembled over the node
    columns from the ground layer by 2 x 2 Gauss points per cell (weight 1):
    P_ab = sum grad phi_a . W grad phi_b, Q_ab = sum grad phi_a . W z' phi_b,
    R_ab = sum (z' . W z' + j2 / a3^2) phi_a phi_b, with J2 the horizontal
    Jacobian, j2 = det J2, W = adj(J2) diag(a1^-2, a2^-2) adj(J2)^T / j2 and
    z' the terrain slope, all in the reference coordinates (Sec. 2)."""
    nx, ny = c.nx, c.ny
    c1, c2, c3 = (np.asarray(c.a, dtype=float) ** -2)
    ncol = (nx + 1) * (ny + 1)
    P, Q, R = (np.zeros((ncol, ncol)) for _ in range(3))
    sx = np.array([-1.0, 1.0, -1.0, 1.0])
    sy = np.array([-1.0, -1.0, 1.0, 1.0])
    gp = 1.0 / np.sqrt(3.0)
    for cj in range(ny):
        for ci in range(nx):
            idx = [(cj + (p >> 1)) * (nx + 1) + ci + (p & 1) for p in range(4)]
            xs, ys, zs = (np.array([A[0].flat[n] for n in idx]) for A in (c.X, c.Y, c.Z))
            for e1 in (-gp, gp):
                for e2 in (-gp, gp):
                    phi = 0.25 * (1 + sx * e1) * (1 + sy * e2)
                    grads = np.stack([0.25 * sx * (1 + sy * e2), 0.25 * sy * (1 + sx * e1)], axis=1)
                    J = np.array([[xs @ grads[:, 0], xs @ grads[:, 1]],
                                  [ys @ grads[:, 0], ys @ grads[:, 1]]])
                    zp = zs @ grads
                    j2 = np.linalg.det(J)
                    adj = np.array([[J[1, 1], -J[0, 1]], [-J[1, 0], J[0, 0]]])
                    W = adj @ np.diag([c1, c2]) @ adj.T / j2
                    blk = np.ix_(idx, idx)
                    P[blk] += grads @ W @ grads.T
                    Q[blk] += np.outer(grads @ W @ zp, phi)
                    R[blk] += (zp @ W @ zp + c3 * j2) * np.outer(phi, phi)
    return P, Q, R


def _layer_factors(h):
    """Vertical factors: exact 1-D integrals of linear elements of thickness
    h_l, sum (h/2) m, sum g and sum (2/h) kappa over the layers."""
    nz = len(h)
    M, G, Kv = (np.zeros((nz + 1, nz + 1)) for _ in range(3))
    m = np.array([[2.0, 1.0], [1.0, 2.0]]) / 3.0
    g = np.array([[-1.0, 1.0], [-1.0, 1.0]]) / 2.0
    kap = np.array([[1.0, -1.0], [-1.0, 1.0]]) / 2.0
    for l, hl in enumerate(h):
        s = slice(l, l + 2)
        M[s, s] += hl / 2.0 * m
        G[s, s] += g
        Kv[s, s] += 2.0 / hl * kap
    return M, G, Kv


@pytest.mark.parametrize("a", [(1.0, 1.0, 1.0), (2.0, 1.0, 0.5)])
def test_shift_form_stiffness_is_a_sum_of_column_layer_products(a):
    """On a terrain-following grid in shift form (z = z_s(x, y) + zeta_k) the
    2x2x2-Gauss stiffness of Eq. 5 equals
      M (x) P - G (x) Q - G^T (x) Q^T + K_v (x) R
    exactly (up to rounding): det J = (h/2) j2 and the vertical parts are
    polynomials the 2-point rule integrates exactly.  The oracle's element
    loop on a curved grid against the factors formed here."""
    c = synth.single_hill(6, 5, 3, sigma=60.0, height=30.0, a=a)
    h = np.diff(c.Z[:, 0, 0])
    assert np.allclose(c.Z - c.Z[:1], (c.Z[:, 0, 0] - c.Z[0, 0, 0])[:, None, None], atol=1e-9)
    P, Q, R = _column_factors(c)
    M, G, Kv = _layer_factors(h)
    Kref = np.kron(M, P) - np.kron(G, Q) - np.kron(G.T, Q.T) + np.kron(Kv, R)
    K = oracle.assemble_K(c).toarray()
    assert np.abs(K - Kref).max() <= 1e-12 * np.abs(K).max()
    # the terrain matters: the Q terms are not zero on this grid
    assert np.abs(Q).max() > 1e-3 * np.abs(P).max()


def test_shift_form_load_vector_is_a_sum_of_column_layer_products():
    """The load vector of Eq. 5 (2x2x2 Gauss, u0 trilinear from the nodes) on
    a shift-form grid: with det J grad N = ((h/2) adj^T grad phi psi -
    adj^T z' phi psi', j2 phi psi') and u0 interpolated,
      f = -[(V_M (x) E_x) u_x + (V_M (x) E_y) u_y - (V_G^T (x) F_x) u_x
            - (V_G^T (x) F_y) u_y + (V_G^T (x) M_z) u_z],
    E_d = sum (adj^T grad phi_a)_d phi_b, F_d = sum (adj^T z')_d phi_a phi_b,
    M_z = sum j2 phi_a phi_b over the 2 x 2 points, V_M = sum (h/2) m,
    V_G = sum g.  Against the oracle's element loop."""
    c = synth.single_hill(6, 5, 3, sigma=60.0, height=30.0, a=(1.0, 2.0, 0.5))
    nx, ny = c.nx, c.ny
    ncol = (nx + 1) * (ny + 1)
    Ex, Ey, Fx, Fy, Mz = (np.zeros((ncol, ncol)) for _ in range(5))
    sx = np.array([-1.0, 1.0, -1.0, 1.0])
    sy = np.array([-1.0, -1.0, 1.0, 1.0])
    gp = 1.0 / np.sqrt(3.0)
    for cj in range(ny):
        for ci in range(nx):
            idx = [(cj + (p >> 1)) * (nx + 1) + ci + (p & 1) for p in range(4)]
            xs, ys, zs = (np.array([A[0].flat[n] for n in idx]) for A in (c.X, c.Y, c.Z))
            for e1 in (-gp, gp):
                for e2 in (-gp, gp):
                    phi = 0.25 * (1 + sx * e1) * (1 + sy * e2)
                    grads = np.stack([0.25 * sx * (1 + sy * e2), 0.25 * sy * (1 + sx * e1)], axis=1)
                    J = np.array([[xs @ grads[:, 0], xs @ grads[:, 1]],
                                  [ys @ grads[:, 0], ys @ grads[:, 1]]])
                    zp = zs @ grads
                    adjT = np.array([[J[1, 1], -J[1, 0]], [-J[0, 1], J[0, 0]]])  # adj(J2)^T
                    ag = grads @ adjT.T          # rows: (adj^T grad phi_a)
                    az = adjT @ zp               # adj^T z'
                    blk = np.ix_(idx, idx)
                    Ex[blk] += np.outer(ag[:, 0], phi)
                    Ey[blk] += np.outer(ag[:, 1], phi)
                    pp = np.outer(phi, phi)
                    Fx[blk] += az[0] * pp
                    Fy[blk] += az[1] * pp
                    Mz[blk] += np.linalg.det(J) * pp
    M, G, _ = _layer_factors(np.diff(c.Z[:, 0, 0]))
    ux, uy, uz = (c.u0[d].ravel() for d in range(3))
    f_ref = -(np.kron(M, Ex) @ ux + np.kron(M, Ey) @ uy - np.kron(G.T, Fx) @ ux
              - np.kron(G.T, Fy) @ uy + np.kron(G.T, Mz) @ uz)
    f = oracle.assemble_f(c)
    assert np.abs(f - f_ref).max() <= 1e-12 * np.abs(f).max()


def test_galerkin_hierarchy_keeps_the_column_layer_form():
    """Eq. 7 on a shift-form grid: with P = P_z (x) P_y (x) P_x and the free
    set a product of free layers and free columns, every level's operator is
    sum_t V_t^l (x) H_t^l with V^{l+1} = P_z^T V^l P_z and H^{l+1} =
    P_h^T H^l P_h (each masked to its free set).  Against the oracle's
    Galerkin hierarchy, level by level; and V_G + V_G^T = -e0 e0^T on every
    level, which leaves three terms above the ground layer."""
    c = synth.single_hill(8, 8, 4, sigma=60.0, height=30.0)
    Hy = oracle.Hierarchy(c, coarsest_max=16)
    assert len(Hy.levels) >= 3
    P, Q, R = _column_factors(c)
    M, G, Kv = _layer_factors(np.diff(c.Z[:, 0, 0]))
    terms = [(M, P), (-G, Q), (-G.T, Q.T), (Kv, R)]
    for l, lev in enumerate(Hy.levels):
        Nx, Ny, Nz = lev["Nx"], lev["Ny"], lev["Nz"]
        ii, jj = np.meshgrid(np.arange(Nx), np.arange(Ny))
        dh = ((ii >= 1) & (ii <= Nx - 2) & (jj >= 1) & (jj <= Ny - 2)).ravel().astype(float)
        dv = (np.arange(Nz) <= Nz - 2).astype(float)
        terms = [(dv[:, None] * V * dv[None, :], dh[:, None] * Hh * dh[None, :]) for V, Hh in terms]
        Kref = sum(np.kron(V, Hh) for V, Hh in terms)
        K = Hy.K[l].toarray()
        assert np.abs(K - Kref).max() <= 1e-12 * np.abs(K).max(), l
        # the three-term form: V_G + V_G^T = -e0 e0^T on the free layers of
        # every level (the ground layer is a node layer of every level)
        B2 = -(terms[1][0] + terms[2][0])
        E = np.zeros_like(B2)
        E[0, 0] = -1.0
        assert np.abs(B2 - E).max() <= 1e-14, l
        if l + 1 < len(Hy.levels):
            Px = oracle._p1d_horizontal(Nx, lev["hx"]).toarray()
            Py = oracle._p1d_horizontal(Ny, lev["hy"]).toarray()
            Pz = oracle._p1d_from_map(Nz, lev["kmap"]).toarray()
            Ph = np.kron(Py, Px)
            terms = [(Pz.T @ V @ Pz, Ph.T @ Hh @ Ph) for V, Hh in terms]


def test_shift_form_center_gradient():
    """Eq. 3 at the element centers of a shift-form grid: J = [[J2, 0],
    [z'^T, h/2]] there, so d lambda/dz = (2/h) g_3 and (d lambda/dx,
    d lambda/dy) = J2^-T (g_h - z' d lambda/dz) with g the reference
    gradient, from the column's center Jacobian and the layer thickness
    alone.  Against the oracle's recovery with its full element Jacobians."""
    c = synth.single_hill(6, 5, 3, sigma=60.0, height=30.0, a=(1.0, 2.0, 0.5))
    rng = np.random.default_rng(3)
    lam = rng.normal(size=(c.nz + 1, c.ny + 1, c.nx + 1))
    a2 = np.asarray(c.a, dtype=float) ** 2
    u = np.zeros((3, c.nz, c.ny, c.nx))
    for j in range(c.ny):
        for i in range(c.nx):
            xs, ys, zs = (A[0, j:j + 2, i:i + 2].ravel() for A in (c.X, c.Y, c.Z))  # p = a + 2b
            J2 = 0.25 * np.array([[(xs[1] - xs[0]) + (xs[3] - xs[2]), (xs[2] - xs[0]) + (xs[3] - xs[1])],
                                  [(ys[1] - ys[0]) + (ys[3] - ys[2]), (ys[2] - ys[0]) + (ys[3] - ys[1])]])
            zp = 0.25 * np.array([(zs[1] - zs[0]) + (zs[3] - zs[2]), (zs[2] - zs[0]) + (zs[3] - zs[1])])
            for k in range(c.nz):
                h = c.Z[k + 1, 0, 0] - c.Z[k, 0, 0]
                l = lam[k:k + 2, j:j + 2, i:i + 2]            # [c][b][a]
                g = 0.125 * np.array([(l[:, :, 1] - l[:, :, 0]).sum(),
                                      (l[:, 1, :] - l[:, 0, :]).sum(),
                                      (l[1] - l[0]).sum()])
                gz = 2.0 / h * g[2]
                gh = np.linalg.solve(J2.T, g[:2] - zp * gz)
                u0c = c.u0[:, k:k + 2, j:j + 2, i:i + 2].mean(axis=(1, 2, 3))
                u[:, k, j, i] = u0c + np.array([gh[0], gh[1], gz]) / a2
    ref = oracle.recover(c, lam.ravel())
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()
