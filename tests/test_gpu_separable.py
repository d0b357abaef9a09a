"""Parity of the separable (column x layer) operator and its float32 cycle
with the oracle, through the C boundary.

On a terrain-following grid in shift form (z = z_s(x, y) + zeta_k, Sec. 2)
the stiffness of Eq. 5 equals sum_t H_t (x) V_t exactly and the Galerkin
products of Eq. 7 keep that form, so the factors must reproduce the
oracle's element-by-element operator and its P^T K P hierarchy on every
level (float64 factors to rounding, float32 factors to float32 rounding),
and the cycle built on them must smooth, restrict and converge like the
oracle's."""
import numpy as np
import pytest

import oracle
import paper_2101_08453_gb300 as m
import synth
from gpu_cases import rel, small_cases, stencil_planes, to_dev

pytestmark = pytest.mark.gpu

CASES = small_cases()
SHIFT = ["hill64", "ragged", "aniso", "penalty"]   # all shift-form grids


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    m.build.build()
    return t


_cache = {}
_lam_ref = {}


def setup(torch, name, coarsest_max=64, **opt):
    key = (name, coarsest_max, tuple(sorted(opt.items())))
    if key in _cache:
        return _cache[key]
    c = CASES[name]
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    plan = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=m.OP_SEPARABLE,
                           coarsest_max=coarsest_max, **opt)
    plan.assemble(X, Y, Z)
    rule = "paper" if plan.options.coarsen_rule == m.RULE_PAPER else "operator"
    H = oracle.Hierarchy(c, coarsest_max=coarsest_max, rule=rule)
    out = (c, plan, (X, Y, Z, u0), H)
    _cache[key] = out
    return out


def level_dims(plan, l):
    d = plan.level(l)
    return d["Nx"], d["Ny"], d["Nz"]


@pytest.mark.parametrize("name", SHIFT)
def test_separable_stencil_all_levels(torch, name):
    """Rows rebuilt from the factors against the oracle's K_FF and its
    Galerkin hierarchy (float64 factors: rounding; float32: float rounding)."""
    c, plan, _, H = setup(torch, name)
    assert plan.num_levels == len(H.levels)
    for l in range(plan.num_levels):
        dims = level_dims(plan, l)
        assert dims == H.dims(l)
        ref = stencil_planes(H.K[l], dims)
        N = dims[0] * dims[1] * dims[2]
        for prec, tol in ((m.PREC_F64, 1e-12), (m.PREC_MIXED, 2e-7)):
            out = torch.empty((27, N), dtype=torch.float64, device="cuda")
            m.mcwind_level_stencil(plan.handle, l, prec, out)
            err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
            assert err <= tol, (l, prec, err)


@pytest.mark.parametrize("name", SHIFT)
@pytest.mark.parametrize("quad", [m.RHS_GAUSS8, m.RHS_CENTER1])
def test_separable_rhs(torch, name, quad):
    """The load vector of Eq. 5: from column x layer factors in float pairs
    (2x2x2 Gauss, nodal u0), element by element for the one-point rule."""
    c, plan, (X, Y, Z, u0), _ = setup(torch, name, rhs_quad=quad)
    f = plan.rhs(u0).cpu().numpy().ravel()
    ref = oracle.assemble_f(c, quad=quad)
    ref[~oracle.case_free_mask(c)] = 0.0
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", SHIFT)
def test_separable_residual(torch, name):
    c, plan, _, H = setup(torch, name)
    rng = np.random.default_rng(1)
    for l in range(plan.num_levels):
        dims = level_dims(plan, l)
        free = H.free[l]
        x = np.where(free, rng.normal(size=free.size), 0.0)
        f = np.where(free, rng.normal(size=free.size), 0.0)
        ref = np.where(free, f - H.K[l] @ x, 0.0)
        scale = np.abs(H.K[l]).max() * np.abs(x).max() * 27
        xd, fd = to_dev(torch, x.reshape(dims[::-1]), f.reshape(dims[::-1]))
        r = torch.empty_like(xd)
        m.mcwind_level_residual(plan.handle, l, m.PREC_MIXED, xd, fd, r)
        err = np.abs(r.cpu().numpy().ravel() - ref).max() / scale
        assert err <= 2e-6, (l, err)


@pytest.mark.parametrize("name", SHIFT)
def test_separable_residual_restrict(torch, name):
    """f_c = P^T (f - K x), Eq. 7 first row: fused on transfers that keep the
    columns, residual then restriction on the others."""
    c, plan, _, H = setup(torch, name)
    rng = np.random.default_rng(3)
    for l in range(plan.num_levels - 1):
        df, dc = level_dims(plan, l), level_dims(plan, l + 1)
        free, fc = H.free[l], H.free[l + 1]
        x = np.where(free, rng.normal(size=free.size), 0.0)
        f = np.where(free, rng.normal(size=free.size), 0.0)
        ref = np.where(fc, H.P[l].T @ np.where(free, f - H.K[l] @ x, 0.0), 0.0)
        scale = np.abs(H.K[l]).max() * np.abs(x).max() * 27 * 8
        xd, fd = to_dev(torch, x.reshape(df[::-1]), f.reshape(df[::-1]))
        out = torch.empty(dc[::-1], dtype=torch.float64, device="cuda")
        m.mcwind_level_residual_restrict(plan.handle, l, m.PREC_MIXED, xd, fd, out)
        err = np.abs(out.cpu().numpy().ravel() - ref).max() / scale
        assert err <= 2e-6, (l, err)
        if l == 0:
            m.mcwind_level_residual_restrict(plan.handle, l, m.PREC_F64, xd, fd, out)
            assert np.abs(out.cpu().numpy().ravel() - ref).max() / scale <= 1e-14
        else:
            # no float64 operator on an intermediate level of the separable form
            with pytest.raises(m.MCWindError) as e:
                m.mcwind_level_residual_restrict(plan.handle, l, m.PREC_F64, xd, fd, out)
            assert e.value.code == m.MCWIND_EINVAL


@pytest.mark.parametrize("name", SHIFT)
@pytest.mark.parametrize("direction", [m.FORWARD, m.BACKWARD])
def test_separable_smoother(torch, name, direction):
    """Two sweeps of the column Gauss-Seidel of Sec. 3 (4 column groups, the
    columns bottom-up or top-down) against the oracle's ordered sweep."""
    c, plan, _, H = setup(torch, name)
    rng = np.random.default_rng(2 + direction)
    for l in range(plan.num_levels - 1):
        dims = level_dims(plan, l)
        free = H.free[l]
        x0 = np.where(free, rng.normal(size=free.size), 0.0)
        f = np.where(free, rng.normal(size=free.size), 0.0)
        ref = x0.copy()
        for _ in range(2):
            oracle.gs_sweep(H.K[l], f, ref, dims, direction)
        xd, fd = to_dev(torch, x0.reshape(dims[::-1]), f.reshape(dims[::-1]))
        m.mcwind_level_smooth(plan.handle, l, m.PREC_MIXED, xd, fd, 2, direction)
        err = rel(xd.cpu().numpy().ravel(), ref)
        assert err <= 1e-4, (l, err)


@pytest.mark.parametrize("name", SHIFT)
def test_separable_vcycle(torch, name):
    c, plan, _, H = setup(torch, name)
    dims = level_dims(plan, 0)
    free = H.free[0]
    rng = np.random.default_rng(11)
    x0 = np.where(free, rng.normal(size=free.size), 0.0)
    f = np.where(free, rng.normal(size=free.size), 0.0)
    ref = H.vcycle(0, f, x0.copy())
    xd, fd = to_dev(torch, x0.reshape(dims[::-1]), f.reshape(dims[::-1]))
    m.mcwind_vcycle(plan.handle, m.PREC_MIXED, xd, fd)
    assert rel(xd.cpu().numpy().ravel(), ref) <= 1e-4
    with pytest.raises(m.MCWindError):
        m.mcwind_vcycle(plan.handle, m.PREC_F64, xd, fd)


@pytest.mark.parametrize("name", SHIFT)
@pytest.mark.parametrize("accel", [m.ACCEL_NONE, m.ACCEL_CG])
def test_separable_solve_and_recover(torch, name, accel):
    """The float64 refinement around the separable float32 cycle reaches the
    oracle's lambda and u (Eq. 3) to 1e-10."""
    c, plan, (X, Y, Z, u0), H = setup(torch, name, coarsest_max=1024, accel=accel)
    lam, st = plan.solve(u0, rtol=1e-12, max_cycles=120)
    assert st.status == m.MCWIND_OK and st.rel_res <= 1e-12, st.history()
    if name not in _lam_ref:
        _lam_ref[name] = oracle.solve(c)
    lam_ref = _lam_ref[name]
    assert rel(lam.cpu().numpy().ravel(), lam_ref) <= 1e-10
    u = plan.recover(u0, lam).cpu().numpy()
    assert rel(u, oracle.recover(c, lam_ref)) <= 1e-10


def test_separable_converges_like_the_stored_form(torch):
    """Same method, same hierarchy: the separable cycle needs the stored
    form's cycle count (within two cycles, checked after every cycle) on the
    150 m hill."""
    c = CASES["hill64"]
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    counts = []
    for form in (m.OP_STORED, m.OP_SEPARABLE):
        plan = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=form, coarsest_max=1024,
                               cycles_per_check=1)
        plan.assemble(X, Y, Z)
        _, st = plan.solve(u0, rtol=1e-10, max_cycles=100)
        assert st.status == m.MCWIND_OK
        counts.append(st.cycles)
    assert abs(counts[0] - counts[1]) <= 2, counts


def test_separable_refuses_a_grid_not_in_shift_form(torch):
    c = CASES["jitter"]
    X, Y, Z = to_dev(torch, c.X, c.Y, c.Z)
    plan = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=m.OP_SEPARABLE)
    with pytest.raises(m.MCWindError) as e:
        plan.assemble(X, Y, Z)
    assert e.value.code == m.MCWIND_ESHIFT
    # a column whose layers are shifted by a different amount is refused too
    c = synth.single_hill(12, 10, 4, sigma=100.0, height=40.0)
    Zb = c.Z.copy()
    Zb[2, 5, 6] += 0.01
    X, Y, Z = to_dev(torch, c.X, c.Y, Zb)
    plan = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=m.OP_SEPARABLE)
    with pytest.raises(m.MCWindError) as e:
        plan.assemble(X, Y, Z)
    assert e.value.code == m.MCWIND_ESHIFT


@pytest.mark.parametrize("name", ["hill64", "ragged"])
def test_separable_float64_element_arithmetic(torch, name):
    """element_arith = ARITH_F64: the column factors, the expanded float64
    rows and the load vector in float64; both arithmetics against the
    oracle's element loop, and against each other."""
    c, plan64, (X, Y, Z, u0), H = setup(torch, name, element_arith=m.ARITH_F64)
    _, plan2, _, _ = setup(torch, name)
    dims = level_dims(plan64, 0)
    N = dims[0] * dims[1] * dims[2]
    ref = stencil_planes(H.K[0], dims)
    rows = []
    for plan in (plan64, plan2):
        out = torch.empty((27, N), dtype=torch.float64, device="cuda")
        m.mcwind_level_stencil(plan.handle, 0, m.PREC_F64, out)
        rows.append(out.cpu().numpy())
        assert np.abs(rows[-1] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(rows[0] - rows[1]).max() <= 1e-13 * np.abs(ref).max()
    # the float64 residual reads the rows expanded from the factors
    rng = np.random.default_rng(5)
    free = H.free[0]
    x = np.where(free, rng.normal(size=free.size), 0.0)
    f = np.where(free, rng.normal(size=free.size), 0.0)
    rref = np.where(free, f - H.K[0] @ x, 0.0)
    scale = np.abs(H.K[0]).max() * np.abs(x).max() * 27
    xd, fd = to_dev(torch, x.reshape(dims[::-1]), f.reshape(dims[::-1]))
    for plan in (plan64, plan2):
        r = torch.empty_like(xd)
        m.mcwind_level_residual(plan.handle, 0, m.PREC_F64, xd, fd, r)
        assert np.abs(r.cpu().numpy().ravel() - rref).max() <= 1e-14 * scale
    fref = oracle.assemble_f(c)
    fref[~oracle.case_free_mask(c)] = 0.0
    f64 = plan64.rhs(u0).cpu().numpy().ravel()
    assert np.abs(f64 - fref).max() <= 1e-13 * np.abs(fref).max()
    lam, st = plan64.solve(u0, rtol=1e-11, max_cycles=120)
    assert st.status == m.MCWIND_OK


@pytest.mark.parametrize("name", ["hill64", "aniso"])
def test_separable_recovery_with_u0_at_centers(torch, name):
    """u0 given at the element centers (the paper's representation of the
    wind, Sec. 2): the load vector element by element, the solve on the
    separable cycle, the recovery from the column's center Jacobian."""
    c = CASES[name]
    rng = np.random.default_rng(4)
    uc = rng.normal(size=(3, c.nz, c.ny, c.nx)) + np.array([5.0, -2.0, 0.0])[:, None, None, None]
    X, Y, Z, ucd = to_dev(torch, c.X, c.Y, c.Z, uc)
    plan = m.Plan.for_case(c, u0_at=m.U0_CENTERS, precision=m.PREC_MIXED,
                           op_form=m.OP_SEPARABLE, coarsest_max=1024)
    plan.assemble(X, Y, Z)
    lam, st = plan.solve(ucd, rtol=1e-12, max_cycles=120)
    assert st.status == m.MCWIND_OK
    f_ref = oracle.assemble_f_centers(c, uc, m.RHS_GAUSS8)
    lam_ref = oracle.solve(c, f=f_ref)
    assert rel(lam.cpu().numpy().ravel(), lam_ref) <= 1e-10
    u = plan.recover(ucd, lam).cpu().numpy()
    assert rel(u, oracle.recover_centers(c, lam_ref, uc)) <= 1e-10


@pytest.mark.parametrize("name", SHIFT)
def test_separable_recovery_of_a_given_lambda(torch, name):
    """The recovery alone (Eq. 3) for a random lambda: the column x layer
    form of the center gradient against the oracle's element Jacobians."""
    c, plan, (X, Y, Z, u0), _ = setup(torch, name)
    rng = np.random.default_rng(9)
    lam = rng.normal(size=(c.nz + 1, c.ny + 1, c.nx + 1))
    lam[~oracle.case_free_mask(c).reshape(lam.shape)] = 0.0
    (lamd,) = to_dev(torch, lam)
    u = plan.recover(u0, lamd).cpu().numpy()
    ref = oracle.recover(c, lam.ravel())
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()
