"""Parity of every CUDA kernel, called through the C boundary, with the CPU
oracle on the same seeded inputs (FP64: rounding-level agreement; FP32
kernels: float32 rounding)."""
import numpy as np
import pytest

import oracle
import paper_2101_08453_gb300 as m
import synth
from gpu_cases import rel, small_cases, stencil_planes, to_dev

pytestmark = pytest.mark.gpu

CASES = small_cases()
NAMES = list(CASES)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    m.build.build()
    return t


_cache = {}
_lam_ref = {}


def setup(torch, name, precision=m.PREC_MIXED, coarsest_max=64, **opt):
    key = (name, precision, coarsest_max, tuple(sorted(opt.items())))
    if key in _cache:
        return _cache[key]
    c = CASES[name]
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    plan = m.Plan.for_case(c, precision=precision, coarsest_max=coarsest_max, **opt)
    plan.assemble(X, Y, Z)
    rule = "paper" if plan.options.coarsen_rule == m.RULE_PAPER else "operator"
    H = oracle.Hierarchy(c, coarsest_max=coarsest_max, rule=rule)
    out = (c, plan, (X, Y, Z, u0), H)
    _cache[key] = out
    return out


def level_dims(plan, l):
    d = plan.level(l)
    return d["Nx"], d["Ny"], d["Nz"]


@pytest.mark.parametrize("name", NAMES)
def test_hierarchy_matches_oracle(torch, name):
    c, plan, _, H = setup(torch, name)
    assert plan.num_levels == len(H.levels)
    for l, lev in enumerate(H.levels):
        assert level_dims(plan, l) == (lev["Nx"], lev["Ny"], lev["Nz"])


@pytest.mark.parametrize("name", NAMES)
def test_stencil_all_levels(torch, name):
    c, plan, _, H = setup(torch, name)
    for l in range(plan.num_levels):
        dims = level_dims(plan, l)
        ref = stencil_planes(H.K[l], dims)
        N = dims[0] * dims[1] * dims[2]
        for prec, tol in ((m.PREC_F64, 1e-12), (m.PREC_MIXED, 2e-7)):
            out = torch.empty((27, N), dtype=torch.float64, device="cuda")
            m.mcwind_level_stencil(plan.handle, l, prec, out)
            got = out.cpu().numpy()
            scale = np.abs(ref).max()
            err = np.abs(got - ref).max() / scale
            assert err <= tol, (l, prec, err)


def test_stencil_f64_ulp_level_on_fine_grid(torch):
    c, plan, _, H = setup(torch, "hill64", element_arith=m.ARITH_F64)
    dims = level_dims(plan, 0)
    ref = stencil_planes(H.K[0], dims)
    out = torch.empty((27, ref.shape[1]), dtype=torch.float64, device="cuda")
    m.mcwind_level_stencil(plan.handle, 0, m.PREC_F64, out)
    got = out.cpu().numpy()
    diag = np.abs(ref[13]).max()
    assert np.abs(got - ref).max() <= 1e-13 * diag
    # row sums of K_FF vanish in rows away from the boundary
    free = oracle.free_mask(*dims)
    Nx, Ny, Nz = dims
    interior = np.zeros((Nz, Ny, Nx), bool)
    interior[1:-2, 2:-2, 2:-2] = True
    assert np.abs(got.sum(axis=0)[interior.ravel()]).max() <= 1e-12 * diag


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("quad", [m.RHS_GAUSS8, m.RHS_CENTER1])
def test_rhs(torch, name, quad):
    c, plan, (X, Y, Z, u0), _ = setup(torch, name, rhs_quad=quad)
    f = plan.rhs(u0).cpu().numpy().ravel()
    ref = oracle.assemble_f(c, quad=quad)
    ref[~oracle.case_free_mask(c)] = 0.0
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", NAMES)
def test_residual(torch, name):
    c, plan, _, H = setup(torch, name)
    rng = np.random.default_rng(1)
    for l in range(plan.num_levels):
        dims = level_dims(plan, l)
        free = H.free[l]
        x = np.where(free, rng.normal(size=free.size), 0.0)
        f = np.where(free, rng.normal(size=free.size), 0.0)
        ref = np.where(free, f - H.K[l] @ x, 0.0)
        scale = np.abs(H.K[l]).max() * np.abs(x).max() * 27
        for prec, tol in ((m.PREC_F64, 1e-14), (m.PREC_MIXED, 2e-6)):
            xd, fd = to_dev(torch, x.reshape(dims[::-1]), f.reshape(dims[::-1]))
            r = torch.empty_like(xd)
            m.mcwind_level_residual(plan.handle, l, prec, xd, fd, r)
            err = np.abs(r.cpu().numpy().ravel() - ref).max() / scale
            assert err <= tol, (l, prec, err)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("direction", [m.FORWARD, m.BACKWARD])
def test_smoother(torch, name, direction):
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
        for prec, tol in ((m.PREC_F64, 1e-11), (m.PREC_MIXED, 1e-4)):
            xd, fd = to_dev(torch, x0.reshape(dims[::-1]), f.reshape(dims[::-1]))
            m.mcwind_level_smooth(plan.handle, l, prec, xd, fd, 2, direction)
            err = rel(xd.cpu().numpy().ravel(), ref)
            assert err <= tol, (l, prec, err)


@pytest.mark.parametrize("name", NAMES)
def test_restrict_prolong(torch, name):
    c, plan, _, H = setup(torch, name)
    rng = np.random.default_rng(5)
    for l in range(plan.num_levels - 1):
        df, dc = level_dims(plan, l), level_dims(plan, l + 1)
        P = H.P[l]
        ff, fc = H.free[l], H.free[l + 1]
        r = np.where(ff, rng.normal(size=ff.size), 0.0)
        ref_c = np.where(fc, P.T @ r, 0.0)
        ec = np.where(fc, rng.normal(size=fc.size), 0.0)
        x = np.where(ff, rng.normal(size=ff.size), 0.0)
        ref_x = np.where(ff, x + P @ ec, 0.0)
        for prec, tol in ((m.PREC_F64, 1e-15), (m.PREC_MIXED, 1e-6)):
            rd, = to_dev(torch, r.reshape(df[::-1]))
            out = torch.empty(dc[::-1], dtype=torch.float64, device="cuda")
            m.mcwind_level_restrict(plan.handle, l, prec, rd, out)
            assert rel(out.cpu().numpy().ravel(), ref_c) <= tol
            ed, xd = to_dev(torch, ec.reshape(dc[::-1]), x.reshape(df[::-1]))
            m.mcwind_level_prolong(plan.handle, l, prec, ed, xd)
            assert rel(xd.cpu().numpy().ravel(), ref_x) <= tol


@pytest.mark.parametrize("name", NAMES)
def test_coarse_solve(torch, name):
    c, plan, _, H = setup(torch, name)
    L = plan.num_levels - 1
    dims = level_dims(plan, L)
    free = H.free[L]
    f = np.where(free, np.random.default_rng(7).normal(size=free.size), 0.0)
    ref = H.coarse_solve(f)
    fd, = to_dev(torch, f.reshape(dims[::-1]))
    x = torch.empty_like(fd)
    m.mcwind_coarse_solve(plan.handle, fd, x)
    assert rel(x.cpu().numpy().ravel(), ref) <= 1e-11


@pytest.mark.parametrize("name", NAMES)
def test_vcycle(torch, name):
    c, plan, _, H = setup(torch, name)
    dims = level_dims(plan, 0)
    free = H.free[0]
    rng = np.random.default_rng(11)
    x0 = np.where(free, rng.normal(size=free.size), 0.0)
    f = np.where(free, rng.normal(size=free.size), 0.0)
    ref = H.vcycle(0, f, x0.copy())
    for prec, tol in ((m.PREC_F64, 1e-11), (m.PREC_MIXED, 1e-4)):
        xd, fd = to_dev(torch, x0.reshape(dims[::-1]), f.reshape(dims[::-1]))
        m.mcwind_vcycle(plan.handle, prec, xd, fd)
        assert rel(xd.cpu().numpy().ravel(), ref) <= tol, prec


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [m.PREC_F64, m.PREC_MIXED])
def test_solve_and_recover(torch, name, precision):
    c, plan, (X, Y, Z, u0), H = setup(torch, name, precision=precision, coarsest_max=1024)
    lam, st = plan.solve(u0, rtol=1e-12, max_cycles=120)
    assert st.status == m.MCWIND_OK and st.rel_res <= 1e-12, st.history()
    if name not in _lam_ref:
        _lam_ref[name] = oracle.solve(c)
    lam_ref = _lam_ref[name]
    el = rel(lam.cpu().numpy().ravel(), lam_ref)
    assert el <= 1e-10, el
    for where in (m.AT_CENTERS, m.AT_GAUSS):
        u = plan.recover(u0, lam, where).cpu().numpy()
        u_ref = oracle.recover(c, lam_ref, where=where)
        assert rel(u, u_ref) <= 1e-10
    # the recovered wind is discretely divergence free (Eq. 5)
    ug = plan.recover(u0, lam, m.AT_GAUSS)
    bu = torch.empty(plan.node_shape, dtype=torch.float64, device="cuda")
    m.mcwind_weak_div(plan.handle, ug, bu)
    bu0 = oracle.weak_div(c, oracle.interp_gauss(c))
    free = oracle.case_free_mask(c)
    assert np.linalg.norm(bu.cpu().numpy().ravel()[free]) <= 1e-9 * np.linalg.norm(bu0[free])


def test_rate_within_paper_bound(torch):
    """Sec. 3: at most about 0.28 per cycle with four smoothing steps (the
    single 150 m hill; steep random terrain converges more slowly)."""
    c, plan, (X, Y, Z, u0), H = setup(torch, "hill64", precision=m.PREC_F64, coarsest_max=1024)
    lam, st = plan.solve(u0, rtol=1e-10, max_cycles=80)
    assert st.status == m.MCWIND_OK
    assert st.rate <= 0.28, st.rate


@pytest.mark.parametrize("name", NAMES)
def test_rate_matches_oracle_cycle(torch, name):
    """The GPU cycle and the oracle's cycle reduce the residual at the same rate."""
    c, plan, (X, Y, Z, u0), H = setup(torch, name, precision=m.PREC_F64, coarsest_max=1024)
    lam, st = plan.solve(u0, rtol=1e-10, max_cycles=100)
    assert st.status == m.MCWIND_OK
    x, hist = H.solve(oracle.assemble_f(c), rtol=1e-10, max_cycles=100)
    assert abs(st.cycles - (len(hist) - 1)) <= 1
    assert np.allclose(st.history()[:6], hist[:6], rtol=1e-6)


def test_weak_div_matches_oracle(torch):
    c, plan, (X, Y, Z, u0), _ = setup(torch, "jitter")
    ug = np.random.default_rng(3).normal(size=(3, 8, c.nz, c.ny, c.nx))
    ugd, = to_dev(torch, ug)
    out = torch.empty(plan.node_shape, dtype=torch.float64, device="cuda")
    m.mcwind_weak_div(plan.handle, ugd, out)
    ref = oracle.weak_div(c, ug)
    assert np.abs(out.cpu().numpy().ravel() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_warm_start(torch):
    c, plan, (X, Y, Z, u0), _ = setup(torch, "hill64", precision=m.PREC_MIXED, coarsest_max=1024)
    lam, st_cold = plan.solve(u0, rtol=1e-10)
    u0b = torch.from_numpy(synth.perturb_wind(c.u0, 0)).to("cuda")
    lam_w = lam.clone()
    lam_w, st_warm = plan.solve(u0b, lam=lam_w, rtol=1e-10, warm=True)
    lam_c, st_c2 = plan.solve(u0b, rtol=1e-10)
    assert st_warm.status == m.MCWIND_OK
    assert st_warm.res_hist[0] < st_c2.res_hist[0]
    assert st_warm.cycles < st_c2.cycles
    assert rel(lam_w.cpu().numpy(), lam_c.cpu().numpy()) <= 1e-8


def test_deterministic(torch):
    c, plan, (X, Y, Z, u0), _ = setup(torch, "ragged", precision=m.PREC_MIXED, coarsest_max=1024)
    a, _ = plan.solve(u0, rtol=1e-10)
    b, _ = plan.solve(u0, rtol=1e-10)
    assert torch.equal(a, b)


def test_uniform_wind_flat_ground(torch):
    c = synth.flat_box(30, 22, 6, stretch=1.2)
    c.u0[0], c.u0[1] = 6.0, -3.0
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    plan = m.Plan.for_case(c)
    plan.assemble(X, Y, Z)
    lam, st = plan.solve(u0, rtol=1e-8)
    assert float(lam.abs().max()) <= 1e-9
    u = plan.recover(u0, lam).cpu().numpy()
    assert np.allclose(u[0], 6.0) and np.allclose(u[1], -3.0) and np.abs(u[2]).max() <= 1e-9


def test_not_converged_status(torch):
    c, plan, (X, Y, Z, u0), _ = setup(torch, "hill64", precision=m.PREC_F64, coarsest_max=1024)
    lam = torch.zeros(plan.node_shape, dtype=torch.float64, device="cuda")
    rc, st = m.mcwind_solve(plan.handle, u0, lam, 1e-14, 1)
    assert rc == m.MCWIND_ENOTCONV and st.cycles == 1 and st.status == m.MCWIND_ENOTCONV
    assert float(lam.abs().max()) > 0


def test_nonfinite_wind(torch):
    c, plan, (X, Y, Z, u0), _ = setup(torch, "hill64", precision=m.PREC_F64, coarsest_max=1024)
    bad = u0.clone()
    bad[0, 3, 10, 10] = float("nan")
    lam = torch.zeros(plan.node_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MCWindError) as e:
        m.mcwind_solve(plan.handle, bad, lam, 1e-8, 10)
    assert e.value.code == m.MCWIND_ENONFINITE


def test_inverted_element(torch):
    c = synth.single_hill(12, 10, 4, sigma=100.0, height=40.0)
    Z = c.Z.copy()
    Z[1, 5, 6], Z[2, 5, 6] = Z[2, 5, 6], Z[1, 5, 6]
    X, Y, Zd = to_dev(torch, c.X, c.Y, Z)
    plan = m.Plan.for_case(c)
    with pytest.raises(m.MCWindError) as e:
        plan.assemble(X, Y, Zd)
    assert e.value.code == m.MCWIND_EGEOM


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [m.PREC_F64, m.PREC_MIXED])
def test_cg_accelerated_solve(torch, name, precision):
    """V-cycle-preconditioned CG reaches the same discrete solution, in no
    more cycles than the plain multigrid iteration."""
    c, plan, (X, Y, Z, u0), H = setup(torch, name, precision=precision, coarsest_max=1024,
                                      accel=m.ACCEL_CG)
    lam, st = plan.solve(u0, rtol=1e-12, max_cycles=120)
    assert st.status == m.MCWIND_OK and st.rel_res <= 1e-12, st.history()
    if name not in _lam_ref:
        _lam_ref[name] = oracle.solve(c)
    assert rel(lam.cpu().numpy().ravel(), _lam_ref[name]) <= 1e-10
    _, plan_mg, _, _ = setup(torch, name, precision=precision, coarsest_max=1024)
    _, st_mg = plan_mg.solve(u0, rtol=1e-12, max_cycles=120)
    assert st.cycles <= st_mg.cycles, (st.cycles, st_mg.cycles)


def test_cg_warm_start(torch):
    c, plan, (X, Y, Z, u0), _ = setup(torch, "ragged", precision=m.PREC_MIXED, coarsest_max=1024,
                                      accel=m.ACCEL_CG)
    lam, st_cold = plan.solve(u0, rtol=1e-10)
    u0b = torch.from_numpy(synth.perturb_wind(c.u0, 0)).to("cuda")
    lam_w, st_warm = plan.solve(u0b, lam=lam.clone(), rtol=1e-10, warm=True)
    lam_c, st_c = plan.solve(u0b, rtol=1e-10)
    assert st_warm.status == m.MCWIND_OK and st_warm.cycles < st_c.cycles
    assert rel(lam_w.cpu().numpy(), lam_c.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("accel", [m.ACCEL_NONE, m.ACCEL_CG])
@pytest.mark.parametrize("precision", [m.PREC_F64, m.PREC_MIXED])
def test_graph_replay_matches_direct_launches(torch, accel, precision):
    """Replaying the captured iteration graph gives bitwise the same solution
    and history as launching the same kernels directly."""
    _, pg, (X, Y, Z, u0), _ = setup(torch, "ragged", precision=precision, coarsest_max=1024,
                                    accel=accel, use_graphs=1)
    _, pd, _, _ = setup(torch, "ragged", precision=precision, coarsest_max=1024, accel=accel,
                        use_graphs=0)
    n0 = m.lib().mcwind_launch_count()
    a, sa = pg.solve(u0, rtol=1e-10, max_cycles=60)
    n1 = m.lib().mcwind_launch_count()
    b, sb = pd.solve(u0, rtol=1e-10, max_cycles=60)
    n2 = m.lib().mcwind_launch_count()
    assert sa.cycles == sb.cycles and sa.history() == sb.history()
    assert torch.equal(a, b)
    assert n1 - n0 == n2 - n1   # replayed kernels are counted too


@pytest.mark.parametrize("quad", [m.RHS_GAUSS8, m.RHS_CENTER1])
def test_wind_at_centers(torch, quad):
    """u0 given at the element centers: load vector, solution and recovered
    wind against the oracle's center-wind routines."""
    c = CASES["ragged"]
    rng = np.random.default_rng(4)
    uc = rng.normal(size=(3, c.nz, c.ny, c.nx)) + np.array([5.0, -2.0, 0.0])[:, None, None, None]
    X, Y, Z, ucd = to_dev(torch, c.X, c.Y, c.Z, uc)
    plan = m.Plan.for_case(c, rhs_quad=quad, u0_at=m.U0_CENTERS, precision=m.PREC_MIXED)
    plan.assemble(X, Y, Z)
    free = oracle.case_free_mask(c)
    f_ref = np.where(free, oracle.assemble_f_centers(c, uc, quad), 0.0)
    f = plan.rhs(ucd).cpu().numpy().ravel()
    assert np.abs(f - f_ref).max() <= 1e-12 * np.abs(f_ref).max()
    lam, st = plan.solve(ucd, rtol=1e-12, max_cycles=120)
    assert st.status == m.MCWIND_OK
    lam_ref = oracle.solve(c, f=oracle.assemble_f_centers(c, uc, quad))
    assert rel(lam.cpu().numpy().ravel(), lam_ref) <= 1e-10
    u = plan.recover(ucd, lam).cpu().numpy()
    assert rel(u, oracle.recover_centers(c, lam_ref, uc)) <= 1e-10


@pytest.mark.parametrize("arith,tol", [(m.ARITH_F64, 1e-13), (m.ARITH_DFLOAT, 1e-12)])
@pytest.mark.parametrize("name", ["ragged", "jitter", "aniso"])
def test_element_arithmetic(torch, arith, tol, name):
    """Stiffness and load vector in float64 and in float pairs against the
    oracle; both give the oracle's solution to 1e-10."""
    c, plan, (X, Y, Z, u0), H = setup(torch, name, coarsest_max=1024, element_arith=arith)
    dims = level_dims(plan, 0)
    ref = stencil_planes(H.K[0], dims)
    out = torch.empty((27, ref.shape[1]), dtype=torch.float64, device="cuda")
    m.mcwind_level_stencil(plan.handle, 0, m.PREC_F64, out)
    assert np.abs(out.cpu().numpy() - ref).max() <= tol * np.abs(ref[13]).max()
    f_ref = np.where(oracle.case_free_mask(c), oracle.assemble_f(c), 0.0)
    f = plan.rhs(u0).cpu().numpy().ravel()
    assert np.abs(f - f_ref).max() <= tol * np.abs(f_ref).max()
    lam, st = plan.solve(u0, rtol=1e-12, max_cycles=120)
    if name not in _lam_ref:
        _lam_ref[name] = oracle.solve(c)
    assert rel(lam.cpu().numpy().ravel(), _lam_ref[name]) <= 1e-10
    # recovery at the element centers (Eq. 7) from the same multiplier:
    # float pairs and float64 agree with the oracle element by element
    lam_h = lam.cpu().numpy().ravel()
    u = plan.recover(u0, lam, m.AT_CENTERS).cpu().numpy()
    u_ref = oracle.recover(c, lam_h, where=m.AT_CENTERS)
    assert np.abs(u - u_ref).max() <= tol * np.abs(u_ref).max()


@pytest.mark.parametrize("name", ["hill64", "aniso"])
def test_cycles_per_check(torch, name):
    """Mixed precision with 1, 2 and 3 V-cycles between float64 checks: each
    reaches the oracle's solution; the cycle count is a multiple of the
    spacing, and the history between two checks is their geometric
    interpolation."""
    c = CASES[name]
    if name not in _lam_ref:
        _lam_ref[name] = oracle.solve(c)
    counts = {}
    for k in (1, 2, 3):
        _, plan, (X, Y, Z, u0), _ = setup(torch, name, precision=m.PREC_MIXED,
                                          coarsest_max=1024, cycles_per_check=k)
        lam, st = plan.solve(u0, rtol=1e-12, max_cycles=120)
        assert st.status == m.MCWIND_OK and st.rel_res <= 1e-12, (k, st.history()[-3:])
        assert st.cycles % k == 0
        assert rel(lam.cpu().numpy().ravel(), _lam_ref[name]) <= 1e-10
        h = st.history()
        for q in range(k, st.cycles + 1, k):
            for r in range(1, k):
                want = h[q - k] * (h[q] / h[q - k]) ** (r / k)
                assert abs(h[q - k + r] - want) <= 1e-12 * want
        counts[k] = st.cycles
    # the float64 check does not change the cycle itself: the spacing costs at
    # most the cycles up to the next check
    assert counts[2] <= counts[1] + 2 and counts[3] <= counts[1] + 3, counts
