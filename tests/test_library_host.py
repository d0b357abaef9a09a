"""Host-side checks of the C library (no GPU needed): it loads, exports every
entry point its header declares, rejects bad arguments, and its planner
reproduces the semicoarsening hierarchy of Sec. 3 as the oracle plans it."""
import os
import re

import pytest

import oracle
import paper_2101_08453_gb300 as m
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    m.build.build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mcwind.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcwind_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    L = m.lib()
    syms = declared_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(L, s), s


def test_strerror_names_codes():
    L = m.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.mcwind_strerror(code)
    assert L.mcwind_strerror(-2) != L.mcwind_strerror(-3)


@pytest.mark.parametrize("args", [
    dict(nx=1, ny=4, nz=3), dict(nx=4, ny=1, nz=3), dict(nx=4, ny=4, nz=0),
    dict(nx=4, ny=4, nz=200),
])
def test_plan_rejects_bad_sizes(args):
    with pytest.raises(m.MCWindError) as e:
        m.mcwind_plan_create(args["nx"], args["ny"], args["nz"], (1, 1, 1), 30.0,
                             [5.0] * max(1, args["nz"]))
    assert e.value.code == m.MCWIND_EINVAL


@pytest.mark.parametrize("bad", [
    dict(a=(0, 1, 1)), dict(a=(1, -1, 1)), dict(h1=0.0), dict(h3=[5, 0, 5]),
    dict(opt=dict(precision=3)), dict(opt=dict(nu_pre=0, nu_post=0)),
    dict(opt=dict(coarsest_max=0)), dict(opt=dict(coarsest_max=100000)),
    dict(opt=dict(coarsen_rule=7)), dict(opt=dict(rhs_quad=2)),
    dict(opt=dict(accel=2)), dict(opt=dict(accel=1, post_reverse=0)),
    dict(opt=dict(use_graphs=2)),
])
def test_plan_rejects_bad_options(bad):
    a = bad.get("a", (1, 1, 1))
    h1 = bad.get("h1", 30.0)
    h3 = bad.get("h3", [5.0, 6.0, 7.0])
    o = m.default_options(**bad.get("opt", {}))
    with pytest.raises(m.MCWindError) as e:
        m.mcwind_plan_create(8, 8, 3, a, h1, h3, o)
    assert e.value.code == m.MCWIND_EINVAL


def test_null_pointer_entry_points_return_einval():
    L = m.lib()
    h, _ = m.mcwind_plan_create(8, 8, 3, (1, 1, 1), 30.0, [5.0, 6.0, 7.0])
    try:
        assert L.mcwind_assemble(h, None, None, None, None, None) == m.MCWIND_EINVAL
        assert L.mcwind_solve(h, None, None, 1e-8, 10, 0, None, None) == m.MCWIND_EINVAL
        assert L.mcwind_recover(h, None, None, None, 0, None) == m.MCWIND_EINVAL
        assert L.mcwind_solve(None, None, None, 1e-8, 10, 0, None, None) == m.MCWIND_EINVAL
        # not assembled yet: state error, not a CUDA call
        import ctypes
        p = ctypes.c_void_p(256)
        assert L.mcwind_solve(h, p, p, 1e-8, 10, 0, None, None) == m.MCWIND_ESTATE
        assert L.mcwind_level_smooth(h, 0, 0, p, p, 1, 0, None) == m.MCWIND_ESTATE
    finally:
        m.mcwind_plan_destroy(h)


CASES = [
    ("hill64", lambda: synth.single_hill(), (1, 1, 1), 0, 1024),
    ("hills512", lambda: synth.single_hill(512, 512, 16), (1, 1, 1), 0, 1024),
    ("hills512_a10_paper", lambda: synth.single_hill(512, 512, 16), (1, 1, 10), 0, 1024),
    ("hills512_a10_op", lambda: synth.single_hill(512, 512, 16), (1, 1, 10), 1, 1024),
    ("odd", lambda: synth.single_hill(37, 23, 7), (1, 1, 1), 0, 16),
    ("odd_a4", lambda: synth.single_hill(45, 61, 13), (1, 2, 4), 1, 64),
    ("thick", lambda: synth.flat_box(40, 40, 5, dz=200.0, stretch=1.0), (1, 1, 1), 0, 32),
]


@pytest.mark.parametrize("name,maker,a,rule,cmax", CASES, ids=[c[0] for c in CASES])
def test_planner_matches_oracle(name, maker, a, rule, cmax):
    c = maker()
    ref = oracle.plan_levels(c.nx, c.ny, c.nz, c.h1, c.h3, a, "paper" if rule == 0 else "operator", cmax)
    plan = m.Plan(c.nx, c.ny, c.nz, a, c.h1, c.h3, coarsen_rule=rule, coarsest_max=cmax)
    assert plan.num_levels == len(ref)
    for l, want in enumerate(ref):
        got = plan.level(l)
        for key in ("Nx", "Ny", "Nz", "hx", "hy", "kmap"):
            if key in want:
                assert got[key] == want[key], (l, key, got, want)


@pytest.mark.parametrize("rule,key", [(0, "levels_paper"), (1, "levels_operator")])
def test_planner_matches_hand_derived_aniso64(rule, key):
    """The library's planner against the hand-derived hierarchies of the
    semicoarsening rule of Sec. 3 (a = (0.5, 1, 10), both ratio readings)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "plan_aniso64.json")))
    c = g["case"]
    h3 = [c["h3_first"] * c["h3_growth"] ** k for k in range(c["nz"])]
    plan = m.Plan(c["nx"], c["ny"], c["nz"], c["a"], c["h1"], h3, coarsen_rule=rule,
                  coarsest_max=c["coarsest_max"])
    assert plan.num_levels == len(g[key])
    for l, want in enumerate(g[key]):
        got = plan.level(l)
        for name, value in want.items():
            assert got[name] == value, (l, name, got, want)


def test_separable_form_needs_mixed_precision():
    h3 = [5.0, 6.0, 7.0, 8.0]
    with pytest.raises(m.MCWindError) as e:
        m.mcwind_plan_create(64, 48, 4, (1, 1, 1), 30.0, h3,
                             m.default_options(op_form=m.OP_SEPARABLE))
    assert e.value.code == m.MCWIND_EINVAL
    with pytest.raises(m.MCWindError):
        m.mcwind_plan_create(64, 48, 4, (1, 1, 1), 30.0, h3,
                             m.default_options(precision=m.PREC_MIXED, op_form=7))


def test_separable_workspace_at_full_size():
    """Memory per grid point (Sec. 1, requirement 3): at 3000 x 3000 x 15 the
    separable form keeps the float64 operator of the finest level (for the
    float64 residual) and drops the float32 copy and the stored coarse
    operators: about half the stored form's workspace."""
    h3 = synth.layer_thicknesses(15)
    _, stored = m.mcwind_plan_create(3000, 3000, 15, (1, 1, 1), 30.0, h3,
                                     m.default_options(precision=m.PREC_MIXED))
    _, sep = m.mcwind_plan_create(3000, 3000, 15, (1, 1, 1), 30.0, h3,
                                  m.default_options(precision=m.PREC_MIXED,
                                                    op_form=m.OP_SEPARABLE))
    nodes = 3001 * 3001 * 16
    assert sep < 0.6 * stored, (sep, stored)
    assert sep / nodes < 420, sep / nodes   # bytes per node, all levels


def test_cg_workspace_is_larger():
    h3 = [5.0, 6.0, 7.0, 8.0]
    _, ws0 = m.mcwind_plan_create(64, 48, 4, (1, 1, 1), 30.0, h3)
    _, ws1 = m.mcwind_plan_create(64, 48, 4, (1, 1, 1), 30.0, h3, m.default_options(accel=1))
    assert ws1 > ws0


def test_full_domain_hierarchy_shape():
    h3 = synth.layer_thicknesses(15)
    plan = m.Plan(3000, 3000, 15, (1, 1, 1), 30.0, h3, precision=m.PREC_MIXED)
    ref = oracle.plan_levels(3000, 3000, 15, 30.0, h3, (1, 1, 1))
    assert plan.num_levels == len(ref)
    last = plan.level(plan.num_levels - 1)
    assert (last["Nx"] - 2) * (last["Ny"] - 2) * (last["Nz"] - 1) <= 1024
    assert plan.workspace_bytes < 150e9


def test_batch_rejects_bad_arguments_without_gpu():
    import ctypes
    L = m.lib()
    assert L.mcwind_batch_workspace_bytes(0) == 0
    assert L.mcwind_batch_workspace_bytes(96) >= 96 * 16
    h, _ = m.mcwind_plan_create(8, 8, 3, (1, 1, 1), 30.0, [5.0, 6.0, 7.0])
    hc, _ = m.mcwind_plan_create(8, 8, 3, (1, 1, 1), 30.0, [5.0, 6.0, 7.0], m.default_options(accel=1))
    try:
        out = ctypes.c_void_p()
        ws = ctypes.c_void_p(256)
        two = (ctypes.c_void_p * 2)(h, h)
        assert L.mcwind_batch_create(2, two, ws, ctypes.byref(out)) == m.MCWIND_EINVAL
        one = (ctypes.c_void_p * 1)(hc)
        assert L.mcwind_batch_create(1, one, ws, ctypes.byref(out)) == m.MCWIND_EINVAL
        assert L.mcwind_batch_create(0, one, ws, ctypes.byref(out)) == m.MCWIND_EINVAL
        assert L.mcwind_plan_set_tuning(h, 0, 0, 4) == m.MCWIND_EINVAL
        assert L.mcwind_plan_set_tuning(h, 2, 2, 3) == m.MCWIND_EINVAL
        assert L.mcwind_plan_set_tuning(h, 3, 3, 8) == m.MCWIND_OK
    finally:
        m.mcwind_plan_destroy(h)
        m.mcwind_plan_destroy(hc)


def test_plan_query_reports_the_check_interval_in_use():
    """cycles_per_check 0 means the default interval: 6 V-cycles per float64
    check in mixed precision, 1 in float64; an explicit value is kept."""
    h3 = [5.0, 6.0, 7.2, 8.64]
    for prec, given, want in ((m.PREC_MIXED, 0, 6), (m.PREC_F64, 0, 1), (m.PREC_MIXED, 3, 3)):
        h, _ = m.mcwind_plan_create(16, 12, 4, (1, 1, 1), 30.0, h3,
                                    m.default_options(precision=prec, cycles_per_check=given))
        try:
            assert m.plan_options(h).cycles_per_check == want
        finally:
            m.lib().mcwind_plan_destroy(h)


def test_plan_bound_wrappers_refuse_short_buffers():
    """Every plan-bound wrapper checks each tensor's element count against
    the plan before any pointer reaches the library (no device needed)."""
    torch = pytest.importorskip("torch")
    h3 = [5.0, 6.0, 7.2, 8.64]
    h, _ = m.mcwind_plan_create(16, 12, 4, (1, 1, 1), 30.0, h3,
                                m.default_options(precision=m.PREC_MIXED, coarsest_max=64))
    try:
        assert m.mcwind_plan_num_levels(h) >= 2
        nodes = 17 * 13 * 5
        cells = 16 * 12 * 4
        ok = torch.zeros(nodes, dtype=torch.float64)
        short = torch.zeros(nodes - 1, dtype=torch.float64)
        u0 = torch.zeros(3 * nodes, dtype=torch.float64)
        calls = [
            ("lam", lambda: m.mcwind_solve(h, u0, short)),
            ("u0", lambda: m.mcwind_solve(h, u0[:-1], ok)),
            ("u", lambda: m.mcwind_recover(h, u0, ok, torch.zeros(3 * cells - 1, dtype=torch.float64))),
            ("f", lambda: m.mcwind_rhs(h, u0, short)),
            ("x", lambda: m.mcwind_level_residual(h, 0, m.PREC_MIXED, short, ok, ok)),
            ("r", lambda: m.mcwind_level_residual(h, 0, m.PREC_MIXED, ok, ok, short)),
            ("x", lambda: m.mcwind_level_smooth(h, 0, m.PREC_MIXED, short, ok, 1, m.FORWARD)),
            ("fc", lambda: m.mcwind_level_residual_restrict(h, 0, m.PREC_MIXED, ok, ok, short)),
            ("norms", lambda: m.mcwind_residual_norm_noalloc(h, ok, ok, torch.zeros(1, dtype=torch.float64))),
        ]
        for name, call in calls:
            with pytest.raises(ValueError, match=name):
                call()
    finally:
        m.lib().mcwind_plan_destroy(h)
