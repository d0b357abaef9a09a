"""The allocation-free residual-norm entry point.

mcwind_residual_norm_noalloc serves callers that cannot call cudaMalloc
when they check a solution (for example a host model whose own pool owns
all device memory, or a loop in which an allocation, which may synchronize
the device, is not allowed).  It must give the norms of the regular path --
the residual from mcwind_level_residual, normed over the free nodes -- and
of the oracle's element-by-element residual, on consecutive calls that
share its static scratch array."""
import numpy as np
import pytest

import oracle
import paper_2101_08453_gb300 as m
import synth
from gpu_cases import to_dev


def test_rejects_plans_beyond_its_static_scratch():
    """No device work is needed to refuse a too-large finest grid."""
    m.build.build()
    h, _ = m.mcwind_plan_create(8000, 8000, 4, (1, 1, 1), 30.0, [5.0, 6.0, 7.0, 8.0])
    try:
        import ctypes
        p = ctypes.c_void_p(256)
        rc = m.lib().mcwind_residual_norm_noalloc(h, p, p, p, None)
        assert rc == m.MCWIND_EINVAL
    finally:
        m.mcwind_plan_destroy(h)


def test_binding_rejects_short_buffers_before_the_library():
    """A norms buffer of one value, or a lambda of the wrong node count, is
    refused on the host before any pointer reaches the library."""
    import torch
    m.build.build()
    h, _ = m.mcwind_plan_create(16, 12, 4, (1, 1, 1), 30.0, [5.0, 6.0, 7.0, 8.0])
    try:
        n = 17 * 13 * 5
        f = torch.zeros(n, dtype=torch.float64)
        with pytest.raises(ValueError, match="norms"):
            m.mcwind_residual_norm_noalloc(h, f, f, torch.zeros(1, dtype=torch.float64))
        with pytest.raises(ValueError, match="lam"):
            m.mcwind_residual_norm_noalloc(h, f, f[:-1], torch.zeros(2, dtype=torch.float64))
    finally:
        m.mcwind_plan_destroy(h)


@pytest.mark.gpu
def test_noalloc_norms_match_level_residual_and_oracle():
    import torch
    assert torch.cuda.is_available()
    m.build.build()
    cases = [synth.single_hill(149, 43, 6, sigma=600.0, height=120.0, noise=0.3),
             synth.jittered(37, 30, 5, seed=4)]
    for c in cases:
        X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
        plan = m.Plan.for_case(c)
        plan.assemble(X, Y, Z)
        f = plan.rhs(u0)
        lam, _ = plan.solve(u0, rtol=1e-4, max_cycles=50)
        free = oracle.case_free_mask(c)
        f_oracle = oracle.assemble_f(c)
        norms = torch.empty(2, dtype=torch.float64, device="cuda")
        # two calls in a row on different iterates, each against the regular
        # path (same operator, same f: equal up to summation order) and against
        # the oracle (its own K applied element by element to the same iterate,
        # its own f).  The library's operator and load vector agree with the
        # oracle's to about 1e-13 of their scale, and ||r|| is about 1e-4 of
        # ||f||, so ||r|| may differ by about 1e-9 relative: tolerance 1e-8.
        for scale in (1.0, 0.5):
            x = lam * scale
            r = torch.empty_like(f)
            m.mcwind_level_residual(plan.handle, 0, m.PREC_F64, x, f, r)
            rh = r.cpu().numpy().ravel()[free]
            fh = f.cpu().numpy().ravel()[free]
            norms.fill_(-1.0)
            m.mcwind_residual_norm_noalloc(plan.handle, f, x, norms)
            got = norms.cpu().numpy()
            assert got[0] == pytest.approx(np.linalg.norm(fh), rel=1e-12)
            assert got[1] == pytest.approx(np.linalg.norm(rh), rel=1e-12)
            r_or, f_or = oracle.residual_norms(c, x.cpu().numpy(), f=f_oracle)
            assert got[0] == pytest.approx(f_or, rel=1e-10)
            assert got[1] == pytest.approx(r_or, rel=1e-8)
        del plan
