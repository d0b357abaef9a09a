"""The allocation-free residual-norm entry point.

mcwind_residual_norm_noalloc serves callers that cannot call cudaMalloc
when they check a solution (for example code running while a CUDA graph is
captured, or a host model whose own pool owns all device memory).  It must
give the same norms as the regular path -- the residual from
mcwind_level_residual, normed over the free nodes -- on consecutive calls
that share its static scratch array."""
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


@pytest.mark.gpu
def test_noalloc_norms_match_level_residual():
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
        norms = torch.empty(2, dtype=torch.float64, device="cuda")
        # two calls in a row on different iterates, each against the regular path
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
        del plan
