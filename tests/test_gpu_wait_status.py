"""Bounded device waits report a status instead of hanging the GPU.

Every wait of the staged kernels (a tile that has not arrived, a stage not
yet released) gives up after a wall-clock limit, sets the plan's device
status word and returns; the host reads it as MCWIND_ETIMEOUT.  The test
makes a wait run out on purpose -- a barrier that nothing completes, waited
on for 2 ms by the same bounded-wait routine -- and checks that the status
comes back, that the GPU stays usable, that solves and batch solves on the
plan report it, and that assembling again clears it."""
import pytest

import paper_2101_08453_gb300 as m
import synth
from gpu_cases import to_dev

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_cleared():
    import torch
    assert torch.cuda.is_available()
    m.build.build()
    c = synth.single_hill(24, 20, 5, sigma=150.0, height=60.0)
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    plan = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=m.OP_SEPARABLE)
    plan.assemble(X, Y, Z)
    lam, st = plan.solve(u0, rtol=1e-8)
    assert st.status == m.MCWIND_OK
    assert m.mcwind_plan_wait_selftest(plan.handle, 2000) == m.MCWIND_ETIMEOUT
    # the context is intact
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
    # the plan's solves report the status until it is assembled again
    with pytest.raises(m.MCWindError) as e:
        plan.solve(u0, rtol=1e-8)
    assert e.value.code == m.MCWIND_ETIMEOUT
    batch = m.Batch([plan])
    rc_lams = torch.zeros(plan.node_shape, dtype=torch.float64, device="cuda")
    rc = m.lib().mcwind_batch_solve(
        batch.handle, (m._vp * 1)(u0.data_ptr()), (m._vp * 1)(rc_lams.data_ptr()), 1e-8, 50, 0,
        None, m._stream(None))
    assert rc == m.MCWIND_ETIMEOUT
    del batch
    plan.assemble(X, Y, Z)
    lam2, st2 = plan.solve(u0, rtol=1e-8)
    assert st2.status == m.MCWIND_OK and torch.equal(lam, lam2)
