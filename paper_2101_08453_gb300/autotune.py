"""Per-domain tuning of the solver: smoothing sweeps and smoother block shape.

For each plan, every candidate (nu_pre = nu_post = nu, smoother thread-block
height) is timed on the device (CUDA events around mcwind_solve to the
requested tolerance, after one untimed warm-up solve), and the fastest
setting is kept on the plan (mcwind_plan_set_tuning).  Sweeps change the
convergence rate and the cost per cycle; the block height changes how well
the smoother's launch fills the GPU on that grid.  The solution does not
depend on the choice beyond the tolerance.
"""
from __future__ import annotations

import itertools

from . import mcwind_plan_set_tuning, mcwind_solve

SWEEPS = (1, 2, 3)
BLOCK_ROWS = (2, 4, 8)


def time_solve(torch, plan, u0, lam, rtol, max_cycles=150):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lam.zero_()
    e0.record()
    rc, st = mcwind_solve(plan.handle, u0, lam, rtol, max_cycles, 0)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, st


def tune_plan(plan, u0, rtol=1e-8, sweeps=SWEEPS, rows=BLOCK_ROWS):
    """Time each (nu, rows) candidate on this plan and set the fastest.
    Returns (best (nu, rows), {candidate: (seconds, cycles, status)})."""
    import torch
    lam = torch.zeros(plan.node_shape, dtype=torch.float64, device="cuda")
    if plan.options.op_form == 1:
        rows = (4,)   # the separable form's staged smoother has a fixed block shape
    table = {}
    for nu, r in itertools.product(sweeps, rows):
        mcwind_plan_set_tuning(plan.handle, nu, nu, r)
        time_solve(torch, plan, u0, lam, rtol)   # warm-up (captures the iteration graph)
        t, st = time_solve(torch, plan, u0, lam, rtol)
        table[(nu, r)] = (t, st.cycles, st.status)
    ok = {k: v for k, v in table.items() if v[2] == 0}
    best = min(ok or table, key=lambda k: table[k][0])
    mcwind_plan_set_tuning(plan.handle, best[0], best[0], best[1])
    return best, table


def tune_batch(plans, u0s, rtol=1e-8, **kw):
    """tune_plan for every (plan, u0) pair; returns the chosen settings."""
    return [tune_plan(p, u, rtol, **kw)[0] for p, u in zip(plans, u0s)]
