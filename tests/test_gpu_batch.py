"""Batches of independent domains of uneven sizes (one graph launch per
solve: a conditional loop with an IF node per domain): every domain's
solution against the oracle, the batch against one-at-a-time solves, and
the autotuner."""
import numpy as np
import pytest

import oracle
import paper_2101_08453_gb300 as m
import synth
from gpu_cases import rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    m.build.build()
    return t


def make(torch, cases, precision=m.PREC_MIXED, op_form=m.OP_STORED):
    plans, u0s = [], []
    for c in cases:
        X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
        p = m.Plan.for_case(c, precision=precision, op_form=op_form)
        p.assemble(X, Y, Z)
        plans.append(p)
        u0s.append(u0)
    return plans, u0s


@pytest.mark.parametrize("op_form", [m.OP_STORED, m.OP_SEPARABLE])
def test_batch_matches_oracle_per_domain(torch, op_form):
    """One graph launch solves every domain (a conditional loop with an IF
    node per domain): each to the oracle's lambda, and bitwise to its own
    mcwind_solve."""
    cases = synth.batch_domains(n=7, seed=1, nmin=12, nmax=40, zmin=3, zmax=8)
    plans, u0s = make(torch, cases, op_form=op_form)
    batch = m.Batch(plans)
    lams, stats = batch.solve(u0s, rtol=1e-11, max_cycles=200)
    for c, lam, st in zip(cases, lams, stats):
        assert st.status == m.MCWIND_OK and st.rel_res <= 1e-11, (c.name, st.history()[-3:])
        err = rel(lam.cpu().numpy().ravel(), oracle.solve(c))
        assert err <= 1e-9, (c.name, err)
    # the same domains one at a time give bitwise the same solutions
    for p, u0, lam, st in zip(plans, u0s, lams, stats):
        lam1, st1 = p.solve(u0, rtol=1e-11, max_cycles=200)
        assert st1.cycles == st.cycles and torch.equal(lam1, lam)


def test_batch_cycles_and_warm_start(torch):
    cases = synth.batch_domains(n=5, seed=2, nmin=16, nmax=48, zmin=4, zmax=10)
    plans, u0s = make(torch, cases, precision=m.PREC_F64)
    batch = m.Batch(plans)
    lams, stats = batch.solve(u0s, rtol=1e-8)
    for p, u0, st in zip(plans, u0s, stats):
        _, st1 = p.solve(u0, rtol=1e-8)
        assert st.cycles == st1.cycles and st.history() == st1.history()
    u0b = [torch.from_numpy(synth.perturb_wind(c.u0, 0)).to("cuda") for c in cases]
    _, warm = batch.solve(u0b, lams=[l.clone() for l in lams], rtol=1e-8, warm=True)
    _, cold = batch.solve(u0b, rtol=1e-8)
    assert all(w.status == 0 for w in warm)
    assert sum(w.cycles for w in warm) < sum(c.cycles for c in cold)


def test_batch_rejects_bad_input(torch):
    cases = synth.batch_domains(n=2, seed=3, nmin=10, nmax=12, zmin=3, zmax=4)
    plans, u0s = make(torch, cases)
    b = m.Batch(plans)
    with pytest.raises(m.MCWindError):
        m.Batch([plans[0]])            # already in a batch
    del b
    cg = m.Plan.for_case(cases[0], accel=m.ACCEL_CG)
    with pytest.raises(m.MCWindError):
        m.Batch([cg])                  # the batch runs the plain cycle


def test_autotune_keeps_solution(torch):
    from paper_2101_08453_gb300 import autotune
    c = synth.batch_domains(n=1, seed=4, nmin=60, nmax=60, zmin=10, zmax=10)[0]
    plans, u0s = make(torch, [c])
    best, table = autotune.tune_plan(plans[0], u0s[0], rtol=1e-9)
    assert best in table and table[best][2] == 0
    assert len(table) == len(autotune.SWEEPS) * len(autotune.BLOCK_ROWS)
    lam, st = plans[0].solve(u0s[0], rtol=1e-11, max_cycles=200)
    assert st.status == 0
    assert rel(lam.cpu().numpy().ravel(), oracle.solve(c)) <= 1e-9
