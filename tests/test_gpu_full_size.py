"""Full-size checks in the launch configuration the benchmark times.

At these sizes the oracle cannot solve, so it certifies instead: it
re-assembles K and f element by element in FP64 (its own code) and
evaluates ||f - K lambda_gpu|| / ||f||; it recomputes the load vector and
the recovered wind everywhere (512 x 512 x 16) or on sampled nodes and a
cropped window (3000 x 3000 x 15); and at a reduced size with the same
recipe it solves with its own multigrid to 1e-13 for an element-wise
lambda comparison."""
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


@pytest.mark.parametrize("a", [(1.0, 1.0, 1.0), (1.0, 1.0, 10.0)])
def test_hills_reduced_lambda_parity(torch, a):
    """Same recipe as the 512 x 512 x 16 case at 128 x 128 x 16 (10 hills)."""
    c = synth.random_hills(128, 128, 16, seed=0, a=a, n_hills=10)
    H = oracle.Hierarchy(c, rule="operator")
    f = oracle.assemble_f(c)
    lam_ref, hist = H.solve(f, rtol=1e-13, max_cycles=400)
    assert hist[-1] <= 1e-13
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    for prec, tol in ((m.PREC_F64, 1e-10), (m.PREC_MIXED, 1e-10)):
        plan = m.Plan.for_case(c, precision=prec)
        plan.assemble(X, Y, Z)
        lam, st = plan.solve(u0, rtol=1e-12, max_cycles=255)
        assert st.status == m.MCWIND_OK, st.history()
        assert rel(lam.cpu().numpy().ravel(), lam_ref) <= tol
        u = plan.recover(u0, lam).cpu().numpy()
        assert rel(u, oracle.recover(c, lam_ref)) <= tol


@pytest.mark.parametrize("a", [(1.0, 1.0, 1.0), (1.0, 1.0, 10.0)])
def test_hills_512(torch, a):
    c = synth.random_hills(512, 512, 16, seed=0, a=a)
    X, Y, Z, u0 = to_dev(torch, c.X, c.Y, c.Z, c.u0)
    f_ref = oracle.assemble_f(c, parallel=True)
    free = oracle.case_free_mask(c)
    lams = {}
    for prec in (m.PREC_F64, m.PREC_MIXED):
        plan = m.Plan.for_case(c, precision=prec)
        plan.assemble(X, Y, Z)
        f = plan.rhs(u0).cpu().numpy().ravel()
        assert np.abs(f - np.where(free, f_ref, 0.0)).max() <= 1e-12 * np.abs(f_ref).max()
        lam, st = plan.solve(u0, rtol=1e-10, max_cycles=255)
        assert st.status == m.MCWIND_OK, st.history()
        lam_h = lam.cpu().numpy().ravel()
        lams[prec] = lam_h
        # oracle residual certificate
        r = f_ref - oracle.apply_K(c, lam_h)
        cert = np.linalg.norm(r[free]) / np.linalg.norm(f_ref[free])
        assert cert <= 2e-10, (prec, cert, st.rel_res)
        u = plan.recover(u0, lam).cpu().numpy()
        assert rel(u, oracle.recover(c, lam_h)) <= 1e-12
        del plan
    assert rel(lams[m.PREC_MIXED], lams[m.PREC_F64]) <= 1e-6


@pytest.fixture(scope="module")
def full_case():
    c = synth.full_domain()
    return c, synth.perturb_wind(c.u0, 0)


@pytest.mark.parametrize("form", [m.OP_SEPARABLE, m.OP_STORED])
def test_full_domain(torch, full_case, form):
    """3000 x 3000 x 15 cells (1.44e8 nodes), mixed precision as benchmarked
    (separable operator), and with the stored operator."""
    c, u0n = full_case
    X, Y, Z, u0, u0b = to_dev(torch, c.X, c.Y, c.Z, c.u0, u0n)
    plan = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=form)
    plan.assemble(X, Y, Z)
    lam, st = plan.solve(u0, rtol=1e-8, max_cycles=100)
    assert st.status == m.MCWIND_OK, (st.history(), st.rate)
    lam_w = lam.clone()
    lam_w, st_w = plan.solve(u0b, lam=lam_w, rtol=1e-8, warm=True)
    assert st_w.status == m.MCWIND_OK and st_w.cycles <= st.cycles
    free = oracle.case_free_mask(c)
    # sampled stencil rows against the oracle's element-by-element rows
    rng = np.random.default_rng(0)
    Nx, Ny, Nz = c.nx + 1, c.ny + 1, c.nz + 1
    pts = [(int(rng.integers(1, Nx - 1)), int(rng.integers(1, Ny - 1)), int(rng.integers(0, Nz - 1)))
           for _ in range(300)] + [(1, 1, 0), (Nx - 2, Ny - 2, Nz - 2), (1, Ny - 2, 0), (Nx - 2, 1, Nz - 2)]
    st_dev = torch.empty((27, Nz * Ny * Nx), dtype=torch.float64, device="cuda")
    m.mcwind_level_stencil(plan.handle, 0, m.PREC_F64, st_dev)
    ids = torch.tensor([(k * Ny + j) * Nx + i for (i, j, k) in pts], device="cuda")
    rows = st_dev[:, ids].cpu().numpy()
    del st_dev
    for q, (i, j, k) in enumerate(pts):
        ref = oracle.stencil_row(c, i, j, k)
        for s in range(27):
            ii, jj, kk = i + s % 3 - 1, j + (s // 3) % 3 - 1, k + s // 9 - 1
            if not (1 <= ii <= Nx - 2 and 1 <= jj <= Ny - 2 and 0 <= kk <= Nz - 2):
                ref[s] = 0.0
        assert np.abs(rows[:, q] - ref).max() <= 1e-12 * abs(ref[13]), (i, j, k)
    # oracle residual certificates of the cold and warm solutions
    for uu, ll, ss in ((c.u0, lam, st), (u0n, lam_w, st_w)):
        lh = ll.cpu().numpy().ravel()
        f_ref = oracle.assemble_f(c, u0=uu, parallel=True)
        r = f_ref - oracle.apply_K(c, lh)
        cert = np.linalg.norm(r[free]) / np.linalg.norm(f_ref[free])
        assert cert <= 1.05e-8, (cert, ss.rel_res)
        assert abs(cert - ss.rel_res) <= 1e-3 * ss.rel_res + 1e-13
    # recovered wind on a cropped window (element-local, so the crop is exact)
    u = plan.recover(u0, lam).cpu().numpy()
    lh = lam.cpu().numpy()
    i0, j0, w = 1400, 1450, 48
    sub = synth.Case("crop", w, w, c.nz, c.a, c.X[:, j0:j0 + w + 1, i0:i0 + w + 1].copy(),
                     c.Y[:, j0:j0 + w + 1, i0:i0 + w + 1].copy(),
                     c.Z[:, j0:j0 + w + 1, i0:i0 + w + 1].copy(),
                     c.u0[:, :, j0:j0 + w + 1, i0:i0 + w + 1].copy(), c.h1, c.h3)
    u_ref = oracle.recover(sub, lh[:, j0:j0 + w + 1, i0:i0 + w + 1].copy())
    assert np.abs(u[:, :, j0:j0 + w, i0:i0 + w] - u_ref).max() <= 1e-12 * np.abs(u_ref).max()
    del plan, X, Y, Z, u0, u0b
    torch.cuda.empty_cache()
