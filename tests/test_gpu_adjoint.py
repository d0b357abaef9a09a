"""Gradients through the hand-written adjoint (torch.autograd.Function):
against the oracle's dense (probed-Jacobian) gradient on small grids, and
against central finite differences of the GPU forward map on the
256 x 256 x 12 case with a loss over 1 % of the element centers."""
import numpy as np
import pytest

import oracle
import paper_2101_08453_gb300 as m
import synth
from gpu_cases import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    m.build.build()
    return t


def grads(torch, model, u0, a, gu):
    from paper_2101_08453_gb300.autograd import downscale
    u0t = u0.clone().requires_grad_(True)
    la = torch.log(torch.tensor(a, dtype=torch.float64, device="cuda")).requires_grad_(True)
    u = downscale(u0t, la, model)
    (u * gu).sum().backward()
    return u.detach(), u0t.grad.detach(), la.grad.detach()


@pytest.mark.parametrize("maker", [
    lambda: synth.single_hill(5, 4, 3, sigma=40.0, height=20.0, noise=0.5, a=(1.0, 1.3, 2.0)),
    lambda: synth.jittered(4, 4, 3, seed=6, a=(2.0, 1.0, 0.7)),
])
def test_adjoint_matches_oracle_dense_gradient(torch, maker):
    from paper_2101_08453_gb300.autograd import WindModel
    c = maker()
    rng = np.random.default_rng(1)
    gu = rng.normal(size=(3, c.nz, c.ny, c.nx))
    g0_ref, gl_ref = oracle.dense_wind_gradient(c, gu)
    for prec in (m.PREC_F64, m.PREC_MIXED):
        model = WindModel.for_case(c, precision=prec, rtol=1e-13, coarsest_max=8)
        u0 = torch.from_numpy(c.u0).cuda()
        u, g0, gl = grads(torch, model, u0, c.a, torch.from_numpy(gu).cuda())
        assert rel(u.cpu().numpy(), oracle.recover(c, oracle.solve(c))) <= 1e-10
        assert rel(g0.cpu().numpy(), g0_ref) <= 1e-9
        assert np.allclose(gl.cpu().numpy(), gl_ref, rtol=1e-6, atol=1e-7 * max(map(abs, gl_ref)))
        assert abs(float(gl.sum())) <= 1e-8 * float(gl.abs().max())


def test_adjoint_config5_finite_differences(torch):
    """256 x 256 x 12 cells, random hills, log-law wind + noise; loss =
    sum over 1 % random element centers of |u - u_obs|^2 with u_obs the
    solution for a second seeded wind; central differences (h = 1e-6 and an
    exact large step for u0, Richardson-extrapolated for log a)."""
    from paper_2101_08453_gb300.autograd import WindModel, downscale
    c = synth.random_hills(256, 256, 12, seed=5, n_hills=10, hmax=300.0)
    c2 = synth.random_hills(256, 256, 12, seed=6, n_hills=10, hmax=300.0)
    model = WindModel.for_case(c, precision=m.PREC_F64, rtol=1e-13, max_cycles=250)
    a = (1.0, 1.0, 1.0)
    u0 = torch.from_numpy(c.u0).cuda()
    u_obs, _, _ = model.forward(torch.from_numpy(c2.u0).cuda(), a)
    rng = np.random.default_rng(7)
    ne = c.nx * c.ny * c.nz
    obs = torch.from_numpy(rng.choice(ne, size=ne // 100, replace=False)).cuda()

    def loss_of(u):
        d = (u - u_obs).reshape(3, -1)[:, obs]
        return (d * d).sum()

    u0t = u0.clone().requires_grad_(True)
    la = torch.zeros(3, dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss_of(downscale(u0t, la, model))
    L.backward()
    g0, gl = u0t.grad, la.grad
    assert abs(float(gl.sum())) <= 1e-7 * float(gl.abs().max())

    def loss_at(u0v, av):
        u, _, _ = model.forward(u0v, av)
        return float(loss_of(u))

    # u is affine in u0, so the loss is quadratic in u0 and a central
    # difference is exact for any step; a large step keeps the difference far
    # above the forward solve's rounding (the loss is ~1e5).
    pts = [(0, 3, 100, 100), (1, 0, 57, 200), (2, 5, 128, 31)]
    scale = float(g0.abs().max())
    for h, tol in ((1.0, 1e-6), (1e-6, 1e-3)):
        for idx in pts:
            up, um = u0.clone(), u0.clone()
            up[idx] += h
            um[idx] -= h
            fd = (loss_at(up, a) - loss_at(um, a)) / (2 * h)
            assert fd == pytest.approx(float(g0[idx]), rel=tol, abs=tol * scale), (h, idx)
    # log a: Richardson-extrapolated central differences, error O(h^4)
    def cd(d, h):
        ap, am = list(a), list(a)
        ap[d] *= np.exp(h)
        am[d] *= np.exp(-h)
        return (loss_at(u0, ap) - loss_at(u0, am)) / (2 * h)

    for d in range(3):
        h = 2e-3
        fd = (4 * cd(d, h / 2) - cd(d, h)) / 3
        assert fd == pytest.approx(float(gl[d]), rel=1e-6, abs=1e-6 * float(gl.abs().max())), d
