"""Differentiable downscaling: u(u0, log a) as a torch.autograd.Function.

Forward: lambda = K(a)^{-1} f(u0) (Eq. 5) by the multigrid solve, then
u = u0 + A^{-1} grad lambda at the element centers (Eq. 3).  Backward: the
hand-written adjoint of the C library -- one more solve with the same
(self-adjoint) operator, mu = K^{-1} G^T A^{-1} (dl/du), then
dl/du0 = C^T dl/du - I^T B^T mu and dl/dlog a_d = 2 a_d^-2 (mu^T K_d lambda -
sum_centers (dl/du)_d d_d lambda).  A change of a changes K, so plans are
kept per penalty vector.
"""
from __future__ import annotations

import torch

from . import (PREC_F64, Plan, mcwind_adjoint_finish, mcwind_recover, mcwind_recover_adjoint,
               mcwind_solve, mcwind_solve_rhs)


class WindModel:
    """A fixed terrain-following grid on the device; assembled plans per a."""

    def __init__(self, nx, ny, nz, h1, h3, X, Y, Z, precision=PREC_F64, rtol=1e-12,
                 max_cycles=200, **options):
        self.dims = (int(nx), int(ny), int(nz))
        self.h1, self.h3 = float(h1), [float(v) for v in h3]
        self.geometry = (X, Y, Z)
        self.precision, self.rtol, self.max_cycles = precision, float(rtol), int(max_cycles)
        self.options = options
        self._plans = {}

    @classmethod
    def for_case(cls, case, **kw):
        X, Y, Z = (torch.from_numpy(v).to("cuda") for v in (case.X, case.Y, case.Z))
        return cls(case.nx, case.ny, case.nz, case.h1, case.h3, X, Y, Z, **kw)

    def plan_for(self, a):
        key = tuple(float(v) for v in a)
        if key not in self._plans:
            p = Plan(*self.dims, key, self.h1, self.h3, precision=self.precision, **self.options)
            p.assemble(*self.geometry)
            self._plans[key] = p
        return self._plans[key]

    def forward(self, u0, a):
        """(u at the centers, lambda) without autograd."""
        plan = self.plan_for(a)
        lam = torch.zeros(plan.node_shape, dtype=torch.float64, device="cuda")
        rc, st = mcwind_solve(plan.handle, u0, lam, self.rtol, self.max_cycles, 0)
        if st.status != 0:
            raise RuntimeError(f"forward solve did not converge: {st.history()[-3:]}")
        u = torch.empty((3, self.dims[2], self.dims[1], self.dims[0]), dtype=torch.float64, device="cuda")
        mcwind_recover(plan.handle, u0, lam, u)
        return u, lam, plan


class Downscale(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, log_a, model):
        a = [float(v) for v in torch.exp(log_a.detach()).cpu().tolist()]
        u, lam, plan = model.forward(u0.detach().contiguous(), a)
        ctx.save_for_backward(lam)
        ctx.plan, ctx.model = plan, model
        return u

    @staticmethod
    def backward(ctx, gu):
        (lam,) = ctx.saved_tensors
        plan, model = ctx.plan, ctx.model
        gu = gu.detach().to(torch.float64).contiguous()
        h = torch.empty(plan.node_shape, dtype=torch.float64, device="cuda")
        du0 = torch.empty((3,) + tuple(plan.node_shape), dtype=torch.float64, device="cuda")
        mcwind_recover_adjoint(plan.handle, gu, h, du0)
        mu = torch.zeros_like(h)
        rc, st = mcwind_solve_rhs(plan.handle, h, mu, model.rtol, model.max_cycles)
        if st.status != 0 and st.norm_f > 0:
            raise RuntimeError(f"adjoint solve did not converge: {st.history()[-3:]}")
        dloga = mcwind_adjoint_finish(plan.handle, mu, lam, gu, du0)
        return du0, torch.tensor(dloga, dtype=torch.float64, device=gu.device), None


def downscale(u0, log_a, model):
    """u at the element centers, differentiable in u0 and log_a."""
    return Downscale.apply(u0, log_a, model)
