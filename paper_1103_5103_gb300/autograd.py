"""torch.autograd.Function around the multi-mass solve.

Forward: multimass_solve (the paper's single-mass scheme).  Backward: the
library's wilson_solve_backward -- one adjoint solve per mass through
M^dag = gamma5 M gamma5 on the same kernels, the link-force kernel and the
mass gradient.  Every step runs in libwilson; this module only wires
tensors.

Gradients flow to
  eta    -- the source (complex, PyTorch's convention dL/dRe + i dL/dIm),
  m0     -- the bare masses (real),
  omega  -- a (4, V, 8) real probe of left perturbations
            U_mu(n) -> exp(i sum_a omega[mu, n, a] T_a) U_mu(n), T_a = lambda_a/2;
            its gradient is the su(3)-projected link gradient dL/dU at omega = 0.
            omega must be zero: the solve uses the handle's links as they are.
"""
from __future__ import annotations

import torch

from . import api


class _WilsonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eta, m0, omega, gauge, prm, store_solutions):
        masses = [float(v) for v in m0.detach().cpu().tolist()]
        if omega is not None and bool(torch.any(omega != 0)):
            raise ValueError("omega is a zero-valued probe for the link gradient")
        xs, stats = api.multimass_solve(gauge, [eta.detach().contiguous()], masses, prm)
        out = torch.stack(xs[0])
        ctx.gauge, ctx.prm, ctx.masses = gauge, prm, masses
        ctx.store = store_solutions
        ctx.save_for_backward(eta.detach(), out if store_solutions else None)
        ctx.stats = stats[0]
        return out

    @staticmethod
    def backward(ctx, grad_out):
        eta, out = ctx.saved_tensors
        grads = [grad_out[i].contiguous() for i in range(len(ctx.masses))]
        xs = [out[i] for i in range(len(ctx.masses))] if ctx.store else None
        want_u = ctx.needs_input_grad[2]
        want_m = ctx.needs_input_grad[1]
        want_b = ctx.needs_input_grad[0]
        dU, dm, db = api.solve_backward(ctx.gauge, eta.contiguous(), grads, ctx.masses, xs=xs, prm=ctx.prm,
                                        want_links=want_u, want_masses=want_m, want_source=want_b)
        g_m0 = torch.tensor(dm, dtype=torch.float64, device=eta.device) if want_m else None
        return db, g_m0, dU, None, None, None


def wilson_solve(gauge: api.Gauge, eta: torch.Tensor, m0: torch.Tensor, omega: torch.Tensor | None = None,
                 prm: api.SolverParams | None = None, store_solutions: bool = True) -> torch.Tensor:
    """Solutions x_i = M_k(m0_i)^{-1} eta, stacked as (n_mass, V, 4, 3),
    differentiable in eta, m0 and (through the probe omega) the links.
    With store_solutions=False the backward re-solves x instead of keeping it."""
    prm = prm or api.params()
    return _WilsonSolve.apply(eta, m0, omega, gauge, prm, store_solutions)
