"""torch.autograd bindings of the residual R(U; theta) of the phase-field
model (Sec. 3.4: R = dPi/dU of the penalty-regularised incremental potential,
Eq. PenPot) with theta = (C11, C12, C44, s_gamma).

``PFMResidual.apply(U, theta, problem, Un)`` evaluates R on the GPU; its
backward gives dL/dU = J^T g (``pfm_jacobian_transpose_apply``) and
dL/dtheta = g . dR/dtheta (``pfm_param_grad``); its forward-mode ``jvp``
gives J v (``pfm_jacobian_apply``). ``adjoint_gradient`` differentiates a
linear functional w . U* of the solution of R(U*, theta) = 0 by one adjoint
FGMRES solve. All arithmetic runs in the library's kernels; this module only
sequences calls.
"""
from __future__ import annotations

import torch

from . import abi
from .binding import Problem


def params_for(constants: dict, tau: float, theta, hencky: str = "log") -> abi.Params:
    """Parameter block with (C11, C12, C44, s_gamma) taken from theta."""
    t = [float(x) for x in theta]
    return abi.params_from_material(constants, tau, C_override=t[:3], gamma_scale=t[3], hencky=hencky)


class PFMResidual(torch.autograd.Function):
    """R(U; theta) with exact reverse- and forward-mode derivatives."""

    @staticmethod
    def forward(ctx, U, theta, problem: Problem, Un, constants: dict, tau: float):
        problem.set_params(params_for(constants, tau, theta))
        problem.set_state(U.detach().contiguous(), Un.contiguous())
        R = problem.residual()
        ctx.problem = problem
        ctx.state = (U.detach().clone(), Un, theta.detach().clone(), constants, tau)
        return R

    @staticmethod
    def _restore(ctx):
        U, Un, theta, constants, tau = ctx.state
        P = ctx.problem
        P.set_params(params_for(constants, tau, theta))
        P.set_state(U, Un)
        return P

    @staticmethod
    def backward(ctx, gR):
        P = PFMResidual._restore(ctx)
        gR = gR.contiguous().to(torch.float64)
        gU = None
        gtheta = None
        if ctx.needs_input_grad[0]:
            P.linearize(abi.PFM_F64)
            gU = P.jacobian_transpose_apply(gR)
        if ctx.needs_input_grad[1]:
            _, wdR = P.param_grad(gR)
            gtheta = torch.as_tensor(wdR, dtype=torch.float64, device=ctx.state[2].device)
        return gU, gtheta, None, None, None, None

    @staticmethod
    def jvp(ctx, dU, dtheta, *unused):
        P = PFMResidual._restore(ctx)
        out = None
        if dU is not None:
            P.linearize(abi.PFM_F64)
            out = P.jacobian_apply(dU.contiguous().to(torch.float64))
        if dtheta is not None:
            # dR/dtheta_k applied to dtheta: the residual of each theta-part, summed
            parts = theta_residuals(P)
            add = sum(float(dtheta[k]) * parts[k] for k in range(4))
            out = add if out is None else out + add
        return out


def theta_residuals(P: Problem):
    """dR/dtheta_k, k = 0..3, as a (4, 9, n_nodes) tensor (``pfm_param_grad``)."""
    dR = torch.empty((4,) + tuple(P.shape), dtype=torch.float64, device="cuda")
    P.param_grad(None, dR)
    return dR


def energy_gradient(P: Problem):
    """dPi/dtheta at the handle's state (``pfm_param_grad``)."""
    dPi, _ = P.param_grad(None)
    return dPi


def adjoint_gradient(P: Problem, w: torch.Tensor, opts: abi.SolveOpts | None = None):
    """d(w . U*)/dtheta for R(U*, theta) = 0: solve J^T lam = w (J symmetric,
    FGMRES with the V-cycle), then dg/dtheta = -lam . dR/dtheta. The handle's
    state must be the solution U*. Returns (dg/dtheta, lam, FGMRES report)."""
    opts = opts or abi.default_opts(abi.PFM_F32, lin_rtol=1e-10, max_lin_it=600)
    P.linearize(opts.precond)
    lam, rep = P.fgmres_solve(w.contiguous().to(torch.float64), opts)
    _, wdR = P.param_grad(lam)
    return -torch.as_tensor(wdR, dtype=torch.float64), lam, rep
