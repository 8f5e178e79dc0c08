"""Load stepping of the indentation problem: a sequence of backward-Euler
steps, each a Newton solve of R(U) = 0 (Sec. 3.4) at a new prescribed cap
depth, with U_n <- U between steps (Sec. 2.3). Host orchestration only: the
cap values come from the input generators, every solve runs in the library.
"""
from __future__ import annotations

import torch

from . import abi, inputs
from .binding import Problem


def load_ramp(P: Problem, state: inputs.State, upto: int, n_steps: int = 10, depth_frac: float = 0.02,
              radius_frac: float = 0.3, opts: abi.SolveOpts | None = None, U: torch.Tensor | None = None):
    """Run load steps 1..upto of a ramp of n_steps to the final cap depth
    depth_frac * L, starting from ``state`` (U and U_n on the host).
    Returns (U on the device after the last step, list of solve reports)."""
    opts = opts or abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-8, lin_rtol=1e-8,
                                    max_lin_it=400)
    U = torch.from_numpy(state.U).cuda() if U is None else U
    Un = torch.from_numpy(state.Un).cuda()
    reports = []
    for k in range(1, upto + 1):
        mask, values = inputs.indentation_dirichlet(state.mesh, k, n_steps, depth_frac, radius_frac)
        P.set_dirichlet(torch.from_numpy(mask).cuda(), torch.from_numpy(values).cuda())
        P.set_state(U, Un)
        rep = P.newton_solve(U, opts)
        reports.append(rep)
        Un = U.clone()
        P.set_state(U, Un)
    return U, reports
