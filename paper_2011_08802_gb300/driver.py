"""Load stepping of the indentation problem: a sequence of backward-Euler
steps, each a Newton solve of R(U) = 0 (Sec. 3.4) at a new prescribed cap
depth, with U_n <- U between steps (Sec. 2.3). Host orchestration only: the
cap values come from the input generators, every solve runs in the library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import abi, inputs
from .binding import Problem


def load_ramp(P: Problem, state: inputs.State, upto: int, n_steps: int = 10, depth_frac: float = 0.02,
              radius_frac: float = 0.3, opts: abi.SolveOpts | None = None, U: torch.Tensor | None = None,
              on_step=None, check: bool = True):
    """Run load steps 1..upto of a ramp of n_steps to the final cap depth
    depth_frac * L, starting from ``state`` (U and U_n on the host).
    ``on_step(k, mask, values, Un, U, report)``, if given, sees every step's
    Dirichlet data, previous state and result (device tensors). Returns (U on
    the device after the last step, list of solve reports)."""
    opts = opts or abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-8, lin_rtol=1e-8,
                                    max_lin_it=400)
    U = torch.from_numpy(state.U).cuda() if U is None else U
    Un = torch.from_numpy(state.Un).cuda()
    reports = []
    for k in range(1, upto + 1):
        mask, values = inputs.indentation_dirichlet(state.mesh, k, n_steps, depth_frac, radius_frac)
        P.set_dirichlet(torch.from_numpy(mask).cuda(), torch.from_numpy(values).cuda())
        P.set_state(U, Un)
        rep = P.newton_solve(U, opts, check=check)
        reports.append(rep)
        if on_step is not None:
            on_step(k, mask, values, Un, U, rep)
        Un = U.clone()
        P.set_state(U, Un)
    return U, reports


# ---------------------------------------------------------------------------
# Adaptive time stepping over a loading-unloading history (Sec. 3.4): the step
# grows when the previous Newton solve needed fewer than the desired number of
# iterations, shrinks when it needed more, and a step whose Newton solve does
# not converge within the limit is rejected and retried with half the step.

@dataclass
class StepControl:
    """Time-step rule of Sec. 3.4. The paper gives the desired (7) and the
    limit (12) Newton iteration counts; the growth and shrink factors are not
    stated and are readings."""
    target_its: int = 7
    max_its: int = 12
    grow: float = 1.25
    shrink: float = 0.8
    tau_min: float = 1e-6
    tau_max: float = float("inf")


def next_step(tau: float, converged: bool, newton_its: int, c: StepControl) -> tuple[bool, float]:
    """(accepted, next tau) after a Newton solve with step tau."""
    if not converged or newton_its > c.max_its:
        return False, max(0.5 * tau, c.tau_min)
    if newton_its < c.target_its:
        tau = tau * c.grow
    elif newton_its > c.target_its:
        tau = tau * c.shrink
    return True, min(max(tau, c.tau_min), c.tau_max)


def depth_history(t: float, depth_max: float, speed: float, unload: bool) -> float:
    """Indenter depth at time t: loading at constant speed to depth_max, then
    (if ``unload``) back to zero at the same speed (Sec. 5.1)."""
    t_turn = depth_max / speed
    if t <= t_turn or not unload:
        return min(speed * t, depth_max)
    return max(depth_max - speed * (t - t_turn), 0.0)


@dataclass
class StepRecord:
    t: float
    tau: float
    depth: float
    accepted: bool
    newton_its: int
    lin_its: int
    res_final: float
    max_Iv: float = 0.0
    mean_Id: float = 0.0
    load: float = 0.0  # indenter load P (contact) after the step


def indentation_history(P: Problem, state: inputs.State, depth_max: float, speed: float = 1.0,
                        tau0: float = 0.128, unload: bool = True, control: StepControl | None = None,
                        radius_frac: float = 0.3, hencky: str = "log", max_steps: int = 1000,
                        opts: abi.SolveOpts | None = None, diagnostics: bool = True, device: str = "cuda",
                        on_accept=None, contact: tuple[float, float] | None = None):
    """Drive the indenter through loading (and unloading) with adaptive steps.
    The load is the prescribed cap (default) or, with contact = (R, eps_N),
    frictionless penalty contact with a rigid sphere of radius R whose lowest
    point sits depth(t) below the top face (Sec. 2.5; top face free, bottom
    clamped). Every attempted step is a Newton solve of R(U) = 0 (Sec. 3.4)
    started from the last accepted state; an accepted step sets U_n <- U
    (after calling ``on_accept(record, U_n, U)`` if given) and records the
    indenter load. Returns (U on the device, list of StepRecord, one per
    attempt)."""
    c = control or StepControl()
    opts = opts or abi.default_opts(abi.PFM_F32, max_newton=c.max_its, newton_rtol=1e-8, lin_rtol=1e-8,
                                    max_lin_it=400)
    opts.max_newton = c.max_its
    params = abi.params_from_material(state.material, tau0, hencky=hencky)
    Un = torch.from_numpy(state.Un).to(device)
    U = torch.from_numpy(state.U).to(device)
    t_end = (2.0 if unload else 1.0) * depth_max / speed
    t, tau, records = 0.0, tau0, []
    while t < t_end * (1.0 - 1e-12) and len(records) < max_steps:
        t_turn = depth_max / speed
        step = min(tau, t_end - t)
        if t < t_turn * (1.0 - 1e-12):
            step = min(step, t_turn - t)  # land on the turning point
        depth = depth_history(t + step, depth_max, speed, unload)
        m = state.mesh
        if contact is None:
            mask, values = inputs.indentation_dirichlet_depth(m, depth, radius_frac)
        else:
            mask = inputs.face_mask(m, bottom=True, top=False)
            values = np.zeros_like(state.U)
            P.set_contact([m.Lx / 2, m.Ly / 2, m.Lz + contact[0] - depth], contact[0], contact[1])
        P.set_dirichlet(torch.from_numpy(mask).to(device), torch.from_numpy(values).to(device))
        params.tau = step
        P.set_params(params)
        U.copy_(Un)
        P.set_state(U, Un)
        rep = P.newton_solve(U, opts, check=False)
        converged = rep.status == 0
        accepted, tau_next = next_step(step, converged, rep.newton_its, c)
        if accepted and step < tau:  # a step cut short at the turning point or the end keeps the running size
            tau_next = max(tau_next, tau)
        rec = StepRecord(t + step, step, depth, accepted, rep.newton_its, rep.lin_its_total, rep.res_final)
        if accepted:
            t += step
            if on_accept is not None:
                on_accept(rec, Un, U)
            Un.copy_(U)
            if diagnostics:
                S = P.diagnostics(U, per_node=False)["planes"]
                rec.max_Iv = float(S[:, 1].max())
                rec.mean_Id = float(S[:, 2].mean())
            if contact is not None:
                rec.load = P.contact_load()[0]
        records.append(rec)
        if not accepted and step <= c.tau_min:
            break
        tau = tau_next
    P.set_state(Un, Un)
    return Un, records
