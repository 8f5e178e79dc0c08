"""Host logic of the adaptive time stepping of Sec. 3.4 (no GPU): the step
rule (desired 7 and limit 12 Newton iterations), the loading-unloading depth
history, and the driver loop run against a stand-in problem whose Newton
iteration count grows with the step."""
import math
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_2011_08802_gb300 import driver, inputs


def test_step_rule():
    c = driver.StepControl()
    assert driver.next_step(0.1, True, 3, c) == (True, pytest.approx(0.125))
    assert driver.next_step(0.1, True, 7, c) == (True, pytest.approx(0.1))
    assert driver.next_step(0.1, True, 9, c) == (True, pytest.approx(0.08))
    assert driver.next_step(0.1, True, 12, c) == (True, pytest.approx(0.08))
    assert driver.next_step(0.1, True, 13, c) == (False, pytest.approx(0.05))
    assert driver.next_step(0.1, False, 12, c) == (False, pytest.approx(0.05))
    c2 = driver.StepControl(tau_max=0.11, tau_min=0.06)
    assert driver.next_step(0.1, True, 1, c2) == (True, pytest.approx(0.11))
    assert driver.next_step(0.1, False, 4, c2) == (False, pytest.approx(0.06))


def test_depth_history():
    f = driver.depth_history
    assert f(0.0, 2.0, 1.0, True) == 0.0
    assert f(1.5, 2.0, 1.0, True) == 1.5
    assert f(2.0, 2.0, 1.0, True) == 2.0
    assert f(2.5, 2.0, 1.0, True) == 1.5
    assert f(4.0, 2.0, 1.0, True) == 0.0
    assert f(5.0, 2.0, 1.0, True) == 0.0
    assert f(5.0, 2.0, 1.0, False) == 2.0


class _FakeProblem:
    """Newton needs ceil(40 tau) iterations and fails beyond 12."""

    def __init__(self):
        self.tau = None
        self.calls = []

    def set_dirichlet(self, mask, values):
        self.depth = float(-values[2].min()) if values[2].size else 0.0

    def set_params(self, p):
        self.tau = p.tau

    def set_state(self, U, Un):
        pass

    def newton_solve(self, U, opts, check=True):
        its = math.ceil(40 * self.tau)
        self.calls.append((self.tau, self.depth))
        ok = its <= opts.max_newton
        return SimpleNamespace(status=0 if ok else 5, newton_its=min(its, opts.max_newton),
                               lin_its_total=10 * its, res_final=1e-12)

    def diagnostics(self, U, per_node=False):
        return {"planes": torch.zeros(3, 4, dtype=torch.float64)}

    def set_contact(self, center, radius, eps_N):
        self.sphere = (list(center), radius, eps_N)

    def contact_load(self):
        # stands in for the load: the current indentation depth of the sphere
        c, R, _ = self.sphere
        return self.Lz + R - c[2], 0.0


def test_driver_covers_the_history_and_adapts():
    st = inputs.config_indentation(4, seed=1, step=1)
    P = _FakeProblem()
    U, recs = driver.indentation_history(P, st, depth_max=1.0, speed=1.0, tau0=0.5, device="cpu")
    acc = [r for r in recs if r.accepted]
    # accepted steps tile [0, 2] and one of them ends exactly at the turning point t = 1
    assert sum(r.tau for r in acc) == pytest.approx(2.0)
    assert any(abs(r.t - 1.0) < 1e-12 and abs(r.depth - 1.0) < 1e-12 for r in acc)
    assert acc[-1].t == pytest.approx(2.0) and acc[-1].depth == pytest.approx(0.0, abs=1e-12)
    # the first attempt (tau 0.5 -> 20 iterations) is rejected and halved until it converges
    assert not recs[0].accepted and recs[1].tau == pytest.approx(0.25)
    # every accepted step converged within the limit; rejected ones exceeded it
    assert all(r.newton_its <= 12 for r in acc)
    # steps settle around the desired 7 iterations (7/40 = 0.175); the steps cut
    # at the turning point and at the end are shorter, and do not shrink the next one
    full = [r for r in acc[2:-1] if abs(r.t - 1.0) > 1e-12]
    assert all(0.15 < r.tau < 0.2 and r.newton_its == 7 for r in full)
    assert U.shape == st.U.shape


def test_driver_moves_the_contact_sphere():
    """With contact the top face is free, the sphere's lowest point follows the
    depth history and each accepted step records the load."""
    st = inputs.config_indentation(4, seed=1, step=0)
    P = _FakeProblem()
    P.depth = 0.0
    P.Lz = st.mesh.Lz
    P.set_dirichlet = lambda mask, values: setattr(P, "mask", mask.numpy().copy())
    U, recs = driver.indentation_history(P, st, depth_max=1.0, speed=1.0, tau0=0.2, device="cpu",
                                         contact=(5.0, 100.0))
    acc = [r for r in recs if r.accepted]
    assert all(abs(r.load - r.depth) < 1e-12 for r in acc)
    assert P.sphere[1] == 5.0 and P.sphere[2] == 100.0
    m = st.mesh
    top = np.arange(m.n_nodes).reshape(m.nz + 1, m.ny + 1, m.nx + 1)[-1].ravel()
    bottom = np.arange(m.n_nodes).reshape(m.nz + 1, m.ny + 1, m.nx + 1)[0].ravel()
    assert P.mask[:, top].sum() == 0 and np.all(P.mask[0:3, bottom] == 1)
