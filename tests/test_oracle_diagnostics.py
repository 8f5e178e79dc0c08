"""Pins of the oracle's microstructure diagnostics (Sec. 5.3) against closed
forms (no GPU)."""
import numpy as np

from oracle import diagnostics as D
from paper_2011_08802_gb300 import inputs


def _state(eta_hat):
    eta_hat = np.asarray(eta_hat, dtype=np.float64)
    U = np.zeros((9, eta_hat.shape[1]))
    U[3:9] = eta_hat
    return U


def test_pure_phases_are_sharp_and_admissible():
    # node 0: austenite; node k: variant k
    eh = np.zeros((6, 7))
    for k in range(1, 7):
        eh[k - 1, k] = 1.0
    U = _state(eh)
    assert np.all(D.violation_index(U) == 0.0)
    assert np.abs(D.diffuseness_index(U)).max() < 1e-15
    assert np.array_equal(D.composite(U), np.array([0, -1, 0, 1, 0, 0, 0], dtype=float))


def test_closed_forms_inside_interfaces():
    # equal mixture of all 7 phases: I_d = 1 - 7 (1/7)^4 = 1 - 1/343
    U = _state(np.full((6, 1), 1.0 / 7.0))
    assert abs(D.diffuseness_index(U)[0] - (1.0 - 1.0 / 343.0)) < 1e-15
    # a 50/50 interface between variants 1 and 3: I_d = 1 - 2/16 = 7/8, eta* = 0
    eh = np.zeros((6, 1)); eh[0] = eh[2] = 0.5
    U = _state(eh)
    assert abs(D.diffuseness_index(U)[0] - 0.875) < 1e-15
    assert D.composite(U)[0] == 0.0


def test_violation_index_counts_every_phase_including_austenite():
    # eta_1 = -0.1, eta_2 = 0.7, eta_3 = 0.5: eta_0 = 1 - 1.1 = -0.1, I_v = 0.2
    eh = np.zeros((6, 1)); eh[0] = -0.1; eh[1] = 0.7; eh[2] = 0.5
    U = _state(eh)
    assert abs(D.violation_index(U)[0] - 0.2) < 1e-15
    eta = D.order_parameters(U)[:, 0]
    assert abs(D.diffuseness_index(U)[0] - (1.0 - (eta ** 4).sum())) < 1e-15
    assert abs(eta.sum() - 1.0) < 1e-15


def test_plane_statistics_layout():
    """Node (i, j, k) -> i + (nx+1)(j + (ny+1)k): plane k holds the nodes with
    that k; put a single violation in one plane and check where it lands."""
    mesh = inputs.Mesh(3, 2, 4, 3.0, 2.0, 4.0)
    nn = mesh.n_nodes
    eh = np.full((6, nn), 1.0 / 7.0)
    i, j, k = 2, 1, 3
    n = i + (mesh.nx + 1) * (j + (mesh.ny + 1) * k)
    eh[0, n] = -0.25  # eta_1 < 0, eta_0 = 1 - 5/7 + 0.25 > 0
    S = D.plane_statistics(mesh, _state(eh))
    assert S.shape == (mesh.nz + 1, 4)
    per_plane = (mesh.nx + 1) * (mesh.ny + 1)
    assert np.all(S[[0, 1, 2, 4], :2] == 0.0)
    assert abs(S[3, 1] - 0.25) < 1e-15 and abs(S[3, 0] - 0.25 / per_plane) < 1e-15
    assert np.allclose(S[[0, 1, 2, 4], 2], 1.0 - 1.0 / 343.0, rtol=0, atol=1e-15)
