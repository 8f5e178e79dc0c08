"""Pins of the oracle's penalty contact with a rigid sphere (Sec. 2.5, Eq.
Ngap, Eq. PenPot) against closed forms and finite differences (no GPU)."""
import math

import numpy as np

from oracle import contact as C
from paper_2011_08802_gb300 import inputs


def _mesh(n, L=16.0):
    return inputs.Mesh(n, n, n // 2, L, L, L / 2)


def test_gap_under_the_apex_is_minus_the_depth():
    m = _mesh(4)
    sph = C.indenter(m, depth=0.3, radius=7.0, eps_N=100.0)
    e, g = C.point_terms(np.array([[m.Lx / 2, m.Ly / 2, m.Lz]]), sph)
    assert abs(g.v[0] + 0.3) < 1e-14
    assert abs(e.v[0] - 0.5 * 100.0 * 0.09) < 1e-12
    # gradient eps g n with n = (0, 0, -1) below the centre
    assert np.allclose(e.g[0], [0.0, 0.0, -100.0 * -0.3], atol=1e-12)


def test_load_on_a_flat_surface_tends_to_the_closed_form():
    """u = 0: P = int eps (R - s)(R - delta)/s dA over the penetrated disc,
    s = sqrt(r^2 + (R - delta)^2), which integrates to pi eps delta^2 (R - delta)."""
    R, d, eps = 20.0, 0.5, 100.0
    exact = math.pi * eps * d * d * (R - d)
    errs = []
    for n in (16, 32, 64):
        m = _mesh(n)
        U = np.zeros((9, m.n_nodes))
        _, _, _, P = C.contact(m, U, C.indenter(m, d, R, eps))
        errs.append(abs(P - exact) / exact)
    assert errs[2] < 0.01 and errs[2] < errs[1] < errs[0], errs


def _random_top_displacement(m, seed, scale=0.2):
    rng = np.random.default_rng(seed)
    U = np.zeros((9, m.n_nodes))
    U[0:3] = scale * rng.standard_normal((3, m.n_nodes))
    return U


def test_residual_and_tangent_are_derivatives_of_the_energy():
    m = _mesh(6)
    sph = C.indenter(m, depth=1.0, radius=6.0, eps_N=100.0)
    U = _random_top_displacement(m, 3)
    E, R, K, _ = C.contact(m, U, sph)
    assert E > 0.0
    rng = np.random.default_rng(4)
    v = np.zeros_like(U)
    v[0:3] = rng.standard_normal((3, m.n_nodes))
    h = 1e-6
    Ep, Rp, _, _ = C.contact(m, U + h * v, sph)
    Em, Rm, _, _ = C.contact(m, U - h * v, sph)
    assert abs((Ep - Em) / (2 * h) - (R * v).sum()) <= 1e-6 * abs((R * v).sum())
    Kv = (K @ v.reshape(-1)).reshape(v.shape)
    fd = (Rp - Rm) / (2 * h)
    assert np.abs(fd - Kv).max() <= 1e-5 * np.abs(Kv).max()
    assert abs(K - K.T).max() <= 1e-12 * abs(K).max()
    assert np.all(R[3:] == 0.0)


def test_load_is_the_depth_derivative_of_the_energy():
    m = _mesh(8)
    U = _random_top_displacement(m, 5, scale=0.05)
    dd = 1e-6
    E = [C.contact(m, U, C.indenter(m, 1.0 + s, 6.0, 100.0))[0] for s in (dd, -dd)]
    P = C.contact(m, U, C.indenter(m, 1.0, 6.0, 100.0))[3]
    assert abs((E[0] - E[1]) / (2 * dd) - P) <= 1e-6 * abs(P)
