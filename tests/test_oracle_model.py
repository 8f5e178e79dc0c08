"""Pins of the oracle's phase-field model against what the paper's model fixes
(Sec. 2, Sec. 3) and closed forms derived from it (no GPU)."""
import copy
import math

import numpy as np
import pytest

from oracle import fe, qp
from paper_2011_08802_gb300 import inputs


def _mat(**kw):
    c = dict(inputs.MATERIAL)
    c.update(kw)
    return qp.material_from(c, tau=0.1)


def _rotation(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def test_pure_variant_is_stress_free():
    """eta = e_i, F = Q U_i: F^e = Q, C^e = I, so the elastic energy, the
    stress P and the elastic driving forces vanish (Sec. 2.1-2.2)."""
    rng = np.random.default_rng(0)
    mat = _mat(F0_martensite=0.0, F0_austenite=0.0, gamma_am=0.0, gamma_mm=0.0)
    for i in range(7):
        eh = np.zeros((1, 6))
        if i > 0:
            eh[0, i - 1] = 1.0
        F = (_rotation(rng) @ mat.U[i])[None]
        W = qp.local_energy(F, eh, eh, mat, order=1)
        assert abs(W.v[0]) < 1e-12
        assert np.abs(W.g[0]).max() < 1e-10


def test_frame_invariance():
    """W(QF) = W(F) and P(QF) = Q P(F) for rotations Q (W depends on C^e)."""
    rng = np.random.default_rng(1)
    B = 16
    F = np.eye(3) + 0.05 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(0.0, 0.3, (B, 6))
    ehn = eh - 0.01
    mat = _mat()
    W = qp.local_energy(F, eh, ehn, mat, order=1)
    Q = np.stack([_rotation(rng) for _ in range(B)])
    WQ = qp.local_energy(Q @ F, eh, ehn, mat, order=1)
    assert np.allclose(WQ.v, W.v, rtol=1e-12, atol=1e-14)
    P = W.g[:, :9].reshape(B, 3, 3)
    PQ = WQ.g[:, :9].reshape(B, 3, 3)
    assert np.allclose(PQ, Q @ P, rtol=1e-10, atol=1e-12)
    assert np.allclose(WQ.g[:, 9:], W.g[:, 9:], rtol=1e-10, atol=1e-12)


def _relax_eta1(mat, eta1_n, steps=30):
    """Solve the 0-D stationarity dW/d eta_1 = 0 (eta_2..6 = 0, F = I,
    elastic part switched off by U_i = I) by Newton with the oracle's exact
    first and second derivatives."""
    mat = copy.deepcopy(mat)
    mat.U[:] = np.eye(3)
    e = eta1_n
    for _ in range(steps):
        eh = np.zeros((1, 6)); eh[0, 0] = e
        ehn = np.zeros((1, 6)); ehn[0, 0] = eta1_n
        W = qp.local_energy(np.eye(3)[None], eh, ehn, mat, order=2)
        e -= W.g[0, 9] / W.H[0, 9, 9]
    return e


def test_backward_euler_step_uses_effective_mobility():
    """Two phases, chemical driving force only: the stationary point of
    Pi_tau is the implicit Euler step eta_1 = eta_1,n - m_01 tau (F_1 - F_0)
    with the effective mobility m_01 = m_0 m_1 / (m_0 + m_1) (Sec. 2.2)."""
    mat = _mat(gamma_am=0.0, gamma_mm=0.0, F0_austenite=0.0, F0_martensite=-0.02)
    mat.m = np.array([4.0, 16.0, 1, 1, 1, 1, 1])
    eta1_n = 0.3
    m01 = 4.0 * 16.0 / 20.0
    expect = eta1_n - m01 * mat.tau * (-0.02)
    assert abs(_relax_eta1(mat, eta1_n) - expect) < 1e-14


def test_penalty_balances_driving_force():
    """With eta_1,n = 0 and F_1 > F_0 the step drives eta_1 below zero, where
    the penalty eps <eta_1>_- enters: eta_1 = -(F_1 - F_0)/(1/(m_01 tau) + eps)."""
    mat = _mat(gamma_am=0.0, gamma_mm=0.0, F0_austenite=0.0, F0_martensite=0.5)
    m01 = mat.m[0] * mat.m[1] / (mat.m[0] + mat.m[1])
    expect = -0.5 / (1.0 / (m01 * mat.tau) + mat.eps_eta)
    assert expect < 0
    assert abs(_relax_eta1(mat, 0.0) - expect) < 1e-15


def test_penalty_acts_on_condensed_austenite():
    """The penalty sum runs from i = 0 (Eq. PenPot): with eta_1,n = 1 and
    F_1 < F_0 the step pushes eta_0 = 1 - eta_1 below zero and
    eta_1 = 1 + (F_0 - F_1)/(1/(m_01 tau) + eps)."""
    mat = _mat(gamma_am=0.0, gamma_mm=0.0, F0_austenite=0.0, F0_martensite=-0.5)
    m01 = mat.m[0] * mat.m[1] / (mat.m[0] + mat.m[1])
    expect = 1.0 + 0.5 / (1.0 / (m01 * mat.tau) + mat.eps_eta)
    assert abs(_relax_eta1(mat, 1.0) - expect) < 1e-14


def _profile_energy(n, pair):
    """Energy per unit area of the stationary double-obstacle profile
    eta = (1 + sin(x/ell))/2 across an i-j interface of width pi*ell."""
    ell = inputs.MATERIAL["ell"]
    Lx = 4 * math.pi * ell
    mesh = inputs.Mesh(n, 1, 1, Lx, 0.5, 0.5)
    X, _, _ = mesh.node_grid()
    x = X.reshape(-1) - Lx / 2
    s = np.clip(x / ell, -math.pi / 2, math.pi / 2)
    eta = 0.5 * (1.0 + np.sin(s))
    U = np.zeros((9, mesh.n_nodes))
    i, j = pair
    if i > 0:
        U[2 + i] = 1.0 - eta
    U[2 + j] = eta
    st = inputs.State(mesh, U, U.copy(), np.zeros((9, mesh.n_nodes), np.uint8), 0.1, {})
    mat = _mat(F0_martensite=0.0)
    mat.U[:] = np.eye(3)
    E = fe.energy(fe.Discretisation(mesh), st, mat)
    return E / (mesh.Ly * mesh.Lz), mat.gamma[i, j]


@pytest.mark.parametrize("pair", [(0, 1), (1, 2)])
def test_interface_energy_equals_gamma(pair):
    """The exact 1-D stationary profile has energy gamma_ij per unit area
    (Eq. IntEnergy with thickness pi*ell); the Q1 discretisation converges at
    O(h^2)."""
    e1, g = _profile_energy(48, pair)
    e2, _ = _profile_energy(96, pair)
    err1, err2 = abs(e1 - g), abs(e2 - g)
    assert err2 < 2e-3 * g
    assert 3.0 < err1 / err2 < 5.0


def test_rotated_variant_mesh_is_stress_free():
    """u = (Q U_1 - I) X and eta_1 = 1 everywhere: zero elastic energy, zero
    mechanical residual at every node, Pi = F_1^0 * volume."""
    rng = np.random.default_rng(4)
    mesh = inputs.Mesh(3, 2, 2, 6.0, 4.0, 4.0)
    mat = _mat()
    G = _rotation(rng) @ mat.U[1] - np.eye(3)
    X, Y, Z = mesh.node_grid()
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])
    U = np.zeros((9, mesh.n_nodes))
    U[0:3] = G @ P
    U[3] = 1.0
    st = inputs.State(mesh, U, U.copy(), np.zeros((9, mesh.n_nodes), np.uint8), 0.1, {})
    disc = fe.Discretisation(mesh)
    R = fe.residual(disc, st, mat)
    assert np.abs(R[0:3]).max() < 1e-10
    vol = mesh.Lx * mesh.Ly * mesh.Lz
    assert abs(fe.energy(disc, st, mat) - mat.F0[1] * vol) < 1e-10 * vol


def test_patch_test_interior_equilibrium():
    """Affine u and uniform eta give a constant stress; the mechanical
    residual vanishes at every interior node."""
    mesh = inputs.Mesh(4, 3, 3, 8.0, 6.0, 6.0)
    rng = np.random.default_rng(5)
    G = 0.03 * rng.standard_normal((3, 3))
    X, Y, Z = mesh.node_grid()
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])
    U = np.zeros((9, mesh.n_nodes))
    U[0:3] = G @ P
    U[3:9] = rng.uniform(0, 0.15, 6)[:, None]
    st = inputs.State(mesh, U, U.copy(), np.zeros((9, mesh.n_nodes), np.uint8), 0.1, {})
    R = fe.residual(fe.Discretisation(mesh), st, _mat())
    Rn = R.reshape(9, 4, 4, 5)[:, 1:-1, 1:-1, 1:-1]
    assert np.abs(Rn[0:3]).max() < 1e-9 * np.abs(R[0:3]).max()


@pytest.fixture(scope="module")
def small_problem():
    st = inputs.config_random(3, 2, 2, seed=7, eta_lo=-0.05, eta_hi=0.3)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    return st, mat, disc, d


def _with_U(st, U):
    s = copy.copy(st)
    s.U = U
    return s


def test_residual_is_gradient_of_energy(small_problem):
    st, mat, disc, d = small_problem
    R = fe.residual(disc, st, mat)
    rng = np.random.default_rng(8)
    for _ in range(3):
        v = rng.standard_normal(st.U.shape)
        v[st.mask.astype(bool)] = 0
        h = 1e-6
        fd = (fe.energy(disc, _with_U(st, st.U + h * v), mat)
              - fe.energy(disc, _with_U(st, st.U - h * v), mat)) / (2 * h)
        assert abs((R * v).sum() - fd) < 1e-7 * abs(fd) + 1e-6


def test_tangent_is_derivative_of_residual(small_problem):
    st, mat, disc, d = small_problem
    K = fe.tangent(disc, st, mat, d)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(st.U.shape)
    v[st.mask.astype(bool)] = 0
    h = 1e-6
    fd = (fe.residual(disc, _with_U(st, st.U + h * v), mat)
          - fe.residual(disc, _with_U(st, st.U - h * v), mat)) / (2 * h)
    Kv = (K @ v.reshape(-1)).reshape(v.shape)
    free = ~st.mask.astype(bool)
    assert np.abs(Kv[free] - fd[free]).max() < 1e-8 * np.abs(Kv).max()


def test_tangent_symmetric_and_jvp_consistent(small_problem):
    st, mat, disc, d = small_problem
    K = fe.tangent(disc, st, mat, d)
    assert abs(K - K.T).max() <= 1e-12 * abs(K).max()
    rng = np.random.default_rng(10)
    v = rng.standard_normal(st.U.shape)
    y = fe.jvp(disc, st, v, d)
    assert np.allclose(y.reshape(-1), K @ v.reshape(-1), rtol=1e-12, atol=1e-12 * abs(K).max())


def test_energy_affine_in_material_parameters():
    """Pi is affine in (C11, C12, C44) and in the interface-energy scale."""
    st = inputs.config_random(2, 2, 2, seed=11)
    disc = fe.Discretisation(st.mesh)
    E = lambda C, s: fe.energy(disc, st, qp.material_from(st.material, st.tau, C=C, gamma_scale=s))  # noqa
    a, b = np.array([141.0, 126.0, 34.0]), np.array([20.0, -5.0, 9.0])
    lhs = E(a + b, 1.0) + E(np.zeros(3), 1.0)
    rhs = E(a, 1.0) + E(b, 1.0)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    assert abs(E(a, 2.0) + E(a, 0.0) - 2 * E(a, 1.0)) < 1e-11 * abs(E(a, 1.0))


def test_newton_correction_solves_linear_system(small_problem):
    st, mat, disc, d = small_problem
    K = fe.tangent(disc, st, mat, d)
    R = fe.residual(disc, st, mat)
    dU = fe.newton_correction(K, R)
    res = K @ dU.reshape(-1) + R.reshape(-1)
    assert np.linalg.norm(res) < 1e-10 * np.linalg.norm(R)
    assert np.all(dU[st.mask.astype(bool)] == 0)
