"""Pins of the oracle's model with N = 12 variants (no GPU): the
twelve-variant workload (15 unknowns per node; the NiTi case named in the
footnote of Sec. 5.4) uses the same model of Sec. 2 with phases 0..12. The
oracle's N-variant code is pinned by what the model fixes for any N (pure
variants stress-free, frame invariance, symmetric Hessian equal to the
derivative of the gradient, the FE patch test, residual = gradient of the
energy) and against the N = 6 oracle: a twelve-variant material whose first
six variants are the CuAlNi ones, evaluated with eta_7..eta_12 = 0, gives
the N = 6 energy, gradient and Hessian exactly."""
import numpy as np
import pytest

from oracle import fe, qp
from paper_2011_08802_gb300 import inputs


def _rotation(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def _mat12(**kw):
    c = inputs.material_nv12()
    c.update(kw)
    return qp.material_from(c, tau=0.1)


def test_variant_set_is_the_cubic_orbit():
    U = inputs.monoclinic_stretches()
    assert U.shape == (13, 3, 3)
    assert np.array_equal(U[0], np.eye(3))
    rots = inputs.cubic_rotations()
    assert len(rots) == 24 and all(abs(np.linalg.det(R) - 1.0) < 1e-15 for R in rots)
    # all twelve distinct, symmetric, positive definite, with U_1's spectrum
    w1 = np.linalg.eigvalsh(U[1])
    for i in range(1, 13):
        assert np.array_equal(U[i], U[i].T)
        assert np.allclose(np.linalg.eigvalsh(U[i]), w1, rtol=0, atol=1e-15)
        for j in range(1, i):
            assert not np.allclose(U[i], U[j])
    # every image of U_1 under the cubic group is one of them (orbit of size 24 / 2)
    images = [R @ U[1] @ R.T for R in rots]
    assert all(any(np.allclose(V, U[i], atol=1e-15) for i in range(1, 13)) for V in images)
    stab = [R for R in rots if np.allclose(R @ U[1] @ R.T, U[1])]
    assert len(stab) == 2


def test_pure_variants_are_stress_free():
    """eta = e_i, F = Q U_i for each of the 13 phases: no elastic energy,
    stress or elastic driving force (Sec. 2.1-2.2)."""
    rng = np.random.default_rng(0)
    mat = _mat12(F0_martensite=0.0, F0_austenite=0.0, gamma_am=0.0, gamma_mm=0.0)
    assert mat.n_var == 12
    for i in range(13):
        eh = np.zeros((1, 12))
        if i > 0:
            eh[0, i - 1] = 1.0
        F = (_rotation(rng) @ mat.U[i])[None]
        W = qp.local_energy(F, eh, eh, mat, order=1)
        assert W.g.shape == (1, 21)
        assert abs(W.v[0]) < 1e-12
        assert np.abs(W.g[0]).max() < 1e-10


def test_frame_invariance_and_hessian():
    rng = np.random.default_rng(1)
    B = 8
    F = np.eye(3) + 0.05 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(0.0, 0.08, (B, 12))
    eh[0, 3] = -0.01  # penalty branch at one point
    ehn = eh - 0.005
    mat = _mat12()
    W = qp.local_energy(F, eh, ehn, mat, order=2)
    Q = np.stack([_rotation(rng) for _ in range(B)])
    WQ = qp.local_energy(Q @ F, eh, ehn, mat, order=1)
    assert np.allclose(WQ.v, W.v, rtol=1e-12, atol=1e-14)
    assert np.allclose(WQ.g[:, :9].reshape(B, 3, 3), Q @ W.g[:, :9].reshape(B, 3, 3), rtol=1e-10, atol=1e-12)
    assert np.allclose(WQ.g[:, 9:], W.g[:, 9:], rtol=1e-10, atol=1e-12)
    # the Hessian is symmetric and is the derivative of the gradient (central differences)
    H = W.H
    assert np.abs(H - np.swapaxes(H, 1, 2)).max() <= 1e-9 * np.abs(H).max()
    h = 1e-6
    z = np.concatenate([F.reshape(B, 9), eh], axis=1)
    for k in (0, 4, 9, 14, 20):
        zp, zm = z.copy(), z.copy()
        zp[:, k] += h
        zm[:, k] -= h
        gp = qp.local_energy(zp[:, :9].reshape(B, 3, 3), zp[:, 9:], ehn, mat, order=1).g
        gm = qp.local_energy(zm[:, :9].reshape(B, 3, 3), zm[:, 9:], ehn, mat, order=1).g
        fd = (gp - gm) / (2 * h)
        assert np.abs(fd - H[:, :, k]).max() <= 1e-5 * np.abs(H).max()


def test_reduces_to_six_variants():
    """Twelve phases whose first six variants are the CuAlNi ones, with
    eta_7..eta_12 = 0: energy, gradient and Hessian in (F, eta_1..6) equal the
    N = 6 oracle's (same constants, one interface energy per pair)."""
    rng = np.random.default_rng(2)
    mat6 = qp.material_from(dict(inputs.MATERIAL), tau=0.1)
    U12 = np.concatenate([mat6.U, inputs.monoclinic_stretches()[1:7]])
    mat12 = qp.material_variants(dict(inputs.MATERIAL), U12, tau=0.1)
    B = 6
    F = np.eye(3) + 0.05 * rng.standard_normal((B, 3, 3))
    eh6 = rng.uniform(0.0, 0.3, (B, 6))
    eh6[1, 2] = -0.02
    ehn6 = eh6 - 0.01
    pad = np.zeros((B, 6))
    W6 = qp.local_energy(F, eh6, ehn6, mat6, order=2)
    W12 = qp.local_energy(F, np.concatenate([eh6, pad], 1), np.concatenate([ehn6, pad], 1), mat12, order=2)
    assert np.allclose(W12.v, W6.v, rtol=1e-14, atol=1e-15)
    assert np.allclose(W12.g[:, :15], W6.g, rtol=1e-13, atol=1e-13)
    assert np.allclose(W12.H[:, :15, :15], W6.H, rtol=1e-12, atol=1e-11)
    g6 = rng.standard_normal((B, 6, 3))
    G6 = qp.gradient_energy(g6, mat6, order=2)
    G12 = qp.gradient_energy(np.concatenate([g6, np.zeros((B, 6, 3))], 1), mat12, order=2)
    assert np.allclose(G12.v, G6.v, rtol=1e-13, atol=1e-14)
    assert np.allclose(G12.H[0][:18, :18], G6.H[0], rtol=1e-13, atol=1e-14)


def test_patch_test_and_residual_gradient():
    """Homogeneous pure variant 7 (F = U_7, eta_7 = 1): zero mechanical
    residual in the interior on a 3^3 mesh; and on a random twelve-variant
    state the residual equals the central difference of the discrete energy."""
    m = inputs.Mesh(3, 3, 3, 6.0, 6.0, 6.0)
    X, Y, Z = m.node_grid()
    pos = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])
    mat = _mat12(F0_martensite=0.0)
    U = np.zeros((15, m.n_nodes))
    U[0:3] = (mat.U[7] - np.eye(3)) @ pos
    U[3 + 6] = 1.0
    st = inputs.State(m, U, U.copy(), np.zeros((15, m.n_nodes), np.uint8), 0.1, inputs.material_nv12())
    disc = fe.Discretisation(m, n_var=12)
    R = fe.residual(disc, st, mat)
    assert np.abs(R[0:3]).max() < 1e-11
    # residual = gradient of the energy on a seeded state
    rng = np.random.default_rng(3)
    U = np.zeros((15, m.n_nodes))
    U[0:3] = 0.02 * rng.standard_normal((3, m.n_nodes))
    U[3:] = rng.uniform(0.0, 0.07, (12, m.n_nodes))
    st = inputs.State(m, U, U - 0.003, np.zeros((15, m.n_nodes), np.uint8), 0.1, inputs.material_nv12())
    R = fe.residual(disc, st, mat)
    v = rng.standard_normal(U.shape)
    h = 1e-6
    sp = inputs.State(m, U + h * v, st.Un, st.mask, 0.1, st.material)
    sm = inputs.State(m, U - h * v, st.Un, st.mask, 0.1, st.material)
    fd = (fe.energy(disc, sp, mat) - fe.energy(disc, sm, mat)) / (2 * h)
    assert abs(fd - np.sum(R * v)) <= 1e-6 * abs(fd)


def test_indentation_state_has_fifteen_fields():
    st = inputs.config_indentation(6, seed=4, step=2, n_var=12)
    assert st.U.shape == (15, 7 ** 3) and st.mask.shape == (15, 7 ** 3)
    assert not st.mask[3:].any()
    assert st.U[3:].min() >= 0.0 and (1.0 - st.U[3:].sum(axis=0)).min() > 0.98
    assert "U" in st.material and len(st.material["U"]) == 13
