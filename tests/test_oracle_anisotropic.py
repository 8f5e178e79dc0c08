"""Pins of the oracle's anisotropic material of Table 1 (cubic austenite,
orthorhombic martensite in each variant's principal axes) and of the [011]
crystal orientation of Sec. 5.1 (no GPU)."""
import numpy as np
import pytest

from oracle import qp
from paper_2011_08802_gb300 import inputs

T1 = inputs.ELASTIC_TABLE1


def _longitudinal(L, n):
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    return np.einsum("ijkl,i,j,k,l->", L, n, n, n, n)


def _shear(L, a, b):
    a = np.asarray(a, float) / np.linalg.norm(a)
    b = np.asarray(b, float) / np.linalg.norm(b)
    return np.einsum("ijkl,i,j,k,l->", L, a, b, a, b)


def _mat(orientation=None):
    return qp.material_anisotropic(dict(inputs.MATERIAL), T1, tau=0.1, orientation=orientation)


def test_variant_moduli_along_their_principal_stretches():
    """Variant 1 stretches by alpha along (1,0,1), beta along (0,1,0) and gamma
    along (-1,0,1): its longitudinal moduli there are c11, c22, c33 and its
    shear moduli in those planes c66 (1-2), c55 (1-3), c44 (2-3)."""
    m = _mat()
    o = T1["orthorhombic"]
    L1 = m.Lt[1]
    a1, a2, a3 = (1, 0, 1), (0, 1, 0), (-1, 0, 1)
    assert _longitudinal(L1, a1) == pytest.approx(o["c11"], rel=1e-12)
    assert _longitudinal(L1, a2) == pytest.approx(o["c22"], rel=1e-12)
    assert _longitudinal(L1, a3) == pytest.approx(o["c33"], rel=1e-12)
    assert _shear(L1, a1, a2) == pytest.approx(o["c66"], rel=1e-12)
    assert _shear(L1, a1, a3) == pytest.approx(o["c55"], rel=1e-12)
    assert _shear(L1, a2, a3) == pytest.approx(o["c44"], rel=1e-12)
    # variant 3 stretches by alpha along (1,1,0): c11 there
    assert _longitudinal(m.Lt[3], (1, 1, 0)) == pytest.approx(o["c11"], rel=1e-12)
    # the austenite keeps the cubic constants in the crystal axes
    c = T1["cubic"]
    assert _longitudinal(m.Lt[0], (1, 0, 0)) == pytest.approx(c["c11"])
    assert _shear(m.Lt[0], (1, 0, 0), (0, 1, 0)) == pytest.approx(c["c44"])


def test_cubic_modulus_along_011_and_symmetries():
    """In the [011] orientation the austenite's modulus along z is the cubic
    closed form (c11 + c12 + 2 c44)/2; every stiffness keeps its major and
    minor symmetries."""
    c = T1["cubic"]
    m = _mat(inputs.ORIENTATION_011)
    assert m.Lt[0][2, 2, 2, 2] == pytest.approx((c["c11"] + c["c12"] + 2 * c["c44"]) / 2, rel=1e-12)
    for L in m.Lt:
        assert np.allclose(L, L.transpose(1, 0, 2, 3)) and np.allclose(L, L.transpose(2, 3, 0, 1))
    R = np.asarray(inputs.ORIENTATION_011)
    assert np.allclose(R @ R.T, np.eye(3)) and np.linalg.det(R) == pytest.approx(1.0)


def test_rotating_crystal_and_deformation_together_changes_nothing():
    """W(R F R^T, eta; crystal turned by R) = W(F, eta; crystal), for the
    anisotropic material and the [011] rotation."""
    rng = np.random.default_rng(3)
    R = np.asarray(inputs.ORIENTATION_011)
    m0, mR = _mat(), _mat(R)
    B = 8
    F = np.eye(3) + 0.05 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(0.0, 0.3, (B, 6))
    W0 = qp.local_energy(F, eh, eh, m0, order=1)
    WR = qp.local_energy(R[None] @ F @ R.T[None], eh, eh, mR, order=1)
    assert np.allclose(WR.v, W0.v, rtol=1e-12, atol=1e-14)
    assert np.allclose(WR.g[:, 9:], W0.g[:, 9:], rtol=1e-10, atol=1e-12)


def test_pure_variants_stay_stress_free():
    rng = np.random.default_rng(4)
    c = dict(inputs.MATERIAL, F0_martensite=0.0, F0_austenite=0.0, gamma_am=0.0, gamma_mm=0.0)
    m = qp.material_anisotropic(c, T1, tau=0.1, orientation=inputs.ORIENTATION_011)
    for i in range(7):
        eh = np.zeros((1, 6))
        if i > 0:
            eh[0, i - 1] = 1.0
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        Q *= np.sign(np.linalg.det(Q))
        W = qp.local_energy((Q @ m.U[i])[None], eh, eh, m, order=1)
        assert abs(W.v[0]) < 1e-12 and np.abs(W.g[0]).max() < 1e-10
