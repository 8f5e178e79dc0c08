"""Pins of the oracle's Pade Hencky strains (Sec. 2.4, Eqs. pade11, pade22,
pade33) against what fixes them independently of the paper's printed
formulas (no GPU):

* on a diagonal (and rotated diagonal) C the matrix formula acts on each
  eigenvalue as 1/2 p(x - 1)/q(x - 1), where p/q is the [m/m] Pade approximant
  of log(1 + z) that mpmath.pade builds (in 30-digit arithmetic) from the
  Taylor coefficients of log(1 + z) = z - z^2/2 + z^3/3 - ...;
* the approximation error against 1/2 logm(C) (scipy.linalg.logm) falls as
  ||C - I||^(2m+1) (error ratios at e, e/2, e/4, Richardson-extrapolated);
* first and second derivatives of the local energy in every Pade mode equal
  central differences of the energy value;
* a stress-free state (C^e = I) stays stress-free, and the energy is frame
  invariant, in every mode."""
import numpy as np
import pytest
import scipy.linalg

from oracle import jet as J
from oracle import qp
from paper_2011_08802_gb300 import inputs

ORDERS = {"pade11": 1, "pade22": 2, "pade33": 3}


def _rotation(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def _library_pade_half_log(m, x):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    an = [mpmath.mpf(0)] + [mpmath.mpf((-1) ** (k + 1)) / k for k in range(1, 2 * m + 1)]
    p, q = mpmath.pade(an, m, m)
    p = np.array([float(c) for c in p])
    q = np.array([float(c) for c in q])
    z = np.asarray(x, dtype=np.float64) - 1.0
    return 0.5 * np.polynomial.polynomial.polyval(z, p) / np.polynomial.polynomial.polyval(z, q)


def _H(C, mode):
    Cj = J.Jet.const(np.asarray(C, dtype=np.float64), 1, 1)
    return qp.hencky_strain(Cj, mode).v


@pytest.mark.parametrize("mode", sorted(ORDERS))
def test_diagonal_matches_library_pade(mode):
    m = ORDERS[mode]
    lam = np.array([[0.55, 1.0, 1.9], [0.8, 1.2, 1.45], [1.7, 0.95, 0.62]])
    C = np.stack([np.diag(l) for l in lam])
    H = _H(C, mode)
    ref = _library_pade_half_log(m, lam)
    assert np.abs(np.diagonal(H, axis1=1, axis2=2) - ref).max() < 1e-13
    off = H - np.stack([np.diag(np.diagonal(h)) for h in H])
    assert np.abs(off).max() < 1e-14


@pytest.mark.parametrize("mode", sorted(ORDERS))
def test_rotated_diagonal_matches_library_pade(mode):
    """H(Q diag(l) Q^T) = Q diag(r(l)) Q^T: a primary matrix function."""
    m = ORDERS[mode]
    rng = np.random.default_rng(4)
    Qs = np.stack([_rotation(rng) for _ in range(8)])
    lam = rng.uniform(0.6, 1.6, (8, 3))
    C = Qs @ np.stack([np.diag(l) for l in lam]) @ np.transpose(Qs, (0, 2, 1))
    H = _H(C, mode)
    ref = Qs @ np.stack([np.diag(_library_pade_half_log(m, l)) for l in lam]) @ np.transpose(Qs, (0, 2, 1))
    assert np.abs(H - ref).max() < 1e-13


@pytest.mark.parametrize("mode", sorted(ORDERS))
def test_error_against_logm_scales_with_order(mode):
    """||H_(m,m)(I + e X) - 1/2 logm(I + e X)|| = c e^(2m+1) (1 + O(e)): the
    error ratio between e and e/2 tends to 2^(2m+1); two ratios extrapolated
    (2 r(e/2) - r(e)) remove the O(e) term."""
    m = ORDERS[mode]
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 3))
    X = 0.5 * (X + X.T)
    X /= np.linalg.norm(X, 2)
    errs = []
    for e in (0.2, 0.1, 0.05):
        C = np.eye(3) + e * X
        errs.append(np.abs(_H(C[None], mode)[0] - 0.5 * scipy.linalg.logm(C).real).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    extrap = 2 * r2 - r1
    assert abs(extrap / 2 ** (2 * m + 1) - 1.0) < 0.05, (errs, r1, r2, extrap)


def test_higher_order_is_closer_to_log():
    rng = np.random.default_rng(6)
    Q = _rotation(rng)
    C = Q @ np.diag([0.7, 1.1, 1.5]) @ Q.T
    ref = 0.5 * scipy.linalg.logm(C).real
    e = [np.abs(_H(C[None], mode)[0] - ref).max() for mode in ("pade11", "pade22", "pade33")]
    assert e[0] > 10 * e[1] > 100 * e[2]
    assert np.abs(_H(C[None], "log")[0] - ref).max() < 1e-13


@pytest.mark.parametrize("mode", sorted(ORDERS))
def test_energy_derivatives_equal_central_differences(mode):
    rng = np.random.default_rng(7)
    c = dict(inputs.MATERIAL)
    mat = qp.material_from(c, tau=0.1, hencky=mode)
    B = 4
    F = np.eye(3) + 0.08 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(0.0, 0.25, (B, 6))
    ehn = eh - 0.02 * rng.uniform(size=(B, 6))
    W = qp.local_energy(F, eh, ehn, mat, order=2)
    h = 1e-5
    z0 = np.concatenate([F.reshape(B, 9), eh], axis=1)

    def val(z):
        return qp.local_energy(z[:, :9].reshape(B, 3, 3), z[:, 9:], ehn, mat, order=1)

    for k in range(15):
        zp, zm = z0.copy(), z0.copy()
        zp[:, k] += h
        zm[:, k] -= h
        Wp, Wm = val(zp), val(zm)
        g_fd = (Wp.v - Wm.v) / (2 * h)
        H_fd = (Wp.g - Wm.g) / (2 * h)
        assert np.abs(g_fd - W.g[:, k]).max() <= 1e-7 * (1 + np.abs(W.g[:, k]).max())
        assert np.abs(H_fd - W.H[:, :, k]).max() <= 1e-6 * (1 + np.abs(W.H).max())


@pytest.mark.parametrize("mode", sorted(ORDERS))
def test_stress_free_and_frame_invariant(mode):
    rng = np.random.default_rng(8)
    c = dict(inputs.MATERIAL, F0_martensite=0.0, F0_austenite=0.0, gamma_am=0.0, gamma_mm=0.0)
    mat = qp.material_from(c, tau=0.1, hencky=mode)
    for i in (0, 3, 6):
        eh = np.zeros((1, 6))
        if i > 0:
            eh[0, i - 1] = 1.0
        W = qp.local_energy((_rotation(rng) @ mat.U[i])[None], eh, eh, mat, order=1)
        assert abs(W.v[0]) < 1e-12 and np.abs(W.g[0]).max() < 1e-10
    mat = qp.material_from(dict(inputs.MATERIAL), tau=0.1, hencky=mode)
    B = 8
    F = np.eye(3) + 0.05 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(0.0, 0.3, (B, 6))
    Q = np.stack([_rotation(rng) for _ in range(B)])
    W = qp.local_energy(F, eh, eh, mat, order=1)
    WQ = qp.local_energy(Q @ F, eh, eh, mat, order=1)
    assert np.allclose(WQ.v, W.v, rtol=1e-12, atol=1e-14)
    assert np.allclose(WQ.g[:, :9].reshape(B, 3, 3), Q @ W.g[:, :9].reshape(B, 3, 3), rtol=1e-10, atol=1e-12)
