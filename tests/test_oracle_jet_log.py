"""Pins of the oracle's differentiation and matrix-logarithm routes against
closed forms and library routines (no GPU)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import jet as J
from oracle import qp


def _rand_spd(rng, n, lo, hi):
    out = []
    for _ in range(n):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        lam = rng.uniform(lo, hi, 3)
        out.append(Q @ np.diag(lam) @ Q.T)
    return np.array(out)


def test_inverse_and_determinant_match_numpy():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 3, 3)) + 3 * np.eye(3)
    Aj = J.Jet.variables(A, 9, 0, 2)
    assert np.allclose(J.inv3(Aj).v, np.linalg.inv(A), rtol=1e-13, atol=1e-14)
    assert np.allclose(J.det3(Aj).v, np.linalg.det(A), rtol=1e-13)


def test_jet_derivatives_of_rational_function():
    # f(x) = x / (1 + x^2): f' = (1 - x^2)/(1 + x^2)^2, f'' = 2x(x^2 - 3)/(1 + x^2)^3
    x = np.linspace(-2, 2, 9)[:, None]
    xj = J.Jet.variables(x, 1, 0, 2)[0]
    f = xj * (xj * xj + 1.0).reciprocal()
    xs = x[:, 0]
    assert np.allclose(f.g[:, 0], (1 - xs ** 2) / (1 + xs ** 2) ** 2, rtol=1e-14, atol=1e-15)
    assert np.allclose(f.H[:, 0, 0], 2 * xs * (xs ** 2 - 3) / (1 + xs ** 2) ** 3, rtol=1e-13, atol=1e-15)


def test_determinant_derivative_is_cofactor():
    # d det A / dA = det(A) A^-T (Jacobi's formula)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((5, 3, 3)) + 2 * np.eye(3)
    d = J.det3(J.Jet.variables(A, 9, 0, 1))
    expect = (np.linalg.det(A)[:, None, None] * np.linalg.inv(A).transpose(0, 2, 1)).reshape(5, 9)
    assert np.allclose(d.g, expect, rtol=1e-12)


def test_log_matches_scipy_logm():
    rng = np.random.default_rng(2)
    C = _rand_spd(rng, 30, 0.3, 3.0)
    L = qp.log_spd(J.Jet.variables(C, 9, 0, 1)).v
    for k in range(len(C)):
        ref = scipy.linalg.logm(C[k]).real
        assert np.abs(L[k] - ref).max() < 1e-13


def test_log_of_diagonal_is_entrywise():
    lam = np.array([[0.5, 1.0, 2.5], [1.0, 1.0, 1.0], [0.9, 1.1, 1.3]])
    C = np.stack([np.diag(l) for l in lam])
    L = qp.log_spd(J.Jet.variables(C, 9, 0, 1)).v
    for k in range(3):
        assert np.allclose(L[k], np.diag(np.log(lam[k])), atol=1e-15)


def test_log_first_derivative_daleckii_krein_at_diagonal():
    # at C = diag(l): D log(C)[E]_ab = E_ab (log l_a - log l_b)/(l_a - l_b), and E_aa / l_a
    lam = np.array([0.6, 1.3, 2.2])
    C = np.diag(lam)[None]
    L = qp.log_spd(J.Jet.variables(C, 9, 0, 1))
    for a in range(3):
        for b in range(3):
            dd = 1 / lam[a] if a == b else (np.log(lam[a]) - np.log(lam[b])) / (lam[a] - lam[b])
            # derivative of log(C)_ab w.r.t. C_ab (E = unit matrix e_a e_b^T)
            assert abs(L.g[0, a, b, 3 * a + b] - dd) < 1e-14


def test_log_second_derivative_at_identity():
    # log(I + tE) = tE - t^2 E^2 / 2 + ...  =>  D^2 log(I)[E, E] = -E^2
    rng = np.random.default_rng(3)
    E = rng.standard_normal((3, 3))
    E = E + E.T
    C = np.eye(3)[None]
    L = qp.log_spd(J.Jet.variables(C, 9, 0, 2))
    e = E.reshape(9)
    second = np.einsum("abnm,n,m->ab", L.H[0], e, e)
    assert np.allclose(second, -E @ E, atol=1e-13)
