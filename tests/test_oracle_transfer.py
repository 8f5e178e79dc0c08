"""Pins of the oracle's multigrid transfers (no GPU): what fixes them is
that Q1 interpolation is exact on affine fields, its weights form a partition
of unity, coincident nodes of nested grids are copied exactly (so injecting a
prolongated field gives it back), and one non-nested 1-D case worked by hand."""
import numpy as np
import pytest

from oracle import transfer as T


def _coords(n3, L=(1.0, 1.0, 1.0)):
    nx, ny, nz = n3
    z, y, x = np.meshgrid(np.linspace(0, L[2], nz + 1), np.linspace(0, L[1], ny + 1),
                          np.linspace(0, L[0], nx + 1), indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


PAIRS = [((8, 8, 8), (4, 4, 4)), ((9, 7, 6), (5, 4, 3)), ((5, 3, 2), (3, 2, 1)), ((1, 1, 300), (1, 1, 150))]


@pytest.mark.parametrize("fine, coarse", PAIRS)
def test_partition_of_unity(fine, coarse):
    np.testing.assert_allclose(T.prolongation(fine, coarse).sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(T.injection(fine, coarse).sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("fine, coarse", PAIRS)
def test_affine_fields_are_reproduced(fine, coarse):
    a = np.array([0.3, -1.2, 2.5, 0.7])
    xf, yf, zf = _coords(fine)
    xc, yc, zc = _coords(coarse)
    ff = a[0] + a[1] * xf + a[2] * yf + a[3] * zf
    fc = a[0] + a[1] * xc + a[2] * yc + a[3] * zc
    np.testing.assert_allclose(T.prolongation(fine, coarse) @ fc, ff, atol=1e-13)
    np.testing.assert_allclose(T.injection(fine, coarse) @ ff, fc, atol=1e-13)


def test_nested_grids_copy_coincident_nodes():
    fine, coarse = (8, 6, 4), (4, 3, 2)
    P, Q = T.prolongation(fine, coarse), T.injection(fine, coarse)
    np.testing.assert_allclose(Q @ P, np.eye(P.shape[1]), atol=1e-14)
    xc = np.random.default_rng(1).standard_normal(P.shape[1])
    fine_at_coarse = (np.arange(0, 9, 2)[None, None, :] + 9 * (np.arange(0, 7, 2)[None, :, None]
                      + 7 * np.arange(0, 5, 2)[:, None, None])).reshape(-1)
    np.testing.assert_allclose((P @ xc)[fine_at_coarse], xc, atol=1e-14)


def test_non_nested_weights_by_hand():
    # 5 -> 3 elements on [0, 1]: fine node i at i/5, coarse nodes at I/3 (spacing 1/3)
    M = T.hat_matrix(5, 3)
    expected = np.array([[1.0, 0.0, 0.0, 0.0],
                         [0.4, 0.6, 0.0, 0.0],    # x = 0.2
                         [0.0, 0.8, 0.2, 0.0],    # x = 0.4
                         [0.0, 0.2, 0.8, 0.0],    # x = 0.6
                         [0.0, 0.0, 0.6, 0.4],    # x = 0.8
                         [0.0, 0.0, 0.0, 1.0]])
    np.testing.assert_allclose(M, expected, atol=1e-14)


def test_restriction_is_the_adjoint_and_respects_masks():
    fine, coarse = (9, 7, 6), (5, 4, 3)
    rng = np.random.default_rng(2)
    nf, nc = 10 * 8 * 7, 6 * 5 * 4
    rf, xc = rng.standard_normal((9, nf)), rng.standard_normal((9, nc))
    zero_c, zero_f = np.zeros((9, nc), dtype=np.uint8), np.zeros((9, nf), dtype=np.uint8)
    lhs = np.sum(T.restrict(fine, coarse, rf, zero_c) * xc)
    rhs = np.sum(rf * T.prolong_add(fine, coarse, xc, np.zeros((9, nf)), zero_f))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    mc = (rng.random((9, nc)) < 0.2).astype(np.uint8)
    assert not T.restrict(fine, coarse, rf, mc)[mc.astype(bool)].any()
    mf = (rng.random((9, nf)) < 0.2).astype(np.uint8)
    xf = rng.standard_normal((9, nf))
    out = T.prolong_add(fine, coarse, xc, xf, mf)
    np.testing.assert_array_equal(out[mf.astype(bool)], xf[mf.astype(bool)])
