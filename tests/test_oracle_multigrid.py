"""Pins of the oracle's multigrid V-cycle (oracle/multigrid.py), no GPU:
the Chebyshev smoother's error after nu steps equals the scaled Chebyshev
polynomial of Saad's Alg. 12.1 evaluated on the spectrum of D^-1 K (closed
form from numpy's Chebyshev series); a V-cycle with the same number of pre-
and post-smoothing steps is a symmetric operator (the smoother is
self-adjoint in the K inner product and R = P^T), also on a non-nested
hierarchy with Dirichlet DOFs carried by the nearest-fine-node rule; a
one-level hierarchy is the exact solve; the block inverses are the inverses
of the nodal blocks; the coarse mask takes the nearest fine node."""
import numpy as np
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb

from oracle import multigrid as mg
from oracle import transfer


def _laplacian(dims, shift=1.0):
    """Shifted 7-point grid Laplacian on the nodes of an nx x ny x nz grid
    (node order i + (nx+1)(j + (ny+1)k)): SPD."""
    def lap1(n):
        m = n + 1
        return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    nx, ny, nz = dims
    Ix, Iy, Iz = (sp.identity(n + 1) for n in (nx, ny, nz))
    L = sp.kron(Iz, sp.kron(Iy, lap1(nx))) + sp.kron(Iz, sp.kron(lap1(ny), Ix)) + sp.kron(lap1(nz), sp.kron(Iy, Ix))
    return (L + shift * sp.identity(L.shape[0])).tocsr()


def test_chebyshev_error_is_the_scaled_chebyshev_polynomial():
    rng = np.random.default_rng(5)
    n = 40
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.linspace(0.3, 4.0, n)
    K = sp.csr_matrix(Q @ np.diag(ev) @ Q.T)
    Dinv = np.ones((n, 1, 1))  # D = I (one unknown per node)
    xs = rng.normal(size=(1, n))
    b = (K @ xs.reshape(-1)).reshape(1, n)
    lam, lo, hi = ev.max(), 0.05, 1.1
    theta, delta = 0.5 * (hi + lo) * lam, 0.5 * (hi - lo) * lam
    for nu in (1, 2, 5, 8):
        x, r = mg.chebyshev(K, Dinv, b, None, nu, lam, lo, hi, True)
        # e_nu = T_nu((theta - A)/delta) / T_nu(theta/delta) e_0 with e_0 = x*
        c = np.zeros(nu + 1)
        c[nu] = 1.0
        g = npcheb.chebval((theta - ev) / delta, c) / npcheb.chebval(theta / delta, c)
        e_ref = Q @ (g * (Q.T @ xs.reshape(-1)))
        np.testing.assert_allclose((xs - x).reshape(-1), e_ref, rtol=0, atol=1e-12 * np.abs(xs).max())
        np.testing.assert_allclose(r, b - (K @ x.reshape(-1)).reshape(b.shape), rtol=0, atol=1e-12)


def _levels(dims_list, shift=1.0):
    levels = []
    for l, dims in enumerate(dims_list):
        K = _laplacian(dims, shift)
        n = K.shape[0]
        L = dict(dims=dims, K=K, mask=np.zeros((1, n), dtype=np.uint8))
        if l < len(dims_list) - 1:
            L["Dinv"] = mg.nodal_block_inverses(K, n, 1)
            Dh = np.sqrt(1.0 / K.diagonal())
            L["lam"] = np.linalg.eigvalsh(Dh[:, None] * K.toarray() * Dh[None, :]).max()
        levels.append(L)
    return levels


def test_symmetric_vcycle_is_a_symmetric_operator():
    levels = _levels([(4, 4, 4), (2, 2, 2), (1, 1, 1)])
    n = levels[0]["K"].shape[0]
    M = np.empty((n, n))
    for i in range(n):
        e = np.zeros((1, n))
        e[0, i] = 1.0
        M[:, i] = mg.vcycle(levels, e, 3, 3, 1.0, 0.05, 1.1).reshape(-1)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    # and it is a convergent preconditioner: spectrum of I - M K inside (-1, 1)
    rho = np.abs(np.linalg.eigvals(np.eye(n) - M @ levels[0]["K"].toarray())).max()
    assert rho < 0.5


def test_one_level_is_the_exact_solve_and_block_inverses():
    levels = _levels([(2, 2, 1)])
    b = np.random.default_rng(2).normal(size=(1, levels[0]["K"].shape[0]))
    x = mg.vcycle(levels, b, 2, 8, 1.25, 0.05, 1.1)
    np.testing.assert_allclose(levels[0]["K"] @ x.reshape(-1), b.reshape(-1), rtol=0, atol=1e-12)
    # nodal blocks of a two-field matrix: field f of node a has index f n + a
    K = sp.random(18, 18, density=0.5, random_state=3) + 10 * sp.identity(18)
    Dinv = mg.nodal_block_inverses(K.tocsr(), 9, 2)
    for a in (0, 4, 8):
        idx = [a, a + 9]
        np.testing.assert_allclose(Dinv[a] @ K.toarray()[np.ix_(idx, idx)], np.eye(2), atol=1e-13)
    assert mg.steps(2, 1.25, 1) == 3 and mg.steps(8, 1.25, 1) == 10 and mg.steps(2, 1.25, 0) == 2
    assert mg.steps(2, 1.25, 2) == 3  # 3.125 -> 3
    f = np.arange(2 * 27).reshape(2, 27).astype(np.uint8) % 2
    np.testing.assert_array_equal(mg.nested_coarse_mask((2, 2, 2), f), f[:, [0, 2, 6, 8, 18, 20, 24, 26]])
    np.testing.assert_allclose(transfer.prolongation((2, 2, 2), (1, 1, 1))[[0, 2, 6, 8, 18, 20, 24, 26]], np.eye(8))


def test_coarse_mask_nearest_fine_node():
    # one axis: 9 -> 5 elements puts coarse nodes at 0, 1.8, 3.6, 5.4, 7.2, 9 fine spacings
    assert [mg.nearest_fine_index(I, 5, 9) for I in range(6)] == [0, 2, 4, 5, 7, 9]
    # 3 -> 2: the middle coarse node lies midway between fine nodes 1 and 2
    assert [mg.nearest_fine_index(I, 2, 3) for I in range(3)] == [0, 2, 3]
    # nested grids: the coincident node
    rng = np.random.default_rng(1)
    f = (rng.random((3, 5 * 3 * 7)) < 0.4).astype(np.uint8)  # fine grid (4, 2, 6)
    np.testing.assert_array_equal(mg.coarse_mask((4, 2, 6), (2, 1, 3), f), mg.nested_coarse_mask((4, 2, 6), f))
    # a non-nested 3-D case checked node by node against the coordinates
    f = (rng.random((2, 10 * 8 * 7)) < 0.3).astype(np.uint8)  # fine grid (9, 7, 6)
    c = mg.coarse_mask((9, 7, 6), (5, 4, 3), f)
    for K in range(4):
        for J in range(5):
            for I in range(6):
                x, y, z = I * 9 / 5, J * 7 / 4, K * 6 / 3
                i, j, k = (int(np.floor(t + 0.5)) for t in (x, y, z))
                np.testing.assert_array_equal(c[:, I + 6 * (J + 5 * K)], f[:, i + 10 * (j + 8 * k)])


def test_non_nested_vcycle_is_symmetric_and_convergent():
    # odd grids: coarse grids by ceil(n / 2), transfers between non-nested grids,
    # coarse Dirichlet DOFs by the nearest fine node
    dims = [(5, 3, 3), (3, 2, 2), (2, 1, 1)]
    levels = _levels(dims)
    n = levels[0]["K"].shape[0]
    # Dirichlet DOFs on the fine x = 0 face, carried to the coarse levels
    mask = np.zeros((1, n), dtype=np.uint8)
    mask.reshape(1, 4, 4, 6)[:, :, :, 0] = 1
    levels[0]["mask"] = mask
    for l in range(1, len(dims)):
        levels[l]["mask"] = mg.coarse_mask(dims[l - 1], dims[l], levels[l - 1]["mask"])
    # Dirichlet rows and columns identity, as the oracle's assembled K has them
    for L in levels:
        d = L["mask"].reshape(-1).astype(bool)
        K = L["K"].tolil()
        for i in np.flatnonzero(d):
            K[i, :] = 0
            K[:, i] = 0
            K[i, i] = 1.0
        L["K"] = K.tocsr()
        if "Dinv" in L:
            L["Dinv"] = mg.nodal_block_inverses(L["K"], L["K"].shape[0], 1)
            Dh = np.sqrt(1.0 / L["K"].diagonal())
            L["lam"] = np.linalg.eigvalsh(Dh[:, None] * L["K"].toarray() * Dh[None, :]).max()
    # the x = 0 face of each coarse grid: 3 x 3 and 2 x 2 nodes
    assert levels[1]["mask"].sum() == 9 and levels[2]["mask"].sum() == 4
    free = ~mask.reshape(-1).astype(bool)
    M = np.empty((n, n))
    for i in range(n):
        e = np.zeros((1, n))
        e[0, i] = 1.0
        M[:, i] = mg.vcycle(levels, e, 2, 2, 1.0, 0.05, 1.1).reshape(-1)
    Mf = M[np.ix_(free, free)]
    assert np.abs(Mf - Mf.T).max() <= 1e-12 * np.abs(Mf).max()
    Kf = levels[0]["K"].toarray()[np.ix_(free, free)]
    # a convergent iteration (0.51 measured with two smoothing steps per side)
    rho = np.abs(np.linalg.eigvals(np.eye(Kf.shape[0]) - Mf @ Kf)).max()
    assert rho < 0.75
