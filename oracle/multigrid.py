"""Multigrid V-cycle of the Newton-step linear solve (oracle; test
infrastructure only: only tests, the smoke check and the CPU baseline of the
benchmark may import it).

Sec. 3.4: the linear system is preconditioned by geometric multigrid on a
hierarchy of uniformly refined meshes, re-discretised on every level, with
point-block Jacobi relaxation (one dense block per node holding all of its
unknowns) and a direct solve on the coarsest level. Readings used here, as in
the CUDA path: the relaxation is accelerated by Chebyshev step lengths on the
interval [lo, hi] * lambda_max(D^-1 K) (the Chebyshev iteration of Saad,
Iterative Methods for Sparse Linear Systems, Alg. 12.1, applied to D^-1 K),
lambda_max being given; level l takes round(nu * growth^l) steps before and
after its coarse correction; transfers and coarse states as in
oracle/transfer.py; the coarsest level is solved exactly (dense LU).

Written from those definitions with assembled matrices (K from oracle/fe.py,
Dirichlet rows and columns identity) and dense nodal blocks, no fusion.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle import transfer


def nodal_block_inverses(K: sp.csr_matrix, n_nodes: int, n_fields: int) -> np.ndarray:
    """(n_nodes, nf, nf): inverses of the nodal diagonal blocks of K, whose
    DOF (field f, node a) has the index f * n_nodes + a."""
    Kd = K.tocsr()
    out = np.empty((n_nodes, n_fields, n_fields))
    for a in range(n_nodes):
        idx = a + n_nodes * np.arange(n_fields)
        out[a] = np.linalg.inv(Kd[idx][:, idx].toarray())
    return out


def apply_block_inverses(Dinv: np.ndarray, r: np.ndarray) -> np.ndarray:
    """D^-1 r for a nodal field r of shape (nf, n_nodes)."""
    return np.einsum("aij,ja->ia", Dinv, r)


def chebyshev(K, Dinv, b, x, nu: int, lam: float, lo: float, hi: float, want_residual: bool):
    """nu Chebyshev steps for K x = b preconditioned by D (Saad, Alg. 12.1 on
    D^-1 K with the eigenvalue interval [lo lam, hi lam]), from x (None: from
    zero). Returns (x, r) with r = b - K x if want_residual, else (x, None)."""
    shape = b.shape
    Kmul = lambda v: (K @ v.reshape(-1)).reshape(shape)  # noqa: E731
    theta = 0.5 * (hi + lo) * lam
    delta = 0.5 * (hi - lo) * lam
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy() if x is None else b - Kmul(x)
    d = apply_block_inverses(Dinv, r) / theta
    x = d.copy() if x is None else x + d
    for _ in range(1, nu):
        r = r - Kmul(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * apply_block_inverses(Dinv, r)
        x = x + d
        rho = rho_new
    if want_residual:
        return x, r - Kmul(d)
    return x, None


def steps(nu: int, growth: float, level: int) -> int:
    """round(nu * growth^level) (halves away from zero), at least 1."""
    return max(1, int(np.floor(nu * growth ** level + 0.5)))


def vcycle(levels, b, nu_pre: int, nu_post: int, growth: float, lo: float, hi: float, level: int = 0):
    """One V-cycle z = M b. ``levels[l]`` is a dict with the grid ``dims``
    (nx, ny, nz), the matrix ``K`` (Dirichlet rows identity), the Dirichlet
    ``mask`` (nf, n_nodes), and for every level but the last ``Dinv`` and
    ``lam``."""
    L = levels[level]
    if level == len(levels) - 1:
        return np.linalg.solve(L["K"].toarray(), b.reshape(-1)).reshape(b.shape)
    x, r = chebyshev(L["K"], L["Dinv"], b, None, steps(nu_pre, growth, level), L["lam"], lo, hi, True)
    C = levels[level + 1]
    bc = transfer.restrict(L["dims"], C["dims"], r, C["mask"])
    xc = vcycle(levels, bc, nu_pre, nu_post, growth, lo, hi, level + 1)
    x = transfer.prolong_add(L["dims"], C["dims"], xc, x, L["mask"])
    if nu_post > 0:
        x, _ = chebyshev(L["K"], L["Dinv"], b, x, steps(nu_post, growth, level), L["lam"], lo, hi, False)
    return x


def nested_coarse_mask(fine_dims, fine_mask: np.ndarray) -> np.ndarray:
    """Dirichlet mask of the next level of a nested hierarchy (every fine
    dimension even): coarse node (I, J, K) is fine node (2I, 2J, 2K), and a
    coarse DOF is prescribed when that node's DOF is (the nearest fine node
    of the general rule coincides with it)."""
    nx, ny, nz = fine_dims
    assert nx % 2 == 0 and ny % 2 == 0 and nz % 2 == 0
    nf = fine_mask.shape[0]
    m = fine_mask.reshape(nf, nz + 1, ny + 1, nx + 1)
    return np.ascontiguousarray(m[:, ::2, ::2, ::2].reshape(nf, -1))


def nearest_fine_index(I: int, n_coarse: int, n_fine: int) -> int:
    """Index of the fine node nearest to coarse node I along one axis of the
    same box (coarse node at I / n_coarse, fine nodes at i / n_fine): the
    nearest integer to I n_fine / n_coarse, a coarse node exactly midway
    between two fine nodes taking the one of larger index."""
    return (2 * I * n_fine + n_coarse) // (2 * n_coarse)


def coarse_mask(fine_dims, coarse_dims, fine_mask: np.ndarray) -> np.ndarray:
    """Dirichlet mask of the next level (reading r16): a coarse DOF is
    prescribed when the DOF of the nearest fine node is."""
    nf = fine_mask.shape[0]
    fx, fy, fz = fine_dims
    cx, cy, cz = coarse_dims
    m = fine_mask.reshape(nf, fz + 1, fy + 1, fx + 1)
    ii = [nearest_fine_index(I, cx, fx) for I in range(cx + 1)]
    jj = [nearest_fine_index(J, cy, fy) for J in range(cy + 1)]
    kk = [nearest_fine_index(K, cz, fz) for K in range(cz + 1)]
    return np.ascontiguousarray(m[:, kk][:, :, jj][:, :, :, ii].reshape(nf, -1))
