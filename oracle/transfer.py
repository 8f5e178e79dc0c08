"""Grid transfers of the geometric multigrid (oracle; test infrastructure
only: only tests, the smoke check and the CPU baseline of the benchmark may
import it).

Sec. 3.4: the multigrid works on a hierarchy of uniformly refined meshes of
the same domain, with the problem re-discretised on every level. Readings
used here (the paper names the transfers but does not define them): the
prolongation P maps a coarse nodal field to the fine nodes by evaluating the
coarse Q1 (trilinear) interpolant there, restriction is R = P^T, and the
state reaching a coarse level is the fine Q1 field evaluated at the coarse
nodes; a level of n elements per direction has ceil(n/2) elements on the next
one, on the same box (non-nested when n is odd).

Written from the definitions: the 1-D Q1 hat function of node I of a grid of
spacing H on [0, L] is max(0, 1 - |x - I H| / H); the 3-D basis is the
tensor product, so P = Pz (x) Py (x) Px in the node order
i + (nx+1)(j + (ny+1)k). Nodal fields are arrays (9, n_nodes).
"""
from __future__ import annotations

import numpy as np


def hat_matrix(n_to: int, n_from: int, length: float = 1.0) -> np.ndarray:
    """(n_to+1, n_from+1): the Q1 hat functions of the n_from-element grid on
    [0, length] evaluated at the nodes of the n_to-element grid."""
    x = np.arange(n_to + 1) * (length / n_to)
    X = np.arange(n_from + 1) * (length / n_from)
    H = length / n_from
    return np.maximum(0.0, 1.0 - np.abs(x[:, None] - X[None, :]) / H)


def _kron3(Az, Ay, Ax):
    return np.kron(Az, np.kron(Ay, Ax))


def prolongation(fine, coarse) -> np.ndarray:
    """P (fine nodes x coarse nodes) for grids given as (nx, ny, nz)."""
    return _kron3(hat_matrix(fine[2], coarse[2]), hat_matrix(fine[1], coarse[1]), hat_matrix(fine[0], coarse[0]))


def injection(fine, coarse) -> np.ndarray:
    """Q (coarse nodes x fine nodes): the fine Q1 field at the coarse nodes."""
    return _kron3(hat_matrix(coarse[2], fine[2]), hat_matrix(coarse[1], fine[1]), hat_matrix(coarse[0], fine[0]))


def prolong_add(fine, coarse, xc, xf, fine_mask) -> np.ndarray:
    """xf + P xc at the free DOFs of the fine level (Dirichlet DOFs unchanged)."""
    P = prolongation(fine, coarse)
    out = xf + xc @ P.T
    keep = fine_mask.astype(bool)
    out[keep] = xf[keep]
    return out


def restrict(fine, coarse, rf, coarse_mask) -> np.ndarray:
    """R rf = P^T rf, zero at the Dirichlet DOFs of the coarse level."""
    P = prolongation(fine, coarse)
    out = rf @ P
    out[coarse_mask.astype(bool)] = 0.0
    return out


def inject(fine, coarse, Uf) -> np.ndarray:
    """The fine Q1 state at the coarse nodes, every field."""
    return Uf @ injection(fine, coarse).T
