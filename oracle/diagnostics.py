"""Microstructure diagnostics of Sec. 5.3 (oracle; test infrastructure only:
only tests, the smoke check and the CPU baseline of the benchmark may import
it).

At every node, with eta_0 = 1 - sum_{k>=1} eta_k (Sec. 3.1):

* violation index I_v = sum_{i=0}^{N} |<eta_i>_-|, the total violation of the
  inequality constraints eta_i >= 0 (Sec. 5.3, penalty study);
* diffuseness index I_d = 1 - sum_{i=0}^{N} eta_i^4, zero in a pure phase and
  positive inside diffuse interfaces (Sec. 5.3, interface-thickness study);
* composite parameter eta* = eta_3 - eta_1 (+1 in variant 3, -1 in variant 1).

The paper reports I_v as the average and the maximum over horizontal planes
as a function of the vertical position z; ``plane_statistics`` gives the mean
and maximum of I_v and of I_d over the nodes of each plane z = const.
"""
from __future__ import annotations

import numpy as np


def order_parameters(U: np.ndarray) -> np.ndarray:
    """eta_0..eta_6 at every node from the nodal state U[9][n_nodes]
    (fields 3..8 are eta_1..eta_6)."""
    eh = U[3:9]
    return np.concatenate([1.0 - eh.sum(axis=0, keepdims=True), eh], axis=0)


def violation_index(U: np.ndarray) -> np.ndarray:
    eta = order_parameters(U)
    return np.abs(np.minimum(eta, 0.0)).sum(axis=0)


def diffuseness_index(U: np.ndarray) -> np.ndarray:
    eta = order_parameters(U)
    return 1.0 - (eta ** 4).sum(axis=0)


def composite(U: np.ndarray) -> np.ndarray:
    return U[3 + 2] - U[3 + 0]


def plane_statistics(mesh, U: np.ndarray) -> np.ndarray:
    """Rows k = 0..nz (plane z = k h_z): (mean I_v, max I_v, mean I_d, max I_d)
    over the (nx + 1)(ny + 1) nodes of the plane."""
    per_plane = (mesh.nx + 1) * (mesh.ny + 1)
    Iv = violation_index(U).reshape(mesh.nz + 1, per_plane)
    Id = diffuseness_index(U).reshape(mesh.nz + 1, per_plane)
    return np.stack([Iv.mean(axis=1), Iv.max(axis=1), Id.mean(axis=1), Id.max(axis=1)], axis=1)
