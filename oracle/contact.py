"""Frictionless penalty contact with a rigid spherical indenter (oracle; test
infrastructure only: only tests, the smoke check and the CPU baseline of the
benchmark may import it).

Sec. 2.5 and Eq. PenPot: the potential contact surface Gamma_c is the top
face z = Lz of the reference box; a point X there sits at x = X + u(X); its
normal gap to the rigid surface is g_N = (x - xbar) . nbar (Eq. Ngap), xbar
its closest-point projection onto the indenter and nbar the indenter's unit
normal there. For a sphere of centre c and radius R the projection is
xbar = c + R (x - c)/|x - c| with nbar = (x - c)/|x - c|, so g_N = |x - c| - R.
The penalty adds int_{Gamma_c} 1/2 eps_N <g_N>_-^2 dS (reference area) to the
incremental potential. The surface integral uses the Q1 face interpolation
of u and the 2x2 Gauss rule on each top-face quad. Derivatives with respect
to x come from the jet arithmetic; the indenter load is the vertical force
the body exerts on the sphere, P = int eps_N <g_N>_- nbar_z dS (positive when
pressing; equal to the derivative of the contact energy with respect to the
indentation depth at fixed u).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .jet import Jet

GA = 0.5 - 0.5 / np.sqrt(3.0)  # 2-point Gauss abscissae on [0, 1]
GB = 0.5 + 0.5 / np.sqrt(3.0)


@dataclass
class Sphere:
    center: np.ndarray  # (3,)
    radius: float
    eps_N: float        # penalty parameter (GPa/nm)


def indenter(mesh, depth: float, radius: float, eps_N: float) -> Sphere:
    """Sphere of the given radius touching the centre of the top face at
    depth 0 and pressed in by ``depth`` (rigid-body position of Sec. 5.1)."""
    return Sphere(np.array([mesh.Lx / 2, mesh.Ly / 2, mesh.Lz + radius - depth]), radius, eps_N)


def top_face(mesh):
    """Top-face quads: node indices (nq, 4) in the order (a&1, a>>1) and the
    2x2 Gauss points' shape values N[q, a] and weights (reference area)."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    quads = []
    for j in range(ny):
        for i in range(nx):
            quads.append([(i + (a & 1)) + (nx + 1) * ((j + (a >> 1)) + (ny + 1) * nz) for a in range(4)])
    pts = [(GA, GA), (GB, GA), (GA, GB), (GB, GB)]
    N = np.array([[(s if a & 1 else 1 - s) * (t if a >> 1 else 1 - t) for a in range(4)] for s, t in pts])
    w = (mesh.Lx / nx) * (mesh.Ly / ny) / 4.0
    return np.array(quads), N, w


def _positions(mesh, U, quads, N):
    X, Y, Z = mesh.node_grid()
    Xn = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)  # node (i fastest) -> X
    xs = Xn + U[0:3].T
    return np.einsum("qa,eai->eqi", N, xs[quads])  # (nq, 4, 3)


def point_terms(x: np.ndarray, sph: Sphere, order: int = 2):
    """Energy density 1/2 eps <g>_-^2, its gradient and Hessian with respect
    to x at points x (B, 3), and the gap, by jets in the 3 seeds x."""
    B = x.shape[0]
    xj = Jet.variables(x, 3, 0, order)
    d = xj - sph.center[None, :]
    r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
    g = r2.sqrt() - sph.radius
    neg = (g.v < 0.0).astype(np.float64)
    e = (g * g) * (0.5 * sph.eps_N * neg)
    return e, g


def contact(mesh, U: np.ndarray, sph: Sphere):
    """Contact energy, residual contribution [9][n_nodes] (u rows only), the
    tangent contribution (CSR over the 9*n_nodes DOFs, field-major) and the
    indenter load P."""
    quads, N, w = top_face(mesh)
    xq = _positions(mesh, U, quads, N).reshape(-1, 3)
    e, g = point_terms(xq, sph)
    nn = mesh.n_nodes
    R = np.zeros((9, nn))
    rows, cols, vals = [], [], []
    ge = e.g.reshape(len(quads), 4, 3)
    He = e.H.reshape(len(quads), 4, 3, 3)
    for qd in range(4):
        for a in range(4):
            np.add.at(R.T, (quads[:, a], slice(0, 3)), w * N[qd, a] * ge[:, qd, :])
            for b in range(4):
                blk = w * N[qd, a] * N[qd, b] * He[:, qd]  # (nq, 3, 3)
                for i in range(3):
                    for k in range(3):
                        rows.append(i * nn + quads[:, a])
                        cols.append(k * nn + quads[:, b])
                        vals.append(blk[:, i, k])
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(9 * nn, 9 * nn))
    energy = float(w * e.v.sum())
    d = xq - sph.center[None, :]
    nz = d[:, 2] / np.linalg.norm(d, axis=1)
    load = float(w * np.sum(sph.eps_N * np.minimum(g.v, 0.0) * nz))
    return energy, R, K, load
