"""Finite-element residual, tangent and Newton correction of the phase-field
model on a structured trilinear-hexahedron mesh (oracle; test
infrastructure only).

The discrete potential is the sum over elements and 2x2x2 Gauss points of
w_q * (W_loc + W_grad) (Sec. 3.3, with the element reading: Q1 hexahedra
instead of the paper's P1 tetrahedra, the same basis for u and eta_hat).
The residual is its gradient and the tangent its Hessian with respect to the
nodal unknowns (Sec. 3.4: R = dPi/dU, K = d^2Pi/dU^2). Dirichlet DOFs get a
zero residual and identity rows and columns. The Newton correction solves
K dU = -R (Eq. linAlgEq) with a sparse direct factorisation.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import qp

N_FIELDS = 9


def reference_element(h):
    """Shape values N[q,a] and physical gradients dN[q,a,d] of the trilinear
    hexahedron at the 2x2x2 Gauss points, and the point weight w.

    Local node a = a0 + 2 a1 + 4 a2 sits at reference corner (a0,a1,a2);
    point q = q0 + 2 q1 + 4 q2 sits at xi_d = (1 + (2 q_d - 1)/sqrt(3)) / 2.
    """
    g = [(1.0 - 1.0 / math.sqrt(3.0)) / 2.0, (1.0 + 1.0 / math.sqrt(3.0)) / 2.0]
    N = np.zeros((8, 8))
    dN = np.zeros((8, 8, 3))
    for q in range(8):
        xi = [g[(q >> d) & 1] for d in range(3)]
        for a in range(8):
            ad = [(a >> d) & 1 for d in range(3)]
            phi = [xi[d] if ad[d] else 1.0 - xi[d] for d in range(3)]
            dphi = [1.0 if ad[d] else -1.0 for d in range(3)]
            N[q, a] = phi[0] * phi[1] * phi[2]
            for d in range(3):
                prod = dphi[d] / h[d]
                for e in range(3):
                    if e != d:
                        prod *= phi[e]
                dN[q, a, d] = prod
    w = h[0] * h[1] * h[2] / 8.0
    return N, dN, w


def connectivity(mesh) -> np.ndarray:
    """conn[e, a] = global node of local node a of element e, with element
    e = i + nx (j + ny k) and node (i,j,k) -> i + (nx+1)(j + (ny+1) k)."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    conn = np.zeros((mesh.n_elems, 8), dtype=np.int64)
    for a in range(8):
        a0, a1, a2 = a & 1, (a >> 1) & 1, (a >> 2) & 1
        conn[:, a] = (i + a0) + (nx + 1) * ((j + a1) + (ny + 1) * (k + a2))
    return conn


def element_dofs(mesh, conn, n_fields: int = N_FIELDS) -> np.ndarray:
    """Global DOF of local DOF f*8 + a of each element: f*n_nodes + conn[e,a]."""
    nv = mesh.n_nodes
    return np.concatenate([f * nv + conn for f in range(n_fields)], axis=1)


def z_maps(N, dN, n_var: int = 6):
    """Per Gauss point, the linear maps from the 8 (3 + n_var) element DOFs
    (local DOF f*8 + a) to the local seeds z = (F_iJ row-major, eta_hat_k)
    (Bz, (9 + n_var) rows; 15 x 72 for six variants) and to grad eta_hat
    (Bg, 3 n_var rows, row 3k + d)."""
    nd = 8 * (3 + n_var)
    Bz = np.zeros((8, 9 + n_var, nd))
    Bg = np.zeros((8, 3 * n_var, nd))
    for q in range(8):
        for a in range(8):
            for i in range(3):
                for J in range(3):
                    Bz[q, 3 * i + J, i * 8 + a] = dN[q, a, J]
            for k in range(n_var):
                Bz[q, 9 + k, (3 + k) * 8 + a] = N[q, a]
                for d in range(3):
                    Bg[q, 3 * k + d, (3 + k) * 8 + a] = dN[q, a, d]
    return Bz, Bg


class Discretisation:
    """Mesh-level data of the oracle: connectivity, element DOF map, Gauss
    point maps. ``elements`` restricts the element loop to a subset;
    ``n_var`` is the number of variants (3 + n_var fields per node)."""

    def __init__(self, mesh, elements=None, n_var: int = 6):
        self.mesh = mesh
        self.n_var = n_var
        self.n_fields = 3 + n_var
        self.conn = connectivity(mesh)
        self.edofs = element_dofs(mesh, self.conn, self.n_fields)
        self.N, self.dN, self.w = reference_element(mesh.h)
        self.Bz, self.Bg = z_maps(self.N, self.dN, n_var)
        self.elements = np.arange(mesh.n_elems) if elements is None else np.asarray(elements)

    def qp_fields(self, U):
        """F (E,8,3,3), eta_hat (E,8,N) and grad eta_hat (E,8,N,3) at every
        Gauss point of the selected elements, from nodal U (3 + N, n_nodes)."""
        ue = U.reshape(-1)[self.edofs[self.elements]]          # (E, 8 (3 + N))
        z = np.einsum("qzl,el->eqz", self.Bz, ue)              # (E, 8, 9 + N)
        gz = np.einsum("qzl,el->eqz", self.Bg, ue)             # (E, 8, 3 N)
        F = z[..., :9].reshape(-1, 8, 3, 3) + np.eye(3)
        return F, z[..., 9:], gz.reshape(-1, 8, self.n_var, 3)


def _flatq(x):
    return x.reshape((-1,) + x.shape[2:])


def energy(disc, state, mat) -> float:
    """Discrete incremental potential sum_e sum_q w (W_loc + W_grad)."""
    F, eh, geh = disc.qp_fields(state.U)
    _, ehn, _ = disc.qp_fields(state.Un)
    W = qp.local_energy(_flatq(F), _flatq(eh), _flatq(ehn), mat, order=1).v
    Wg = qp.gradient_energy(_flatq(geh), mat, order=1).v
    return float(disc.w * (W.sum() + Wg.sum()))


def qp_derivatives(disc, state, mat, order=2):
    """Per Gauss point of the selected elements: gradient (E,8,9+N) and
    Hessian (E,8,9+N,9+N) of W_loc in (F, eta_hat), gradient (E,8,3N) and
    Hessian (3N,3N) of W_grad in grad eta_hat (N = 6: 15 and 18)."""
    F, eh, geh = disc.qp_fields(state.U)
    _, ehn, _ = disc.qp_fields(state.Un)
    E = F.shape[0]
    W = qp.local_energy(_flatq(F), _flatq(eh), _flatq(ehn), mat, order=order)
    Wg = qp.gradient_energy(_flatq(geh), mat, order=order)
    nz = 9 + disc.n_var
    out = dict(g=W.g.reshape(E, 8, nz), gg=Wg.g.reshape(E, 8, 3 * disc.n_var))
    if order >= 2:
        out["H"] = W.H.reshape(E, 8, nz, nz)
        out["HG"] = Wg.H[0]
    return out


def residual(disc, state, mat, d=None) -> np.ndarray:
    """R = dPi/dU as (3 + N, n_nodes), zero at Dirichlet DOFs. The selected
    elements' contributions only (all elements by default)."""
    if d is None:
        d = qp_derivatives(disc, state, mat, order=1)
    re = disc.w * (np.einsum("qzl,eqz->el", disc.Bz, d["g"]) + np.einsum("qzl,eqz->el", disc.Bg, d["gg"]))
    R = np.zeros(state.U.size)
    np.add.at(R, disc.edofs[disc.elements].ravel(), re.ravel())
    R = R.reshape(state.U.shape)
    R[state.mask.astype(bool)] = 0.0
    return R


def element_matrices(disc, d) -> np.ndarray:
    """K_e = sum_q w (Bz_q^T H_q Bz_q + Bg_q^T HG Bg_q), shape (E, 8 nf, 8 nf)
    with nf = 3 + N fields (72 x 72 for six variants)."""
    K = np.einsum("qzl,eqzy,qym->elm", disc.Bz, d["H"], disc.Bz, optimize=True)
    K += np.einsum("qzl,zy,qym->lm", disc.Bg, d["HG"], disc.Bg, optimize=True)[None]
    return disc.w * K


def tangent(disc, state, mat, d=None) -> sp.csr_matrix:
    """Assembled sparse tangent K = d^2 Pi / dU^2 with Dirichlet rows and
    columns replaced by identity."""
    if d is None:
        d = qp_derivatives(disc, state, mat, order=2)
    Ke = element_matrices(disc, d)
    ed = disc.edofs[disc.elements]
    nd = ed.shape[1]
    rows = np.repeat(ed, nd, axis=1).ravel()
    cols = np.tile(ed, (1, nd)).ravel()
    n = state.U.size
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    D = state.mask.reshape(-1).astype(bool)
    keep = sp.diags((~D).astype(np.float64))
    K = keep @ K @ keep + sp.diags(D.astype(np.float64))
    return K.tocsr()


def jvp(disc, state, v, d) -> np.ndarray:
    """y = K v element by element from the Gauss-point Hessians, with the
    Dirichlet rows/columns of K replaced by identity. v: (9, n_nodes)."""
    D = state.mask.astype(bool)
    vm = np.where(D, 0.0, v)
    ve = vm.reshape(-1)[disc.edofs[disc.elements]]
    z = np.einsum("qzl,el->eqz", disc.Bz, ve)
    gz = np.einsum("qzl,el->eqz", disc.Bg, ve)
    s = np.einsum("eqzy,eqy->eqz", d["H"], z)
    sg = np.einsum("zy,eqy->eqz", d["HG"], gz)
    ye = disc.w * (np.einsum("qzl,eqz->el", disc.Bz, s) + np.einsum("qzl,eqz->el", disc.Bg, sg))
    y = np.zeros(v.size)
    np.add.at(y, disc.edofs[disc.elements].ravel(), ye.ravel())
    y = y.reshape(v.shape)
    y[D] = v[D]
    return y


def newton_correction(K: sp.csr_matrix, R: np.ndarray) -> np.ndarray:
    """dU solving K dU = -R (Eq. linAlgEq) by sparse LU (SuperLU)."""
    lu = spla.splu(K.tocsc())
    return -lu.solve(R.reshape(-1)).reshape(R.shape)
