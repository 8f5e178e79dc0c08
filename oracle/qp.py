"""Local energy density of the multivariant phase-field model at one
quadrature point, with exact first and second derivatives (oracle; test
infrastructure only: only tests, the smoke check and the CPU baseline of the
benchmark may import it).

Everything follows the model of Sec. 2 and the penalty form of Sec. 3.1, in
the paper's notation:

* order parameters eta_0..eta_N with eta_0 = 1 - sum_{i>=1} eta_i (Sec. 3.1);
* linear mixing of the transformation stretch F^t = sum_i eta_i U_i^t, U_0 = I
  (Eq. LinMix), F = F^e F^t (Sec. 2.1);
* Hencky elastic energy F_el = 1/2 det(F^t) H^e . L(eta) H^e with
  H^e = 1/2 log C^e, C^e = F^eT F^e, F^e = F (F^t)^-1, L = sum_i eta_i L_i
  (Eq. elasticEn);
* chemical energy sum_i eta_i F_i^0 (Sec. 2.2);
* double-obstacle interface energy sum_{i<j} 4 gamma_ij/(pi ell_ij)
  (eta_i eta_j - ell_ij^2 grad eta_i . grad eta_j) (Eq. IntEnergy), split here
  into its local part (eta_i eta_j) and its gradient part;
* backward-Euler viscous dissipation sum_i tau/(2 m_i) ((eta_i - eta_i,n)/tau)^2
  (Sec. 2.3);
* penalty sum_i 1/2 eps_eta <eta_i>_-^2 (Eq. PenPot), sums from i = 0.

The matrix logarithm is evaluated by its integral representation
log C = int_0^1 (C - I) (s C + (1 - s) I)^-1 ds (Higham, Functions of
Matrices, Thm. 11.1) with Gauss-Legendre quadrature; its derivatives come
from the jet arithmetic, so no eigen-decomposition is used anywhere here.
The Pade alternatives of Sec. 2.4 (Eqs. pade11, pade22, pade33) replace
1/2 log C by the paper's explicit rational matrix formulas, evaluated as
written (matrix polynomials times the inverse of a matrix polynomial).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .jet import Jet, det3, inv3, matmul, transpose, stack, trace

N_PHASES = 7          # austenite + 6 martensite variants (Sec. 5.1)
N_LOCAL = 15          # seeds: F (9, row-major F_iJ) then eta_1..eta_6
N_GRAD = 18           # seeds: d eta_k / d X_d at index 3*k + d
LOG_QUAD_POINTS = 24  # Gauss-Legendre points of the log integral
# The model is written for any number N of variants (Sec. 2.1: phases
# 0..N); N is read from the material (U has N + 1 entries), the constants
# above are those of the N = 6 CuAlNi data of Sec. 5.1.


@dataclass
class Material:
    U: np.ndarray        # (N+1,3,3) transformation stretches, U[0] = I
    Lt: np.ndarray       # (N+1,3,3,3,3) stiffness tensors L_i
    F0: np.ndarray       # (N+1,) chemical energies
    m: np.ndarray        # (N+1,) mobilities
    gamma: np.ndarray    # (N+1,N+1) interface energies (symmetric)
    ell: np.ndarray      # (N+1,N+1) interface thickness parameters (symmetric)
    eps_eta: float
    tau: float
    hencky: str = "log"  # "log" (exact 1/2 log C) or "pade11" / "pade22" / "pade33" (Sec. 2.4)

    @property
    def n_var(self) -> int:
        """Number N of martensite variants (phases 1..N)."""
        return self.U.shape[0] - 1

    def obstacle(self) -> np.ndarray:
        """Coefficients 4 gamma_ij / (pi ell_ij) of Eq. IntEnergy."""
        c = 4.0 * self.gamma / (math.pi * self.ell)
        np.fill_diagonal(c, 0.0)
        return c


def variant_stretches(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """U_0 = I and the six orthorhombic CuAlNi stretches U_1..U_6 of Sec. 5.1
    (the '+' sign for odd, '-' for even variant numbers)."""
    a = 0.5 * (alpha + gamma)
    b = 0.5 * (alpha - gamma)
    U = np.zeros((7, 3, 3))
    U[0] = np.eye(3)
    for sgn, idx in ((1.0, 1), (-1.0, 2)):
        U[idx] = [[a, 0, sgn * b], [0, beta, 0], [sgn * b, 0, a]]
    for sgn, idx in ((1.0, 3), (-1.0, 4)):
        U[idx] = [[a, sgn * b, 0], [sgn * b, a, 0], [0, 0, beta]]
    for sgn, idx in ((1.0, 5), (-1.0, 6)):
        U[idx] = [[beta, 0, 0], [0, a, sgn * b], [0, sgn * b, a]]
    return U


def cubic_stiffness(C11: float, C12: float, C44: float) -> np.ndarray:
    """Fourth-order cubic stiffness with axes along x, y, z:
    L_iiii = C11, L_iijj = C12 (i != j), L_ijij = L_ijji = C44 (i != j)."""
    L = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                L[i, i, i, i] = C11
            else:
                L[i, i, j, j] = C12
                L[i, j, i, j] = C44
                L[i, j, j, i] = C44
    return L


def orthorhombic_stiffness(c: dict) -> np.ndarray:
    """Fourth-order orthorhombic stiffness in its own axes from the nine
    constants (Voigt pairs 11, 22, 33, 23 -> 4, 13 -> 5, 12 -> 6)."""
    L = np.zeros((3, 3, 3, 3))
    diag = {(0, 0): c["c11"], (1, 1): c["c22"], (2, 2): c["c33"],
            (0, 1): c["c12"], (0, 2): c["c13"], (1, 2): c["c23"]}
    for (i, j), v in diag.items():
        L[i, i, j, j] = L[j, j, i, i] = v
    for (i, j), v in (((1, 2), c["c44"]), ((0, 2), c["c55"]), ((0, 1), c["c66"])):
        L[i, j, i, j] = L[j, i, j, i] = L[i, j, j, i] = L[j, i, i, j] = v
    return L


def rotate_stiffness(L: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """L'_ijkl = Q_ip Q_jq Q_kr Q_ls L_pqrs: the tensor L expressed in the
    frame whose vector components are v' = Q v."""
    return np.einsum("ip,jq,kr,ls,pqrs->ijkl", Q, Q, Q, Q, L)


def variant_axes(U: np.ndarray, alpha: float, beta: float, gamma: float) -> np.ndarray:
    """Principal directions of a variant stretch as the columns of Q, ordered
    by the stretches (alpha, beta, gamma) they carry."""
    w, V = np.linalg.eigh(U)
    order = [int(np.argmin(np.abs(w - t))) for t in (alpha, beta, gamma)]
    return V[:, order]


def material_anisotropic(constants: dict, table: dict, tau: float, orientation=None) -> Material:
    """Material with the anisotropic constants of Table 1: cubic austenite in
    the crystal axes, orthorhombic martensite in each variant's principal
    axes (its orthorhombic axes 1, 2, 3 along the stretches alpha, beta,
    gamma), all turned into the lab frame by ``orientation`` (rows = lab axes
    in crystal coordinates; Sec. 5.1 uses [011] along z)."""
    base = material_from(constants, tau)
    al, be, ga = constants["stretch_alpha"], constants["stretch_beta"], constants["stretch_gamma"]
    cub = table["cubic"]
    Lt = [cubic_stiffness(cub["c11"], cub["c12"], cub["c44"])]
    L_orth = orthorhombic_stiffness(table["orthorhombic"])
    for i in range(1, N_PHASES):
        Lt.append(rotate_stiffness(L_orth, variant_axes(base.U[i], al, be, ga)))
    Lt = np.stack(Lt)
    U = base.U.copy()
    if orientation is not None:
        R = np.asarray(orientation, dtype=np.float64)
        U = np.einsum("ip,npq,jq->nij", R, U, R)
        Lt = np.stack([rotate_stiffness(L, R) for L in Lt])
    return Material(U, Lt, base.F0, base.m, base.gamma, base.ell, base.eps_eta, tau, base.hencky)


def material_from(constants: dict, tau: float, C=None, gamma_scale: float = 1.0,
                  hencky: str = "log") -> Material:
    """Material of Sec. 5.1 from raw constants. ``C`` optionally overrides
    (C11, C12, C44); ``gamma_scale`` multiplies every interface energy;
    ``hencky`` selects the Hencky strain (exact or a Pade approximant). When
    the constants carry the stretches themselves (key "U", N + 1 matrices with
    U[0] = I) any number N of variants is built (``material_variants``)."""
    if "U" in constants:
        mat = material_variants(constants, constants["U"], tau, hencky)
        if C is not None:
            mat.Lt[:] = cubic_stiffness(*C)
        mat.gamma = gamma_scale * mat.gamma
        return mat
    U = variant_stretches(constants["stretch_alpha"], constants["stretch_beta"],
                          constants["stretch_gamma"])
    C11, C12, C44 = C if C is not None else (constants["C11"], constants["C12"], constants["C44"])
    Lt = np.stack([cubic_stiffness(C11, C12, C44)] * N_PHASES)
    F0 = np.array([constants["F0_austenite"]] + [constants["F0_martensite"]] * 6)
    m = np.full(N_PHASES, constants["mobility"])
    g = np.full((7, 7), constants["gamma_mm"])
    g[0, :] = g[:, 0] = constants["gamma_am"]
    np.fill_diagonal(g, 0.0)
    ell = np.full((7, 7), constants["ell"])
    return Material(U, Lt, F0, m, gamma_scale * g, ell, constants["eps_eta"], tau, hencky)


def material_variants(constants: dict, U: np.ndarray, tau: float, hencky: str = "log") -> Material:
    """Material with the transformation stretches U (N+1,3,3), U[0] = I, of
    any number N of variants and the remaining constants of Sec. 5.1: one
    cubic stiffness (C11, C12, C44) for every phase, the martensite chemical
    energy, mobility and interface data for each variant, the austenite ones
    for phase 0."""
    U = np.asarray(U, dtype=np.float64)
    n_phases = U.shape[0]
    Lt = np.stack([cubic_stiffness(constants["C11"], constants["C12"], constants["C44"])] * n_phases)
    F0 = np.array([constants["F0_austenite"]] + [constants["F0_martensite"]] * (n_phases - 1))
    m = np.full(n_phases, constants["mobility"])
    g = np.full((n_phases, n_phases), constants["gamma_mm"])
    g[0, :] = g[:, 0] = constants["gamma_am"]
    np.fill_diagonal(g, 0.0)
    ell = np.full((n_phases, n_phases), constants["ell"])
    return Material(U, Lt, F0, m, g, ell, constants["eps_eta"], tau, hencky)


# ---------------------------------------------------------------------------

def _gauss_legendre_01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def log_spd(C: Jet, n_quad: int = LOG_QUAD_POINTS) -> Jet:
    """log C = int_0^1 (C - I) (s C + (1 - s) I)^-1 ds for symmetric positive
    definite C (value shape (3,3)), by Gauss-Legendre quadrature on [0,1]."""
    I = np.eye(3)
    CmI = C - I
    acc = None
    for s, w in zip(*_gauss_legendre_01(n_quad)):
        M = C * s + I * (1.0 - s)
        t = matmul(CmI, inv3(M)) * w
        acc = t if acc is None else acc + t
    return acc


HENCKY_MODES = ("log", "pade11", "pade22", "pade33")


def hencky_strain(C: Jet, mode: str = "log") -> Jet:
    """Elastic Hencky strain H^e of C = C^e (Eq. elasticEn, Sec. 2.4):
    "log": 1/2 log C exactly (integral representation above);
    "pade11": (C - I)(C + I)^-1                                     (Eq. pade11);
    "pade22": 3/2 (C^2 - I)(C^2 + 4C + I)^-1                         (Eq. pade22);
    "pade33": 1/6 (11C^3 + 27C^2 - 27C - 11I)(C^3 + 9C^2 + 9C + I)^-1 (Eq. pade33)."""
    if mode == "log":
        return log_spd(C) * 0.5
    I = np.eye(3)
    if mode == "pade11":
        num, den, scale = C - I, C + I, 1.0
    elif mode == "pade22":
        C2 = matmul(C, C)
        num, den, scale = C2 - I, C2 + C * 4.0 + I, 1.5
    elif mode == "pade33":
        C2 = matmul(C, C)
        C3 = matmul(C2, C)
        num = C3 * 11.0 + C2 * 27.0 - C * 27.0 - I * 11.0
        den = C3 + C2 * 9.0 + C * 9.0 + I
        scale = 1.0 / 6.0
    else:
        raise ValueError(f"unknown Hencky mode {mode!r}")
    return matmul(num, inv3(den)) * scale


def order_parameters(eta_hat: Jet, n_var: int = 6) -> list:
    """eta_0 = 1 - sum eta_hat (Sec. 3.1) followed by eta_1..eta_N."""
    s = eta_hat[0]
    for k in range(1, n_var):
        s = s + eta_hat[k]
    return [1.0 - s] + [eta_hat[k] for k in range(n_var)]


def _contract(Lt: np.ndarray, h: Jet) -> Jet:
    """(L : h)_ij = sum_kl L_ijkl h_kl for a constant tensor L."""
    rows = []
    for i in range(3):
        row = []
        for j in range(3):
            acc = None
            for k in range(3):
                for l in range(3):
                    c = Lt[i, j, k, l]
                    if c == 0.0:
                        continue
                    t = h[k, l] * c
                    acc = t if acc is None else acc + t
            row.append(acc if acc is not None else h[0, 0] * 0.0)
        rows.append(row)
    return stack([stack(r, axis=0) for r in rows], axis=0)


def _ddot(A: Jet, B: Jet) -> Jet:
    acc = None
    for i in range(3):
        for j in range(3):
            t = A[i, j] * B[i, j]
            acc = t if acc is None else acc + t
    return acc


def _neg_part_sq(x: Jet) -> Jet:
    """<x>_-^2 with <x>_- = x for x < 0 and 0 otherwise (Sec. 3.1)."""
    return (x * x) * (x.v < 0.0).astype(np.float64)


def local_energy(F: np.ndarray, eta_hat: np.ndarray, eta_hat_n: np.ndarray, mat: Material,
                 order: int = 2, parts: bool = False):
    """Local energy density W(F, eta_hat) at B points (everything but the
    gradient part of the interface energy), as a jet in the 9 + N seeds
    (F_iJ row-major, eta_1..eta_N; 15 for the N = 6 data of Sec. 5.1).

    F: (B,3,3); eta_hat, eta_hat_n: (B,N). Returns the scalar jet W, or with
    ``parts`` a dict of the separate terms.
    """
    B = F.shape[0]
    nv = mat.n_var
    n_phases = nv + 1
    n_local = 9 + nv
    z = Jet.variables(np.concatenate([F.reshape(B, 9), eta_hat], axis=1), n_local, 0, order)
    Fj = Jet(z.v[:, :9].reshape(B, 3, 3), z.g[:, :9].reshape(B, 3, 3, n_local),
             None if z.H is None else z.H[:, :9].reshape(B, 3, 3, n_local, n_local))
    eh = z[slice(9, n_local)]
    eta = order_parameters(eh, nv)
    eta_n = [1.0 - eta_hat_n.sum(axis=1)] + [eta_hat_n[:, k] for k in range(nv)]

    # transformation stretch and elastic kinematics (Sec. 2.1, Eq. elasticEn)
    Ft = None
    for i in range(n_phases):
        Ui = np.broadcast_to(mat.U[i], (B, 3, 3))
        t = _scalar_times_matrix(eta[i], Ui)
        Ft = t if Ft is None else Ft + t
    Fe = matmul(Fj, inv3(Ft))
    Ce = matmul(transpose(Fe), Fe)
    He = hencky_strain(Ce, mat.hencky)
    LH = None
    for i in range(n_phases):
        t = _scalar_jet_times_matrix_jet(eta[i], _contract(mat.Lt[i], He))
        LH = t if LH is None else LH + t
    W_el = det3(Ft) * _ddot(He, LH) * 0.5

    W_chem = None
    for i in range(n_phases):
        t = eta[i] * mat.F0[i]
        W_chem = t if W_chem is None else W_chem + t
    c = mat.obstacle()
    W_obst = None
    for i in range(n_phases):
        for j in range(i + 1, n_phases):
            t = eta[i] * eta[j] * c[i, j]
            W_obst = t if W_obst is None else W_obst + t
    W_diss = None
    for i in range(n_phases):
        d = (eta[i] - eta_n[i]) * (1.0 / mat.tau)
        t = d * d * (mat.tau / (2.0 * mat.m[i]))
        W_diss = t if W_diss is None else W_diss + t
    W_pen = None
    for i in range(n_phases):
        t = _neg_part_sq(eta[i]) * (0.5 * mat.eps_eta)
        W_pen = t if W_pen is None else W_pen + t

    if parts:
        return dict(elastic=W_el, chemical=W_chem, obstacle=W_obst, dissipation=W_diss,
                    penalty=W_pen, Ce=Ce, He=He, Ft=Ft)
    return W_el + W_chem + W_obst + W_diss + W_pen


def _scalar_times_matrix(s: Jet, M: np.ndarray) -> Jet:
    """Scalar jet s (B,) times constant matrices M (B,3,3)."""
    v = s.v[:, None, None] * M
    g = M[..., None] * s.g[:, None, None, :]
    H = None if s.H is None else M[..., None, None] * s.H[:, None, None, :, :]
    return Jet(v, g, H)


def _scalar_jet_times_matrix_jet(s: Jet, M: Jet) -> Jet:
    v = s.v[:, None, None] * M.v
    g = s.v[:, None, None, None] * M.g + M.v[..., None] * s.g[:, None, None, :]
    H = None
    if s.H is not None:
        H = (s.v[:, None, None, None, None] * M.H + M.v[..., None, None] * s.H[:, None, None]
             + M.g[..., :, None] * s.g[:, None, None, None, :]
             + s.g[:, None, None, :, None] * M.g[..., None, :])
    return Jet(v, g, H)


def gradient_energy(grad_eta_hat: np.ndarray, mat: Material, order: int = 2) -> Jet:
    """Gradient part of Eq. IntEnergy, -sum_{i<j} 4 gamma_ij ell_ij/pi
    grad eta_i . grad eta_j with grad eta_0 = -sum_k grad eta_k, as a jet in
    the 3N seeds d eta_k / d X_d (index 3k + d). grad_eta_hat: (B,N,3)."""
    B = grad_eta_hat.shape[0]
    nv = mat.n_var
    z = Jet.variables(grad_eta_hat.reshape(B, 3 * nv), 3 * nv, 0, order)
    g = [[z[3 * k + d] for d in range(3)] for k in range(nv)]
    g0 = [None] * 3
    for d in range(3):
        s = g[0][d]
        for k in range(1, nv):
            s = s + g[k][d]
        g0[d] = -s
    grads = [g0] + g
    c = mat.obstacle()
    acc = None
    for i in range(nv + 1):
        for j in range(i + 1, nv + 1):
            dot = grads[i][0] * grads[j][0] + grads[i][1] * grads[j][1] + grads[i][2] * grads[j][2]
            t = dot * (-c[i, j] * mat.ell[i, j] ** 2)
            acc = t if acc is None else acc + t
    return acc
