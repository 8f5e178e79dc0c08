"""Seeded synthetic inputs for the Newton-step solve of the multivariant
finite-strain phase-field model (CuAlNi nano-indentation problem, Sec. 5.1).

This module holds data only: the material constants stated in Sec. 5.1 and
Table 1 (with the readings listed below), structured-mesh sizes, seeded random
fields and Dirichlet data. It performs no part of the method's arithmetic (no
kinematics, energy, residual, tangent or solve), so the CUDA path and the CPU
oracle both take their inputs from here and share nothing else.

Units are GPa, nm and s (1 J/m^2 = 1 GPa nm; 1 MPa = 1e-3 GPa).

Readings of the paper used here:
* the elastic constants are one cubic set for every phase (C11=141, C12=126,
  C44=34 GPa), crystal axes along x, y, z (the [011] orientation is left out);
* the unit cube of the synthetic workloads is a cube of edge L = 64 nm, which
  gives lambda/h = pi*ell/h ~ 1.57 at 32^3 (Sec. 5.1 quotes lambda/h ~ 1.5);
* interface energies gamma_am = 0.2, gamma_mm = 0.02 GPa nm, ell = 1 nm,
  chemical energies F_a = 0, F_m = 5 MPa, mobility m = 0.01 (MPa s)^-1 =
  10 (GPa s)^-1, penalty eps_eta = 1e3 GPa (Sec. 5.1);
* vectors are stored field-major, ``[9][n_nodes]``: fields 0..2 are the
  displacement components u_x, u_y, u_z, fields 3..8 the condensed order
  parameters eta_1..eta_6 (Sec. 3.1); node (i, j, k) has index
  ``i + (nx+1) * (j + (ny+1) * k)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage

N_FIELDS = 9
N_VARIANTS = 6

#: Material constants of Sec. 5.1 / Table 1 (see the module docstring).
MATERIAL = dict(
    stretch_alpha=1.0619,
    stretch_beta=0.9178,
    stretch_gamma=1.0230,
    C11=141.0,
    C12=126.0,
    C44=34.0,
    gamma_am=0.2,
    gamma_mm=0.02,
    ell=1.0,
    F0_austenite=0.0,
    F0_martensite=0.005,
    mobility=10.0,
    eps_eta=1.0e3,
)

#: Anisotropic elastic constants of CuAlNi (Table 1, GPa): cubic austenite
#: (c11, c44, c12) and orthorhombic martensite in its own axes.
ELASTIC_TABLE1 = dict(
    cubic=dict(c11=142.0, c44=96.0, c12=126.0),
    orthorhombic=dict(c11=189.0, c22=141.0, c33=205.0, c44=54.9, c55=19.7, c66=62.6,
                      c12=124.0, c13=45.5, c23=115.0),
)

#: Crystal orientation of the indentation example (Sec. 5.1): the austenite
#: [011] axis along the loading direction z. Rows are the lab axes x, y, z in
#: crystal coordinates ([100], [01-1]/sqrt2, [011]/sqrt2), so a crystal-frame
#: vector v has lab components R v.
ORIENTATION_011 = [[1.0, 0.0, 0.0],
                   [0.0, 0.5 ** 0.5, -(0.5 ** 0.5)],
                   [0.0, 0.5 ** 0.5, 0.5 ** 0.5]]

#: Edge of the synthetic cube (nm).
CUBE_EDGE = 64.0

#: Twelve-variant set (N = 12, 15 unknowns per node; the paper names NiTi as
#: such a case in the footnote of Sec. 5.4 but gives no data for it). Reading:
#: a monoclinic stretch of the NiTi B19' type,
#: U_1 = [[gamma, eps, eps], [eps, alpha, delta], [eps, delta, alpha]], with the
#: parameter values below, and variants 2..12 its distinct images R U_1 R^T
#: under the 24 rotations of the cubic group (the stabiliser of U_1 has order
#: 2: the identity and the half turn about [0 1 -1]). All other constants are
#: those of Sec. 5.1 above, one per phase.
MONOCLINIC = dict(alpha=1.0243, gamma=0.9563, delta=0.0580, eps=-0.0427)


def cubic_rotations() -> list:
    """The 24 proper rotations of the cube as signed permutation matrices
    (determinant +1), in a fixed order: permutations in lexicographic order,
    then sign patterns in binary order."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            R = np.zeros((3, 3))
            for i in range(3):
                R[i, perm[i]] = signs[i]
            if np.linalg.det(R) > 0:
                out.append(R)
    return out


def monoclinic_stretches(c: dict = MONOCLINIC) -> np.ndarray:
    """U_0 = I and the 12 monoclinic variant stretches (13, 3, 3): U_1 from
    ``c`` and the distinct R U_1 R^T over ``cubic_rotations()`` in order of
    first appearance."""
    a, g, d, e = c["alpha"], c["gamma"], c["delta"], c["eps"]
    U1 = np.array([[g, e, e], [e, a, d], [e, d, a]])
    U = [np.eye(3)]
    for R in cubic_rotations():
        V = R @ U1 @ R.T
        if not any(np.array_equal(V, W) for W in U[1:]):
            U.append(V)
    return np.stack(U)


def material_nv12() -> dict:
    """Material constants of the twelve-variant workload: Sec. 5.1's, with
    the stretches of ``monoclinic_stretches()`` under the key "U"."""
    return dict(MATERIAL, U=monoclinic_stretches())


@dataclasses.dataclass(frozen=True)
class Mesh:
    """Structured grid of nx*ny*nz trilinear hexahedra on [0,Lx]x[0,Ly]x[0,Lz]."""

    nx: int
    ny: int
    nz: int
    Lx: float = CUBE_EDGE
    Ly: float = CUBE_EDGE
    Lz: float = CUBE_EDGE

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_dofs(self) -> int:
        return N_FIELDS * self.n_nodes

    @property
    def h(self) -> tuple[float, float, float]:
        return (self.Lx / self.nx, self.Ly / self.ny, self.Lz / self.nz)

    def node_grid(self):
        """Node coordinates as three arrays of shape (nz+1, ny+1, nx+1)."""
        x = np.linspace(0.0, self.Lx, self.nx + 1)
        y = np.linspace(0.0, self.Ly, self.ny + 1)
        z = np.linspace(0.0, self.Lz, self.nz + 1)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z


@dataclasses.dataclass
class State:
    """One Newton-step input: mesh, current iterate U, previous-step state Un,
    Dirichlet mask (1 = prescribed DOF) and the time increment tau."""

    mesh: Mesh
    U: np.ndarray      # (3 + N, n_nodes) float64 (N = 6 variants: 9 fields)
    Un: np.ndarray     # (3 + N, n_nodes) float64
    mask: np.ndarray   # (3 + N, n_nodes) uint8
    tau: float
    material: dict


def smooth_noise(shape, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Gaussian-filtered iid N(0,1) noise on a node grid (reflecting edges)."""
    g = rng.standard_normal(shape)
    return ndimage.gaussian_filter(g, sigma=sigma, mode="reflect")


def _to_unit_interval(f: np.ndarray) -> np.ndarray:
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.full_like(f, 0.5)


def _flat(field_zyx: np.ndarray) -> np.ndarray:
    """(nz+1, ny+1, nx+1) node array -> flat node order i + (nx+1)(j + (ny+1)k)."""
    return np.ascontiguousarray(field_zyx).reshape(-1)


def simplex_eta(mesh: Mesh, rng: np.random.Generator, sigma: float = 1.5) -> np.ndarray:
    """Seven smooth fields mapped to [0,1] and normalised to sum one; returns
    the six condensed order parameters eta_1..eta_6, shape (6, n_nodes)."""
    shape = (mesh.nz + 1, mesh.ny + 1, mesh.nx + 1)
    g = np.stack([_to_unit_interval(smooth_noise(shape, sigma, rng)) + 1e-3 for _ in range(7)])
    g /= g.sum(axis=0, keepdims=True)
    return np.stack([_flat(g[k]) for k in range(1, 7)])


def smooth_displacement(mesh: Mesh, rng: np.random.Generator, max_grad: float,
                        sigma: float = 1.5) -> np.ndarray:
    """u = (z/Lz) g(x) with g smooth seeded noise, scaled so that the largest
    nodal finite-difference gradient entry is max_grad; u = 0 on z = 0."""
    X, Y, Z = mesh.node_grid()
    shape = X.shape
    u = np.stack([(Z / mesh.Lz) * smooth_noise(shape, sigma, rng) for _ in range(3)])
    hx, hy, hz = mesh.h
    gmax = 0.0
    for c in range(3):
        for ax, hh in ((2, hx), (1, hy), (0, hz)):
            gmax = max(gmax, np.abs(np.diff(u[c], axis=ax)).max() / hh)
    u *= max_grad / gmax
    return np.stack([_flat(u[c]) for c in range(3)])


def face_mask(mesh: Mesh, bottom: bool = True, top: bool = False, n_var: int = N_VARIANTS) -> np.ndarray:
    """Dirichlet mask with all three displacement components prescribed on the
    bottom (z = 0) and optionally the top (z = Lz) face (3 + n_var fields)."""
    X, Y, Z = mesh.node_grid()
    m = np.zeros((3 + n_var, mesh.n_nodes), dtype=np.uint8)
    sel = np.zeros(X.shape, dtype=bool)
    if bottom:
        sel[0] = True
    if top:
        sel[-1] = True
    m[0:3, _flat(sel)] = 1
    return m


def config_smooth(n: int = 8, seed: int = 1, tau: float = 0.1, max_grad: float = 0.04) -> State:
    """Unit cube of n^3 hexes, seeded smooth eta on the simplex and smooth u with
    |grad u| < 0.05; bottom face clamped, top face prescribed to the initial u
    (so the iterate satisfies its Dirichlet data); eta_n = eta."""
    mesh = Mesh(n, n, n)
    rng = np.random.default_rng(seed)
    U = np.zeros((N_FIELDS, mesh.n_nodes))
    U[0:3] = smooth_displacement(mesh, rng, max_grad)
    U[3:9] = simplex_eta(mesh, rng)
    return State(mesh, U, U.copy(), face_mask(mesh, True, True), tau, dict(MATERIAL))


def cap_displacement(mesh: Mesh, depth: float, radius: float) -> tuple[np.ndarray, np.ndarray]:
    """Prescribed vertical displacement of a spherical cap of base radius
    ``radius`` and depth ``depth`` centred on the top face: for top nodes with
    r <= radius, u_z = -(depth - (R - sqrt(R^2 - r^2))) with
    R = (radius^2 + depth^2) / (2 depth). Returns (node indices, u_z values)."""
    X, Y, Z = mesh.node_grid()
    r = np.hypot(X[-1] - mesh.Lx / 2, Y[-1] - mesh.Ly / 2)
    top_idx = _flat(np.arange(mesh.n_nodes).reshape(X.shape)[-1])
    r = _flat(r)
    sel = r <= radius + 1e-12 * mesh.Lx
    if depth <= 0.0:
        return top_idx[sel], np.zeros(int(sel.sum()))
    R = (radius ** 2 + depth ** 2) / (2.0 * depth)
    uz = -(depth - (R - np.sqrt(R * R - r[sel] ** 2)))
    return top_idx[sel], uz


def indentation_dirichlet(mesh: Mesh, step: int, n_steps: int = 10, depth_frac: float = 0.02,
                          radius_frac: float = 0.3, n_var: int = N_VARIANTS):
    """Mask and values of the indentation load at load step ``step``: bottom
    clamped, u_z prescribed under the cap of depth depth_frac*L*step/n_steps."""
    return indentation_dirichlet_depth(mesh, depth_frac * mesh.Lz * step / n_steps, radius_frac, n_var)


def indentation_dirichlet_depth(mesh: Mesh, depth: float, radius_frac: float = 0.3, n_var: int = N_VARIANTS):
    """Mask and values of the indentation load at cap depth ``depth``: bottom
    clamped, u_z prescribed under the cap of base radius radius_frac*L (the
    cap nodes stay prescribed at depth 0, with u_z = 0)."""
    mask = face_mask(mesh, bottom=True, top=False, n_var=n_var)
    idx, uz = cap_displacement(mesh, depth, radius_frac * mesh.Lx)
    mask[2, idx] = 1
    values = np.zeros((3 + n_var, mesh.n_nodes))
    values[2, idx] = uz
    return mask, values


def config_indentation(n: int, seed: int, step: int = 1, n_steps: int = 10,
                       depth_frac: float = 0.02, radius_frac: float = 0.3,
                       noise: float = 1e-3, tau: float = 0.128, n_var: int = N_VARIANTS) -> State:
    """Nano-indentation-like load on an n^3 cube: eta_hat = noise * U[0,1) per
    node and variant (seeded; one-signed so the initial state lies in the
    admissible simplex eta_i >= 0, sum eta_i = 1), u = 0 except the prescribed
    cap values of load step ``step``, eta_n = eta, bottom clamped. ``n_var``
    = 12 gives the twelve-variant workload (3 + 12 fields, ``material_nv12``)."""
    mesh = Mesh(n, n, n)
    rng = np.random.default_rng(seed)
    mask, values = indentation_dirichlet(mesh, step, n_steps, depth_frac, radius_frac, n_var)
    U = np.zeros((3 + n_var, mesh.n_nodes))
    U[3:] = noise * rng.random((n_var, mesh.n_nodes))
    U[mask.astype(bool)] = values[mask.astype(bool)]
    Un = U.copy()
    Un[0:3] = 0.0
    material = dict(MATERIAL) if n_var == N_VARIANTS else material_nv12()
    return State(mesh, U, Un, mask, tau, material)


def config_random(nx: int, ny: int, nz: int, seed: int, max_grad: float = 0.04,
                  eta_lo: float = 0.0, eta_hi: float = 0.35, tau: float = 0.1,
                  Lx: float = CUBE_EDGE, Ly: float = CUBE_EDGE, Lz: float = CUBE_EDGE,
                  un_shift: float = 0.02, top: bool = True, n_var: int = N_VARIANTS) -> State:
    """Parity-test state on a box of nx*ny*nz hexes: smooth u, smooth eta_hat
    mapped to [eta_lo, eta_hi] (negative eta_lo exercises the penalty branch),
    eta_n = eta minus a smooth seeded shift of size un_shift; ``n_var`` = 12
    for the twelve-variant material."""
    mesh = Mesh(nx, ny, nz, Lx, Ly, Lz)
    rng = np.random.default_rng(seed)
    shape = (nz + 1, ny + 1, nx + 1)
    U = np.zeros((3 + n_var, mesh.n_nodes))
    U[0:3] = smooth_displacement(mesh, rng, max_grad, sigma=1.0)
    for k in range(n_var):
        U[3 + k] = _flat(eta_lo + (eta_hi - eta_lo) * _to_unit_interval(smooth_noise(shape, 1.0, rng)))
    Un = U.copy()
    for k in range(n_var):
        Un[3 + k] -= un_shift * _flat(smooth_noise(shape, 1.0, rng))
    material = dict(MATERIAL) if n_var == N_VARIANTS else material_nv12()
    return State(mesh, U, Un, face_mask(mesh, True, top, n_var), tau, material)


def direction_vectors(state: State, count: int, seed: int) -> np.ndarray:
    """``count`` iid N(0,1) vectors in DOF space, Dirichlet DOFs zeroed;
    shape (count, 9, n_nodes)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((count,) + state.U.shape)
    v[:, state.mask.astype(bool)] = 0.0
    return v


def batch_sizes(count: int = 64, seed: int = 4, lo: int = 8, hi: int = 24):
    """Per-problem mesh edge n ~ U{lo..hi} and indentation depth fraction
    ~ U[0.005, 0.03] for a batch of independent problems."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(lo, hi + 1, size=count)
    depths = rng.uniform(0.005, 0.03, size=count)
    return [int(n) for n in ns], [float(d) for d in depths]
