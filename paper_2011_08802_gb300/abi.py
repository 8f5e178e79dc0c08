"""ctypes declarations of the C ABI in include/pfm.h and loading of the
CUDA library (argument marshalling only: every step of the computation runs
in the library's kernels). The library must have been built (see
``paper_2011_08802_gb300.build``); importing the binding without it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs

LIB_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libpfm.so")

PFM_F32 = 0
PFM_F64 = 1

PROF_JAPPLY_F32, PROF_JAPPLY_F64, PROF_LINEARIZE, PROF_RESIDUAL, PROF_VCYCLE, PROF_JAPPLY_F16 = range(6)

STATUS = {
    0: "PFM_OK", 1: "PFM_ERR_INVALID_ARG", 2: "PFM_ERR_CUDA", 3: "PFM_ERR_OOM",
    4: "PFM_ERR_NONFINITE", 5: "PFM_ERR_NOT_CONVERGED", 6: "PFM_ERR_BREAKDOWN",
    7: "PFM_ERR_TIMEOUT", 8: "PFM_ERR_STATE",
}


class MeshDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("n_levels", C.c_int)]


def _params_class(n_var: int):
    """ctypes layout of pfm_params for a library built with N = n_var variants
    (N + 1 phases)."""
    P = n_var + 1

    class _Params(C.Structure):
        _fields_ = [("Ut", (C.c_double * 9) * P), ("Lvoigt", (C.c_double * 36) * P),
                    ("F0", C.c_double * P), ("mobility", C.c_double * P),
                    ("gamma", (C.c_double * P) * P), ("ell", (C.c_double * P) * P),
                    ("eps_eta", C.c_double), ("tau", C.c_double), ("gamma_scale", C.c_double),
                    ("hencky", C.c_int)]
        N_VAR = n_var

    _Params.__name__ = _Params.__qualname__ = "Params" if n_var == 6 else f"Params{n_var}"
    return _Params


#: pfm_params of libpfm.so (N = 6) and of libpfm_nv12.so (N = 12)
Params = _params_class(6)
PARAMS = {6: Params, 12: _params_class(12)}


# Hencky strain modes of pfm_params.hencky (Sec. 2.4)
HENCKY = {"log": 0, "pade11": 1, "pade22": 2, "pade33": 3}


class CubicMaterial(C.Structure):
    """pfm_cubic_material: the scalar model data of Sec. 5.1."""
    _fields_ = [(n, C.c_double) for n in (
        "stretch_alpha", "stretch_beta", "stretch_gamma", "C11", "C12", "C44", "F0_austenite",
        "F0_martensite", "mobility", "gamma_am", "gamma_mm", "ell", "eps_eta")]


class SolveOpts(C.Structure):
    _fields_ = [("max_newton", C.c_int), ("restart", C.c_int), ("max_lin_it", C.c_int),
                ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("newton_rtol", C.c_double), ("lin_rtol", C.c_double), ("omega", C.c_double),
                ("precond", C.c_int), ("smoother", C.c_int), ("cheb_lo", C.c_double),
                ("cheb_hi", C.c_double), ("cycle_gamma", C.c_int), ("nu_growth", C.c_double),
                ("deterministic", C.c_int), ("krylov", C.c_int), ("switch_rtol", C.c_double)]


class SolveReport(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("lin_its_total", C.c_int), ("lin_its_last", C.c_int),
                ("res0", C.c_double), ("res_final", C.c_double), ("lin_res_final", C.c_double),
                ("lin_outer_last", C.c_int), ("ms_residual", C.c_double), ("ms_linearize", C.c_double),
                ("ms_solve", C.c_double), ("ms_total", C.c_double), ("status", C.c_int)]


def default_opts(precond: int = PFM_F32, **kw) -> SolveOpts:
    o = SolveOpts(max_newton=1, restart=30, max_lin_it=300, nu_pre=2, nu_post=8,
                  newton_rtol=1e-8, lin_rtol=1e-8, omega=0.7, precond=precond,
                  smoother=0, cheb_lo=0.05, cheb_hi=1.1, cycle_gamma=1, nu_growth=1.25,
                  deterministic=0, krylov=0, switch_rtol=1e-3)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def params_from_material(constants: dict, tau: float, C_override=None,
                         gamma_scale: float = 1.0, hencky: str = "log") -> Params:
    """Fill the parameter block from the raw constants of Sec. 5.1: variant
    stretches U_1..U_6 from (alpha, beta, gamma), or all N + 1 stretches when
    the constants carry them (key "U"; the block then has N + 1 phases for the
    library built with N variants), the cubic Voigt stiffness
    from (C11, C12, C44) for every phase, gamma_0i = gamma_am,
    gamma_ij = gamma_mm, one ell, F_0 = F_a, F_i = F_m, one mobility;
    ``hencky`` names the Hencky strain ("log" or a Pade mode, Sec. 2.4)."""
    if "U" in constants:  # the stretches themselves (any number N of variants)
        U = [np.asarray(x, dtype=np.float64) for x in constants["U"]]
    else:
        al, be, ga = constants["stretch_alpha"], constants["stretch_beta"], constants["stretch_gamma"]
        p, q = 0.5 * (al + ga), 0.5 * (al - ga)
        U = [np.eye(3)]
        for s in (1.0, -1.0):
            U.append(np.array([[p, 0, s * q], [0, be, 0], [s * q, 0, p]]))
        for s in (1.0, -1.0):
            U.append(np.array([[p, s * q, 0], [s * q, p, 0], [0, 0, be]]))
        for s in (1.0, -1.0):
            U.append(np.array([[be, 0, 0], [0, p, s * q], [0, s * q, p]]))
    n_ph = len(U)
    C11, C12, C44 = C_override if C_override is not None else (
        constants["C11"], constants["C12"], constants["C44"])
    Lv = np.zeros((6, 6))
    Lv[:3, :3] = C12
    np.fill_diagonal(Lv[:3, :3], C11)
    Lv[3, 3] = Lv[4, 4] = Lv[5, 5] = C44
    P = PARAMS[n_ph - 1]()
    for i in range(n_ph):
        for k in range(9):
            P.Ut[i][k] = U[i].reshape(9)[k]
        for k in range(36):
            P.Lvoigt[i][k] = Lv.reshape(36)[k]
        P.F0[i] = constants["F0_austenite"] if i == 0 else constants["F0_martensite"]
        P.mobility[i] = constants["mobility"]
        for j in range(n_ph):
            g = 0.0 if i == j else (constants["gamma_am"] if (i == 0 or j == 0) else constants["gamma_mm"])
            P.gamma[i][j] = g
            P.ell[i][j] = constants["ell"]
    P.eps_eta = constants["eps_eta"]
    P.tau = tau
    P.gamma_scale = gamma_scale
    P.hencky = HENCKY[hencky]
    return P


def _bond(a: np.ndarray) -> np.ndarray:
    """6x6 Bond matrix M of the rotation a (x' = a x) for stiffness in the
    Voigt order (11, 22, 33, 23, 13, 12) with engineering shear strains:
    C' = M C M^T."""
    M = np.zeros((6, 6))
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for I, (i, j) in enumerate(pairs):
        for J, (k, l) in enumerate(pairs):
            if J < 3:
                M[I, J] = a[i, k] * a[j, k]
            else:
                M[I, J] = a[i, k] * a[j, l] + a[i, l] * a[j, k]
    return M


def params_anisotropic(constants: dict, table: dict, tau: float, orientation=None,
                       hencky: str = "log") -> Params:
    """Parameter block with the anisotropic constants of Table 1: cubic
    austenite in the crystal axes, orthorhombic martensite in each variant's
    principal axes (orthorhombic axes 1, 2, 3 along the stretches alpha, beta,
    gamma), every stretch and stiffness turned into the lab frame by
    ``orientation`` (rows = lab axes in crystal coordinates). Voigt matrices
    are rotated with Bond matrices."""
    P = params_from_material(constants, tau, hencky=hencky)
    al, be, ga = constants["stretch_alpha"], constants["stretch_beta"], constants["stretch_gamma"]
    c = table["cubic"]
    Lc = np.zeros((6, 6))
    Lc[:3, :3] = c["c12"]
    np.fill_diagonal(Lc[:3, :3], c["c11"])
    Lc[3, 3] = Lc[4, 4] = Lc[5, 5] = c["c44"]
    o = table["orthorhombic"]
    Lo = np.array([[o["c11"], o["c12"], o["c13"], 0, 0, 0],
                   [o["c12"], o["c22"], o["c23"], 0, 0, 0],
                   [o["c13"], o["c23"], o["c33"], 0, 0, 0],
                   [0, 0, 0, o["c44"], 0, 0],
                   [0, 0, 0, 0, o["c55"], 0],
                   [0, 0, 0, 0, 0, o["c66"]]], dtype=np.float64)
    R = np.eye(3) if orientation is None else np.asarray(orientation, dtype=np.float64)
    for i in range(7):
        U = np.array([P.Ut[i][k] for k in range(9)]).reshape(3, 3)
        if i == 0:
            L = Lc
        else:
            w, V = np.linalg.eigh(U)
            axes = np.stack([V[:, int(np.argmin(np.abs(w - t)))] for t in (al, be, ga)], axis=1)
            Mv = _bond(axes)  # variant frame -> crystal frame
            L = Mv @ Lo @ Mv.T
        Mr = _bond(R)
        L = Mr @ L @ Mr.T
        U = R @ U @ R.T
        for k in range(9):
            P.Ut[i][k] = U.reshape(9)[k]
        for k in range(36):
            P.Lvoigt[i][k] = L.reshape(36)[k]
    return P


_libs = {}


def lib_path(n_var: int = 6) -> str:
    """Path of the library built for n_var variants."""
    return LIB_PATH if n_var == 6 else os.path.join(LIB_DIR, f"nv{n_var}", f"libpfm_nv{n_var}.so")


def lib(n_var: int = 6):
    """The loaded CUDA library for n_var variants (6: libpfm.so, 12:
    libpfm_nv12.so); raises if it has not been built."""
    if n_var in _libs:
        return _libs[n_var]
    if n_var not in PARAMS:
        raise ValueError(f"no library for {n_var} variants (built: {sorted(PARAMS)})")
    path = lib_path(n_var)
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} not built: run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = C.CDLL(path)
    Params = PARAMS[n_var]
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int, C.c_double
    H = C.c_void_p
    sig = {
        "pfm_version": (C.c_char_p, []),
        "pfm_variants": (C.c_int, []),
        "pfm_create": (i32, [C.POINTER(MeshDesc), C.POINTER(Params), C.POINTER(H)]),
        "pfm_destroy": (None, [H]),
        "pfm_last_error": (C.c_char_p, [H]),
        "pfm_get_sizes": (i32, [H, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
        "pfm_set_stream": (i32, [H, vp]),
        "pfm_get_level": (i32, [H, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(dp)]),
        "pfm_set_power_iterations": (i32, [H, i32]),
        "pfm_set_outer_operator": (i32, [H, i32]),
        "pfm_set_deterministic": (i32, [H, i32]),
        "pfm_set_params": (i32, [H, C.POINTER(Params)]),
        "pfm_set_dirichlet": (i32, [H, vp, vp]),
        "pfm_set_state": (i32, [H, vp, vp]),
        "pfm_get_state": (i32, [H, vp]),
        "pfm_residual": (i32, [H, vp, C.POINTER(dp)]),
        "pfm_diagnostics": (i32, [H, vp, vp, vp, vp, vp]),
        "pfm_set_contact": (i32, [H, C.POINTER(dp), dp, dp]),
        "pfm_set_linearize_arithmetic": (i32, [H, i32]),
        "pfm_set_residual_arithmetic": (i32, [H, i32]),
        "pfm_set_preconditioner_store": (i32, [H, i32]),
        "pfm_contact_load": (i32, [H, C.POINTER(dp), C.POINTER(dp)]),
        "pfm_linearize": (i32, [H, i32]),
        "pfm_linearize_residual": (i32, [H, i32, vp, C.POINTER(dp)]),
        "pfm_jacobian_apply": (i32, [H, vp, vp, i32]),
        "pfm_jacobian_transpose_apply": (i32, [H, vp, vp, i32]),
        "pfm_jacobian_apply_host": (i32, [H, vp, vp, i32]),
        "pfm_jacobian_apply_mixed": (i32, [H, vp, vp]),
        "pfm_vcycle": (i32, [H, vp, vp, i32, C.POINTER(SolveOpts)]),
        "pfm_fgmres_solve": (i32, [H, C.POINTER(SolveOpts), vp, vp, C.POINTER(SolveReport)]),
        "pfm_newton_solve": (i32, [H, C.POINTER(SolveOpts), vp, C.POINTER(SolveReport)]),
        "pfm_qp_eval": (i32, [H, i64, vp, vp, vp, vp, vp, vp]),
        "pfm_get_hessians": (i32, [H, i64, i64, vp]),
        "pfm_get_block_inverses": (i32, [H, i32, i64, i64, vp]),
        "pfm_profile_enable": (i32, [H, i32]),
        "pfm_profile_get": (i32, [H, i32, C.POINTER(i64), C.POINTER(dp)]),
        "pfm_launch_count": (i64, []),
        "pfm_arith_peak": (i32, [i32, C.POINTER(dp)]),
        "pfm_param_grad": (i32, [H, vp, C.POINTER(dp), C.POINTER(dp), vp]),
        "pfm_batch_create": (i32, [C.POINTER(H), i32, C.POINTER(H)]),
        "pfm_batch_destroy": (None, [H]),
        "pfm_batch_last_error": (C.c_char_p, [H]),
        "pfm_batch_newton_solve": (i32, [H, C.POINTER(SolveOpts), C.POINTER(vp), C.POINTER(SolveReport)]),
        "pfm_batch_set_mode": (i32, [H, i32]),
        "pfm_residual_noalloc": (i32, [C.POINTER(MeshDesc), C.POINTER(Params), vp, vp, vp, vp,
                                       C.POINTER(dp), vp]),
        "pfm_noalloc_last_error": (C.c_char_p, []),
        "pfm_params_from_cubic": (i32, [C.POINTER(CubicMaterial), dp, i32, C.POINTER(Params)]),
        "pfm_params_orthorhombic_stiffness": (i32, [C.POINTER(Params), C.POINTER(dp), C.POINTER(dp),
                                                    C.POINTER(dp)]),
        "pfm_params_rotate": (i32, [C.POINTER(Params), C.POINTER(dp)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if L.pfm_variants() != n_var:
        raise RuntimeError(f"{path} was built for {L.pfm_variants()} variants, not {n_var}")
    _libs[n_var] = L
    return L


def n_var_of(params) -> int:
    """Number of variants of a parameter block (its library)."""
    return type(params).N_VAR


def exported_symbols():
    """Names of the entry points declared in include/pfm.h."""
    return [
        "pfm_version", "pfm_variants", "pfm_create", "pfm_destroy", "pfm_last_error", "pfm_get_sizes",
        "pfm_set_stream", "pfm_get_level", "pfm_set_power_iterations", "pfm_set_outer_operator", "pfm_set_deterministic", "pfm_set_params", "pfm_set_dirichlet", "pfm_set_state", "pfm_get_state",
        "pfm_residual", "pfm_diagnostics", "pfm_set_contact", "pfm_contact_load", "pfm_set_linearize_arithmetic", "pfm_set_residual_arithmetic", "pfm_set_preconditioner_store", "pfm_linearize", "pfm_linearize_residual", "pfm_jacobian_apply", "pfm_jacobian_transpose_apply",
        "pfm_jacobian_apply_host", "pfm_jacobian_apply_mixed", "pfm_vcycle", "pfm_fgmres_solve", "pfm_newton_solve",
        "pfm_qp_eval", "pfm_get_hessians", "pfm_get_block_inverses", "pfm_profile_enable", "pfm_profile_get",
        "pfm_launch_count", "pfm_arith_peak", "pfm_param_grad", "pfm_batch_create", "pfm_batch_destroy",
        "pfm_batch_last_error", "pfm_batch_newton_solve", "pfm_batch_set_mode", "pfm_residual_noalloc", "pfm_noalloc_last_error",
        "pfm_params_from_cubic", "pfm_params_orthorhombic_stiffness", "pfm_params_rotate",
    ]


__all__ = ["MeshDesc", "Params", "SolveOpts", "SolveReport", "params_from_material", "lib",
           "default_opts", "PFM_F32", "PFM_F64", "STATUS", "inputs"]
