"""Thin Python binding of the C ABI (include/pfm.h). Each method has the name
of the entry point it calls (without the ``pfm_`` prefix) and only marshals
arguments: torch CUDA tensors are passed as device pointers, ctypes structs
as pointers, and a non-zero status raises ``PfmError`` with the library's
message. No computation happens here.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import abi
from .abi import PFM_F32, PFM_F64


class PfmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{abi.STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return C.c_void_p(t.ctypes.data)
    return t


def _prec(dtype) -> int:
    if dtype in (torch.float32, np.float32):
        return PFM_F32
    if dtype in (torch.float64, np.float64):
        return PFM_F64
    raise ValueError(f"unsupported dtype {dtype}")


class Problem:
    """One problem handle (``pfm_create``) on the current CUDA device, in the
    library built for the parameter block's number of variants (6 or 12)."""

    def __init__(self, nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float,
                 params, n_levels: int = 0, stream=None):
        self.n_var = abi.n_var_of(params)
        L = abi.lib(self.n_var)
        self._lib = L
        desc = abi.MeshDesc(nx, ny, nz, Lx, Ly, Lz, n_levels)
        h = C.c_void_p()
        st = L.pfm_create(C.byref(desc), C.byref(params), C.byref(h))
        if st != 0:
            raise PfmError(st, L.pfm_last_error(None).decode())
        self.h = h
        self.nx, self.ny, self.nz = nx, ny, nz
        nn, ne, nl = C.c_int64(), C.c_int64(), C.c_int()
        self._check(L.pfm_get_sizes(h, C.byref(nn), C.byref(ne), C.byref(nl)))
        self.n_nodes, self.n_elems, self.n_levels = nn.value, ne.value, nl.value
        self.shape = (3 + self.n_var, self.n_nodes)
        self.n_local = 9 + self.n_var                         # unknowns at a Gauss point
        self.n_hess = self.n_local * (self.n_local + 1) // 2  # packed Hessian entries
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())

    # -- helpers ---------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise PfmError(st, self._lib.pfm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.pfm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points ----------------------------------------------------
    def set_stream(self, stream):
        self.stream = stream
        self._check(self._lib.pfm_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def get_level(self, level: int):
        """(nx, ny, nz, lambda_max estimate) of multigrid level ``level``."""
        nx, ny, nz, lam = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        self._check(self._lib.pfm_get_level(self.h, level, C.byref(nx), C.byref(ny), C.byref(nz), C.byref(lam)))
        return nx.value, ny.value, nz.value, lam.value

    def set_outer_operator(self, double_float: bool):
        self._check(self._lib.pfm_set_outer_operator(self.h, int(double_float)))

    def set_deterministic(self, on: bool):
        """``pfm_set_deterministic``: atomic-free, bitwise reproducible element kernels."""
        self._check(self._lib.pfm_set_deterministic(self.h, int(on)))

    def set_power_iterations(self, its: int):
        self._check(self._lib.pfm_set_power_iterations(self.h, its))

    def set_params(self, params: abi.Params):
        self._check(self._lib.pfm_set_params(self.h, C.byref(params)))

    def set_dirichlet(self, mask: torch.Tensor, values: torch.Tensor | None = None):
        assert mask.dtype == torch.uint8 and mask.shape == self.shape
        if values is not None:
            assert values.dtype == torch.float64 and values.shape == self.shape
        self._check(self._lib.pfm_set_dirichlet(self.h, _ptr(mask), _ptr(values)))

    def set_state(self, U: torch.Tensor, Un: torch.Tensor):
        assert U.dtype == torch.float64 and U.shape == self.shape and Un.shape == self.shape
        self._check(self._lib.pfm_set_state(self.h, _ptr(U), _ptr(Un)))

    def get_state(self, U: torch.Tensor | None = None) -> torch.Tensor:
        U = torch.empty(self.shape, dtype=torch.float64, device="cuda") if U is None else U
        self._check(self._lib.pfm_get_state(self.h, _ptr(U)))
        return U

    def residual(self, R: torch.Tensor | None = None, energy: bool = False):
        R = torch.empty(self.shape, dtype=torch.float64, device="cuda") if R is None else R
        e = C.c_double()
        self._check(self._lib.pfm_residual(self.h, _ptr(R), C.byref(e) if energy else None))
        return (R, e.value) if energy else R

    def set_linearize_arithmetic(self, double_float: bool):
        """``pfm_set_linearize_arithmetic``: FP64 (False) or double-float (True)
        point physics in the FP64-class linearisation."""
        self._check(self._lib.pfm_set_linearize_arithmetic(self.h, int(bool(double_float))))

    def set_residual_arithmetic(self, double_float: bool):
        """``pfm_set_residual_arithmetic``: residual point physics in FP64 (False) or double-float (True)."""
        self._check(self._lib.pfm_set_residual_arithmetic(self.h, int(bool(double_float))))

    def set_preconditioner_store(self, half: bool):
        """``pfm_set_preconditioner_store``: the FP32 preconditioner reads its
        Gauss-point Hessians from the FP32 store (False) or from per-level
        binary16 copies scaled by a power of two (True)."""
        self._check(self._lib.pfm_set_preconditioner_store(self.h, int(bool(half))))

    def set_contact(self, center, radius: float, eps_N: float):
        """``pfm_set_contact``: rigid sphere (centre, radius) pressed on the top
        face with penalty eps_N; radius <= 0 switches contact off."""
        c = (C.c_double * 3)(*[float(x) for x in center])
        self._check(self._lib.pfm_set_contact(self.h, c, float(radius), float(eps_N)))

    def contact_load(self):
        """``pfm_contact_load``: (indenter load P, contact energy) at the current iterate."""
        P, E = C.c_double(), C.c_double()
        self._check(self._lib.pfm_contact_load(self.h, C.byref(P), C.byref(E)))
        return P.value, E.value

    def diagnostics(self, U: torch.Tensor | None = None, per_node: bool = True):
        """``pfm_diagnostics``: violation index I_v, diffuseness index I_d and
        eta* = eta_3 - eta_1 per node (if ``per_node``) and the per-plane
        statistics [nz+1][4] = (mean I_v, max I_v, mean I_d, max I_d) of U
        (default: the current iterate). Returns a dict of device tensors."""
        if U is not None:
            assert U.dtype == torch.float64 and U.shape == self.shape and U.is_contiguous()
        nn = self.shape[1]
        out = {}
        if per_node:
            for k in ("Iv", "Id", "eta_star"):
                out[k] = torch.empty(nn, dtype=torch.float64, device="cuda")
        out["planes"] = torch.empty(self.nz + 1, 4, dtype=torch.float64, device="cuda")
        self._check(self._lib.pfm_diagnostics(self.h, _ptr(U), _ptr(out.get("Iv")), _ptr(out.get("Id")),
                                              _ptr(out.get("eta_star")), _ptr(out["planes"])))
        return out

    def linearize(self, precond: int = PFM_F32):
        self._check(self._lib.pfm_linearize(self.h, precond))

    def linearize_residual(self, precond: int = PFM_F32, R: torch.Tensor | None = None, energy: bool = False):
        """linearize and residual of the same state in one pass."""
        R = torch.empty(self.shape, dtype=torch.float64, device="cuda") if R is None else R
        e = C.c_double()
        self._check(self._lib.pfm_linearize_residual(self.h, precond, _ptr(R), C.byref(e) if energy else None))
        return (R, e.value) if energy else R

    def jacobian_apply(self, v: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        y = torch.empty_like(v) if y is None else y
        self._check(self._lib.pfm_jacobian_apply(self.h, _ptr(v), _ptr(y), _prec(v.dtype)))
        return y

    def jacobian_transpose_apply(self, v: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        y = torch.empty_like(v) if y is None else y
        self._check(self._lib.pfm_jacobian_transpose_apply(self.h, _ptr(v), _ptr(y), _prec(v.dtype)))
        return y

    def jacobian_apply_mixed(self, v: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        """FP32 input, FP64 output, double-float arithmetic (pfm_jacobian_apply_mixed)."""
        assert v.dtype == torch.float32
        y = torch.empty(v.shape, dtype=torch.float64, device=v.device) if y is None else y
        self._check(self._lib.pfm_jacobian_apply_mixed(self.h, _ptr(v), _ptr(y)))
        return y

    def jacobian_apply_host(self, v: np.ndarray | torch.Tensor, y=None):
        if y is None:
            y = torch.empty_like(v) if isinstance(v, torch.Tensor) else np.empty_like(v)
        self._check(self._lib.pfm_jacobian_apply_host(self.h, _ptr(v), _ptr(y), _prec(v.dtype)))
        return y

    def vcycle(self, r: torch.Tensor, z: torch.Tensor | None = None, opts: abi.SolveOpts | None = None):
        z = torch.empty_like(r) if z is None else z
        self._check(self._lib.pfm_vcycle(self.h, _ptr(r), _ptr(z), _prec(r.dtype),
                                         C.byref(opts) if opts is not None else None))
        return z

    def fgmres_solve(self, b: torch.Tensor, opts: abi.SolveOpts, x: torch.Tensor | None = None,
                     check: bool = True):
        x = torch.empty_like(b) if x is None else x
        rep = abi.SolveReport()
        st = self._lib.pfm_fgmres_solve(self.h, C.byref(opts), _ptr(b), _ptr(x), C.byref(rep))
        if check:
            self._check(st)
        return x, rep

    def newton_solve(self, U: torch.Tensor, opts: abi.SolveOpts, check: bool = True):
        rep = abi.SolveReport()
        st = self._lib.pfm_newton_solve(self.h, C.byref(opts), _ptr(U), C.byref(rep))
        if check:
            self._check(st)
        return rep

    def qp_eval(self, F: torch.Tensor, eta: torch.Tensor, eta_n: torch.Tensor, hessian: bool = True):
        n = F.shape[0]
        W = torch.empty(n, dtype=torch.float64, device="cuda")
        g = torch.empty(n, self.n_local, dtype=torch.float64, device="cuda")
        H = torch.empty(n, self.n_hess, dtype=torch.float64, device="cuda") if hessian else None
        self._check(self._lib.pfm_qp_eval(self.h, n, _ptr(F), _ptr(eta), _ptr(eta_n), _ptr(W), _ptr(g), _ptr(H)))
        return W, g, H

    def param_grad(self, w: torch.Tensor | None = None, dR: torch.Tensor | None = None):
        """(dPi/dtheta, w . dR/dtheta) for theta = (C11, C12, C44, s_gamma);
        dR (device double (4, 9, n_nodes)), if given, receives dR/dtheta."""
        dPi = (C.c_double * 4)()
        wdR = (C.c_double * 4)()
        self._check(self._lib.pfm_param_grad(self.h, _ptr(w), dPi, wdR, _ptr(dR)))
        return np.array(dPi[:]), (np.array(wdR[:]) if w is not None else None)

    def profile_enable(self, enable: bool = True):
        self._check(self._lib.pfm_profile_enable(self.h, int(enable)))

    def profile_get(self, phase: int):
        n, ms = C.c_int64(), C.c_double()
        self._check(self._lib.pfm_profile_get(self.h, phase, C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def get_block_inverses(self, level: int, n0: int, count: int) -> np.ndarray:
        """``pfm_get_block_inverses``: (count, nf, nf) inverted nodal diagonal blocks."""
        nf = self.shape[0]
        out = np.empty((count, nf, nf))
        self._check(self._lib.pfm_get_block_inverses(self.h, level, n0, count, _ptr(out)))
        return out

    def get_hessians(self, e0: int, count: int) -> np.ndarray:
        out = np.empty((count, 8, self.n_hess))
        self._check(self._lib.pfm_get_hessians(self.h, e0, count, _ptr(out)))
        return out


class Batch:
    """``pfm_batch_create`` over existing problems (which must outlive it)."""

    def __init__(self, problems):
        self.problems = list(problems)
        L = abi.lib(self.problems[0].n_var if self.problems else 6)
        self._lib = L
        arr = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        b = C.c_void_p()
        st = L.pfm_batch_create(arr, len(self.problems), C.byref(b))
        if st != 0:
            raise PfmError(st, L.pfm_batch_last_error(None).decode())
        self.b = b

    def set_mode(self, mode: int):
        """``pfm_batch_set_mode``: 0 = batched engine (default), 1 = lockstep."""
        st = self._lib.pfm_batch_set_mode(self.b, int(mode))
        if st != 0:
            raise PfmError(st, self._lib.pfm_batch_last_error(self.b).decode())

    def newton_solve(self, states, opts: abi.SolveOpts, check: bool = True):
        arr = (C.c_void_p * len(states))(*[U.data_ptr() for U in states])
        reps = (abi.SolveReport * len(states))()
        st = self._lib.pfm_batch_newton_solve(self.b, C.byref(opts), arr, reps)
        if check and st != 0:
            raise PfmError(st, self._lib.pfm_batch_last_error(self.b).decode())
        return list(reps)

    def close(self):
        if getattr(self, "b", None):
            self._lib.pfm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def residual_noalloc(mesh, params: abi.Params, mask: torch.Tensor, U: torch.Tensor, Un: torch.Tensor,
                     R: torch.Tensor | None = None, stream=None):
    """``pfm_residual_noalloc``: residual and potential without a handle and
    without device allocation by the library (R is allocated here by torch
    only when the caller passes none). Returns (R, energy)."""
    L = abi.lib(abi.n_var_of(params))
    R = torch.empty_like(U) if R is None else R
    desc = abi.MeshDesc(mesh.nx, mesh.ny, mesh.nz, mesh.Lx, mesh.Ly, mesh.Lz, 0)
    e = C.c_double()
    s = stream if stream is not None else torch.cuda.current_stream()
    st = L.pfm_residual_noalloc(C.byref(desc), C.byref(params), _ptr(mask), _ptr(U), _ptr(Un), _ptr(R),
                                C.byref(e), C.c_void_p(s.cuda_stream))
    if st != 0:
        raise PfmError(st, L.pfm_noalloc_last_error().decode())
    return R, e.value


def arith_peak(precision: int) -> float:
    """``pfm_arith_peak``: measured FMA throughput (TFLOP/s) of the current device."""
    t = C.c_double()
    st = abi.lib().pfm_arith_peak(precision, C.byref(t))
    if st != 0:
        raise PfmError(st, "arithmetic peak probe failed")
    return t.value


def launch_count() -> int:
    """Kernel launches issued by the library in this process (``pfm_launch_count``)."""
    return int(abi.lib().pfm_launch_count())


def levels_to(n: int, coarsest: int = 4) -> int:
    """Number of levels of the ceil-halving hierarchy of an n-element edge
    down to the first level with at most ``coarsest`` elements per edge (the
    library's default is coarsest = 4)."""
    levels = 1
    while n > coarsest and n > 1:
        n = (n + 1) // 2
        levels += 1
    return levels


def problem_from_state(state, n_levels: int = 0, params=None) -> Problem:
    """Create a handle for an ``inputs.State`` and load its mask and state."""
    m = state.mesh
    if params is None:
        params = abi.params_from_material(state.material, state.tau)
    P = Problem(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz, params, n_levels)
    P.set_dirichlet(torch.from_numpy(state.mask).cuda())
    P.set_state(torch.from_numpy(state.U).cuda(), torch.from_numpy(state.Un).cuda())
    return P
