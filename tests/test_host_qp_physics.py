"""The CUDA path's point physics (csrc/qp_physics.cuh: energy, gradient and
the packed 15x15 Hessian in the condensed unknowns, Secs. 2-3) compiled for
the host by g++ in a test-only shim and compared with the oracle on the same
inputs (no GPU). The header's host branch is the code the kernels run, with
the FP64 eigensolve's FP32 seed included; the GPU tests repeat the comparison
through the C ABI. Cases: random states with the penalty branch active,
C^e = I exactly and nearly (pure variants), repeated and nearly repeated
eigenvalues, large stretches; every Hencky mode; the anisotropic material."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import qp
from paper_2011_08802_gb300 import abi, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHIM = r'''
#include "paper_2011_08802_gb300/csrc/params.h"
extern "C" void qp_host(const pfm_params* prm, int B, const double* F, const double* eh,
                        const double* ehn, double* W, double* g, double* H) {
  pfm::DevParams P;
  pfm::make_dev_params(*prm, P);
  for (int b = 0; b < B; ++b)
    pfm::qp_local<double, true>(P, F + 9 * b, eh + 6 * b, ehn + 6 * b, W + b, g + 15 * b, H + 120 * b);
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("qp_host")
    src, so = d / "qp_host.cpp", d / "qp_host.so"
    src.write_text(SHIM)
    subprocess.check_call([cxx, "-O2", "-shared", "-fPIC", "-std=c++17", "-I", ROOT, "-o", str(so), str(src)])
    return C.CDLL(str(so))


def _run(lib, prm, F, eh, ehn):
    B = F.shape[0]
    W, g, H = np.zeros(B), np.zeros((B, 15)), np.zeros((B, 120))

    def dp(a):
        return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(C.POINTER(C.c_double))

    Fc, ec, enc = (np.ascontiguousarray(x, dtype=np.float64) for x in (F.reshape(B, 9), eh, ehn))
    lib.qp_host(C.byref(prm), B, dp(Fc), dp(ec), dp(enc), dp(W), dp(g), dp(H))
    return W, g, H


def _states():
    rng = np.random.default_rng(41)
    st = inputs.config_random(2, 2, 2, seed=1)
    mat0 = qp.material_from(st.material, st.tau)
    B = 64
    F = np.eye(3) + 0.06 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(-0.05, 0.4, (B, 6))
    ehn = eh + 0.02 * rng.standard_normal((B, 6))
    for k in range(8):  # pure variants: C^e = I exactly, then perturbed by 1e-7
        e = np.zeros(6)
        e[k % 6] = 0.3 * (k + 1) / 8
        F[k] = np.einsum("i,ijk->jk", np.concatenate([[1 - e.sum()], e]), mat0.U)
        eh[k] = e
        if k >= 4:
            F[k] = F[k] @ (np.eye(3) + 1e-7 * rng.standard_normal((3, 3)))
    F[8] = np.diag([1.02, 1.02, 0.97]); eh[8] = 0            # a repeated eigenvalue
    F[9] = np.diag([1.3, 0.8, 1.1]); eh[9] = 0               # large stretches
    F[10] = np.diag([1.0, 1.0 + 1e-5, 1.0 + 3e-4]); eh[10] = 0  # a narrow spread
    F[11] = np.diag([1.01, 1.012, 1.008]); eh[11] = 0        # a spread near the series threshold
    return st, F, eh, ehn


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("mode", ["log", "pade11", "pade22", "pade33"])
def test_point_physics_matches_oracle(lib, mode):
    st, F, eh, ehn = _states()
    mat = qp.material_from(st.material, st.tau, hencky=mode)
    prm = abi.params_from_material(st.material, st.tau, hencky=mode)
    ref = qp.local_energy(F, eh, ehn, mat, order=2)
    W, g, H = _run(lib, prm, F, eh, ehn)
    iu = np.triu_indices(15)
    assert _rel(W, ref.v) < 1e-13
    assert _rel(g, ref.g) < 1e-13
    assert _rel(H, ref.H[:, iu[0], iu[1]]) < 1e-12


def test_anisotropic_point_physics_matches_oracle(lib):
    """Per-phase stiffness (Table 1 constants turned to [011]): the eta-
    dependence of L enters the gradient and every eta block of the Hessian."""
    st, F, eh, ehn = _states()
    mat = qp.material_anisotropic(st.material, inputs.ELASTIC_TABLE1, st.tau, inputs.ORIENTATION_011)
    prm = abi.params_anisotropic(st.material, inputs.ELASTIC_TABLE1, st.tau, inputs.ORIENTATION_011)
    ref = qp.local_energy(F, eh, ehn, mat, order=2)
    W, g, H = _run(lib, prm, F, eh, ehn)
    iu = np.triu_indices(15)
    assert _rel(W, ref.v) < 1e-13
    assert _rel(g, ref.g) < 1e-13
    assert _rel(H, ref.H[:, iu[0], iu[1]]) < 1e-12
