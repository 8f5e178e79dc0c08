"""The largest eigenvalue of the Lanczos tridiagonal matrix behind the
smoother's eigenvalue estimate (csrc/common.cuh: tridiag_max_eig, bisection on
Sturm counts) compiled for the host by nvcc in a test-only shim and compared
with LAPACK's symmetric eigensolver (numpy.linalg.eigvalsh), and the cut at a
Lanczos breakdown (no GPU)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHIM = r'''
#include "paper_2011_08802_gb300/csrc/common.cuh"
extern "C" double host_tridiag_max(const double* a, const double* b2, int m) { return pfm::tridiag_max_eig(a, b2, m); }
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    d = tmp_path_factory.mktemp("lanczos")
    src, so = d / "lanczos.cu", d / "lanczos.so"
    src.write_text(SHIM)
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                           "-gencode", "arch=compute_103a,code=sm_103a", "-I", ROOT, "-o", str(so), str(src)])
    f = C.CDLL(str(so)).host_tridiag_max
    f.restype = C.c_double
    f.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int]
    return f


def _call(f, a, b2):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b2 = np.ascontiguousarray(np.append(b2, 0.0), dtype=np.float64)
    return f(a.ctypes.data_as(C.POINTER(C.c_double)), b2.ctypes.data_as(C.POINTER(C.c_double)), len(a))


def _exact(a, b2):
    T = np.diag(a) + np.diag(np.sqrt(b2), 1) + np.diag(np.sqrt(b2), -1)
    return np.linalg.eigvalsh(T).max()


def test_random_tridiagonals(lib):
    rng = np.random.default_rng(3)
    for m in list(range(1, 12)) + [20, 40, 64]:
        for _ in range(10):
            a = rng.normal(size=m) * rng.choice([1e-3, 1.0, 1e3])
            b2 = rng.random(m - 1) ** 2 * rng.choice([1e-6, 1.0, 1e4])
            ref = _exact(a, b2)
            assert abs(_call(lib, a, b2) - ref) <= 1e-12 * max(abs(ref), np.abs(a).max(), 1e-300), (m, a, b2)


def test_clustered_and_repeated_eigenvalues(lib):
    # T of a Lanczos run on a matrix with a dense top of the spectrum
    lam = np.concatenate([np.linspace(0.5, 3.9, 200), [4.0, 4.0 - 1e-9]])
    rng = np.random.default_rng(4)
    q = rng.normal(size=lam.size)
    q /= np.linalg.norm(q)
    a, b2, qp, beta = [], [], np.zeros_like(q), 0.0
    for _ in range(30):  # the Lanczos three-term recurrence on diag(lam) in FP64
        u = lam * q - beta * qp
        al = q @ u
        u -= al * q
        a.append(al)
        bb = u @ u
        b2.append(bb)
        qp, q, beta = q, u / np.sqrt(bb), np.sqrt(bb)
    a, b2 = np.array(a), np.array(b2[:-1])
    ref = _exact(a, b2)
    assert abs(_call(lib, a, b2) - ref) <= 1e-12 * ref
    assert 3.9 < ref <= 4.0 + 1e-12


def test_cut_at_breakdown_and_non_finite(lib):
    a = np.array([2.0, 5.0, 1.0, 7.0])
    # beta2 = 0 after step 2: an invariant subspace; only the leading 2 x 2 block counts
    b2 = np.array([1.0, 0.0, 4.0])
    assert abs(_call(lib, a, b2) - _exact(a[:2], b2[:1])) <= 1e-13 * 6
    b2 = np.array([1.0, np.nan, 4.0])
    assert abs(_call(lib, a, b2) - _exact(a[:2], b2[:1])) <= 1e-13 * 6
    a2 = np.array([2.0, 5.0, np.inf, 7.0])
    assert abs(_call(lib, a2, np.array([1.0, 1.0, 1.0])) - _exact(a2[:2], np.array([1.0]))) <= 1e-13 * 6
    assert np.isnan(_call(lib, np.array([np.nan]), np.array([])))
