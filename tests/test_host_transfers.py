"""The CUDA path's multigrid transfers (csrc/mg_device.cuh: prolongation,
restriction, state injection at one node) compiled for the host by nvcc in a
test-only shim and compared with the oracle's definitions (oracle/transfer.py)
on nested, non-nested and one-column grids with Dirichlet masks (no GPU).
The CUDA side uses integer-exact weights, the oracle floating-point
coordinates, so they agree to rounding."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import transfer as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHIM = r'''
#include "paper_2011_08802_gb300/csrc/mg_device.cuh"
using namespace pfm;
static Grid grid(const int* n) {
  Grid g;
  g.nx = n[0]; g.ny = n[1]; g.nz = n[2];
  g.hx = g.hy = g.hz = 1.0;
  return g;
}
extern "C" void host_prolong(const int* fn, const int* cn, const double* xc, const unsigned short* mf, double* xf) {
  const Grid f = grid(fn), c = grid(cn);
  for (int64_t i = 0; i < f.nn(); ++i) prolong_node<double>(f, c, xc, mf, xf, i);
}
extern "C" void host_restrict(const int* fn, const int* cn, const double* rf, const unsigned short* mc, double* rc) {
  const Grid f = grid(fn), c = grid(cn);
  for (int64_t i = 0; i < c.nn(); ++i) restrict_node<double>(f, c, rf, mc, rc, i);
}
extern "C" void host_prolong_nested(const int* fn, const int* cn, const double* xc, const unsigned short* mf,
                                    double* xf) {
  const Grid f = grid(fn), c = grid(cn);
  for (int k = 0; k <= f.nz; ++k)
    for (int j = 0; j <= f.ny; ++j)
      for (int i = 0; i <= f.nx; ++i) prolong_node_nested<double>(f, c, xc, mf, xf, i, j, k);
}
extern "C" void host_restrict_nested(const int* fn, const int* cn, const double* rf, const unsigned short* mc,
                                     double* rc) {
  const Grid f = grid(fn), c = grid(cn);
  for (int k = 0; k <= c.nz; ++k)
    for (int j = 0; j <= c.ny; ++j)
      for (int i = 0; i <= c.nx; ++i) restrict_node_nested<double>(f, c, rf, mc, rc, i, j, k);
}
extern "C" void host_restrict_nested_f32(const int* fn, const int* cn, const float* rf, const unsigned short* mc,
                                         float* rc) {
  const Grid f = grid(fn), c = grid(cn);
  for (int k = 0; k <= c.nz; ++k)
    for (int j = 0; j <= c.ny; ++j)
      for (int i = 0; i <= c.nx; ++i) restrict_node_nested<float>(f, c, rf, mc, rc, i, j, k);
}
extern "C" int host_nested(const int* fn, const int* cn) { return nested(grid(fn), grid(cn)) ? 1 : 0; }
extern "C" void host_inject(const int* fn, const int* cn, const double* Uf, double* Uc) {
  const Grid f = grid(fn), c = grid(cn);
  for (int64_t i = 0; i < c.nn(); ++i) inject_node(f, c, Uf, Uc, i);
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    d = tmp_path_factory.mktemp("transfers")
    src, so = d / "transfers.cu", d / "transfers.so"
    src.write_text(SHIM)
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                           "-gencode", "arch=compute_103a,code=sm_103a", "-I", ROOT, "-o", str(so), str(src)])
    return C.CDLL(str(so))


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _bits(mask):
    """(9, n) 0/1 mask -> one uint16 per node, bit f = field f prescribed."""
    return np.ascontiguousarray((mask.astype(np.uint16) << np.arange(9, dtype=np.uint16)[:, None]).sum(0),
                                dtype=np.uint16)


PAIRS = [((8, 8, 8), (4, 4, 4)), ((9, 7, 6), (5, 4, 3)), ((5, 3, 2), (3, 2, 1)), ((1, 1, 300), (1, 1, 150)),
         ((24, 17, 11), (12, 9, 6))]


def _n(d):
    return (d[0] + 1) * (d[1] + 1) * (d[2] + 1)


@pytest.mark.parametrize("fine, coarse", PAIRS)
def test_transfers_match_oracle(lib, fine, coarse):
    rng = np.random.default_rng(sum(fine) + 7 * sum(coarse))
    nf, nc = _n(fine), _n(coarse)
    fn, cn = np.array(fine, dtype=np.int32), np.array(coarse, dtype=np.int32)
    mf = (rng.random((9, nf)) < 0.15).astype(np.uint8)
    mc = (rng.random((9, nc)) < 0.15).astype(np.uint8)
    d = C.c_double

    xc = rng.standard_normal((9, nc))
    xf0 = rng.standard_normal((9, nf))
    xf = xf0.copy()
    lib.host_prolong(_p(fn, C.c_int), _p(cn, C.c_int), _p(xc, d), _p(_bits(mf), C.c_ushort), _p(xf, d))
    np.testing.assert_allclose(xf, T.prolong_add(fine, coarse, xc, xf0, mf), rtol=0, atol=1e-13)

    rf = rng.standard_normal((9, nf))
    rc = np.zeros((9, nc))
    lib.host_restrict(_p(fn, C.c_int), _p(cn, C.c_int), _p(rf, d), _p(_bits(mc), C.c_ushort), _p(rc, d))
    np.testing.assert_allclose(rc, T.restrict(fine, coarse, rf, mc), rtol=0, atol=1e-12)

    Uf = rng.standard_normal((9, nf))
    Uc = np.zeros((9, nc))
    lib.host_inject(_p(fn, C.c_int), _p(cn, C.c_int), _p(Uf, d), _p(Uc, d))
    np.testing.assert_allclose(Uc, T.inject(fine, coarse, Uf), rtol=0, atol=1e-13)


@pytest.mark.parametrize("fine, coarse", [((8, 8, 8), (4, 4, 4)), ((24, 18, 10), (12, 9, 5)), ((2, 2, 2), (1, 1, 1)),
                                          ((2, 2, 300), (1, 1, 150))])
def test_nested_transfers_match_oracle(lib, fine, coarse):
    """The nested-grid node bodies (weights 1, 1/2 per axis) against the
    oracle's P and R = P^T, in FP64 and, for the restriction, in FP32."""
    rng = np.random.default_rng(3 * sum(fine) + sum(coarse))
    nf, nc = _n(fine), _n(coarse)
    fn, cn = np.array(fine, dtype=np.int32), np.array(coarse, dtype=np.int32)
    assert lib.host_nested(_p(fn, C.c_int), _p(cn, C.c_int)) == 1
    mf = (rng.random((9, nf)) < 0.15).astype(np.uint8)
    mf[:, 0] = 1  # one node with every field prescribed
    mc = (rng.random((9, nc)) < 0.15).astype(np.uint8)
    d = C.c_double
    xc = rng.standard_normal((9, nc))
    xf0 = rng.standard_normal((9, nf))
    xf = xf0.copy()
    lib.host_prolong_nested(_p(fn, C.c_int), _p(cn, C.c_int), _p(xc, d), _p(_bits(mf), C.c_ushort), _p(xf, d))
    np.testing.assert_allclose(xf, T.prolong_add(fine, coarse, xc, xf0, mf), rtol=0, atol=1e-13)
    rf = rng.standard_normal((9, nf))
    rc = np.zeros((9, nc))
    lib.host_restrict_nested(_p(fn, C.c_int), _p(cn, C.c_int), _p(rf, d), _p(_bits(mc), C.c_ushort), _p(rc, d))
    ref = T.restrict(fine, coarse, rf, mc)
    np.testing.assert_allclose(rc, ref, rtol=0, atol=1e-12)
    rf32 = rf.astype(np.float32)
    rc32 = np.zeros((9, nc), dtype=np.float32)
    lib.host_restrict_nested_f32(_p(fn, C.c_int), _p(cn, C.c_int), _p(rf32, C.c_float),
                                 _p(_bits(mc), C.c_ushort), _p(rc32, C.c_float))
    ref32 = T.restrict(fine, coarse, rf32.astype(np.float64), mc)
    np.testing.assert_allclose(rc32, ref32, rtol=0, atol=2e-6 * np.abs(ref32).max())


def test_non_nested_pairs_are_not_nested(lib):
    for fine, coarse in PAIRS[1:3]:
        fn, cn = np.array(fine, dtype=np.int32), np.array(coarse, dtype=np.int32)
        assert lib.host_nested(_p(fn, C.c_int), _p(cn, C.c_int)) == 0
