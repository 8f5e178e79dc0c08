"""The element-index division of the staged tangent application
(csrc/common.cuh: FastDiv, a multiply-high and a shift) compiled for the host
by nvcc in a test-only shim and compared with integer division (no GPU): every
divisor 1..2048 and the grid extents up to 2^16, numerators at both ends of
the range the kernel uses (n < 2^31), multiples of d and their neighbours."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHIM = r'''
#include "paper_2011_08802_gb300/csrc/common.cuh"
extern "C" long long host_fastdiv_mismatches(const unsigned* d, int nd, const unsigned* n, int nn) {
  long long bad = 0;
  for (int i = 0; i < nd; ++i) {
    const pfm::FastDiv f = pfm::FastDiv::make(d[i]);
    for (int j = 0; j < nn; ++j) {
      const unsigned x = n[j] & 0x7fffffffu;
      if (f.div(x) != x / d[i]) ++bad;
      // multiples of d and their neighbours
      const unsigned q = x / d[i];
      const unsigned long long m = (unsigned long long)q * d[i];
      if (m > 0 && f.div(unsigned(m - 1)) != unsigned(m - 1) / d[i]) ++bad;
      if (f.div(unsigned(m)) != q) ++bad;
    }
  }
  return bad;
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    d = tmp_path_factory.mktemp("fastdiv")
    src, so = d / "fastdiv.cu", d / "fastdiv.so"
    src.write_text(SHIM)
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                           "-gencode", "arch=compute_103a,code=sm_103a", "-I", ROOT, "-o", str(so), str(src)])
    return C.CDLL(str(so))


def test_fastdiv_equals_integer_division(lib):
    rng = np.random.default_rng(11)
    divisors = np.concatenate([np.arange(1, 2049), rng.integers(2049, 1 << 16, 2000),
                               np.array([1 << 16, (1 << 16) - 1, 3 * 5 * 7 * 11 * 13, 1 << 20, 1000003])])
    divisors = np.ascontiguousarray(divisors, dtype=np.uint32)
    nums = np.concatenate([np.arange(0, 4096), (1 << 31) - 1 - np.arange(0, 4096),
                           rng.integers(0, 1 << 31, 20000)])
    nums = np.ascontiguousarray(nums, dtype=np.uint32)
    lib.host_fastdiv_mismatches.restype = C.c_longlong
    bad = lib.host_fastdiv_mismatches(divisors.ctypes.data_as(C.POINTER(C.c_uint)), len(divisors),
                                      nums.ctypes.data_as(C.POINTER(C.c_uint)), len(nums))
    assert bad == 0
