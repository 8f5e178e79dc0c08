"""The C ABI library loads and exports every entry point that include/*.h
declares (no GPU needed, no compute call)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

from paper_2011_08802_gb300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(pfm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(abi.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and nvcc unavailable")
        from paper_2011_08802_gb300 import build
        build.build()
    return ctypes.CDLL(abi.LIB_PATH)


def test_header_declares_the_entry_points():
    names = _declared()
    assert set(abi.exported_symbols()) <= set(names)
    assert set(names) <= set(abi.exported_symbols()), set(names) - set(abi.exported_symbols())


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_string(lib):
    f = lib.pfm_version
    f.restype = ctypes.c_char_p
    assert f().decode().startswith("pfm")


def _body(src, signature):
    """Text of the function whose definition starts with ``signature`` (brace matched)."""
    i = src.index(signature)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[j:k + 1]
    raise AssertionError(f"unbalanced braces after {signature}")


def test_noalloc_path_names_no_allocator():
    """pfm_residual_noalloc and the two launchers it calls make no device
    allocation: no call of cudaMalloc* (or cudaFree*) anywhere in its file or in
    those launchers' bodies."""
    csrc = os.path.join(ROOT, "paper_2011_08802_gb300", "csrc")
    call = re.compile(r"\b(cudaMalloc\w*|cudaFree\w*|cuMemAlloc\w*)\s*\(")
    code = lambda t: re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", t, flags=re.S))
    noalloc = code(open(os.path.join(csrc, "noalloc.cu")).read())
    assert not call.search(noalloc)
    fe = code(open(os.path.join(csrc, "fe_kernels.cu")).read())
    kr = code(open(os.path.join(csrc, "krylov_kernels.cu")).read())
    assert not call.search(_body(fe, "void launch_residual("))
    assert not call.search(_body(kr, "void launch_build_mask("))


@pytest.mark.parametrize("n_var", [6, 12])
def test_libraries_export_only_the_c_abi(lib, n_var):
    """Both libraries (6 and 12 variants, built from the same sources) export
    the pfm_* entry points and nothing else, and define no process-wide unique
    symbols, so one process can load both without their internal state (e.g.
    function-local statics of templates) being merged."""
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("no nm")
    path = abi.lib_path(n_var)
    if not os.path.exists(path):
        pytest.skip("library not built")
    import subprocess
    out = subprocess.check_output([nm, "-D", "--defined-only", path], text=True).split("\n")
    names = [ln.split()[-1] for ln in out if ln.strip()]
    assert names and all(n.startswith("pfm_") for n in names), [n for n in names if not n.startswith("pfm_")][:5]
    kinds = [ln.split()[1] for ln in subprocess.check_output([nm, path], text=True).split("\n") if len(ln.split()) == 3]
    assert "u" not in kinds
