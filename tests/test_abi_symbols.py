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
