"""The C ABI's parameter builders (pfm_params_from_cubic,
pfm_params_orthorhombic_stiffness, pfm_params_rotate; host functions of the
library, no GPU) give the same parameter block as the binding's Python
construction from the constants of Sec. 5.1 and Table 1, and the printed
variant stretch patterns. Built library required (no compute call)."""
import ctypes as C
import os

import numpy as np
import pytest

from paper_2011_08802_gb300 import abi, inputs

pytestmark = pytest.mark.skipif(not os.path.exists(abi.lib_path(6)), reason="library not built")


def _arr(P, name):
    return np.array(getattr(P, name)).astype(np.float64)


def _same(Pa, Pb, tol=1e-13):
    for name, _ in Pa._fields_:
        a, b = np.array(getattr(Pa, name), dtype=np.float64), np.array(getattr(Pb, name), dtype=np.float64)
        scale = max(1.0, float(np.abs(b).max()))
        assert np.abs(a - b).max() <= tol * scale, name


def _from_cubic(hencky=0, tau=0.128):
    m = abi.CubicMaterial(**{k: inputs.MATERIAL[k] for k, _ in abi.CubicMaterial._fields_})
    P = abi.PARAMS[6]()
    assert abi.lib(6).pfm_params_from_cubic(C.byref(m), tau, hencky, C.byref(P)) == 0
    return P


def test_from_cubic_equals_python_builder():
    for hencky, name in ((0, "log"), (2, "pade22")):
        _same(_from_cubic(hencky), abi.params_from_material(inputs.MATERIAL, 0.128, hencky=name))


def test_orthorhombic_and_rotation_equal_python_builder():
    t = inputs.ELASTIC_TABLE1
    cub = (C.c_double * 3)(t["cubic"]["c11"], t["cubic"]["c12"], t["cubic"]["c44"])
    o = t["orthorhombic"]
    orth = (C.c_double * 9)(*[o[k] for k in ("c11", "c22", "c33", "c44", "c55", "c66", "c12", "c13", "c23")])
    axes = (C.c_double * 3)(*[inputs.MATERIAL[k] for k in ("stretch_alpha", "stretch_beta", "stretch_gamma")])
    R = (C.c_double * 9)(*np.asarray(inputs.ORIENTATION_011).reshape(9))
    P = _from_cubic()
    L = abi.lib(6)
    assert L.pfm_params_orthorhombic_stiffness(C.byref(P), cub, orth, axes) == 0
    assert L.pfm_params_rotate(C.byref(P), R) == 0
    _same(P, abi.params_anisotropic(inputs.MATERIAL, t, 0.128, inputs.ORIENTATION_011), tol=1e-12)


def test_printed_stretch_patterns_and_errors():
    P = _from_cubic()
    a, b, g = (inputs.MATERIAL[k] for k in ("stretch_alpha", "stretch_beta", "stretch_gamma"))
    U = _arr(P, "Ut").reshape(7, 3, 3)
    assert np.allclose(U[0], np.eye(3), rtol=0, atol=0)
    # the variants are stretches (symmetric), with eigenvalues alpha, beta, gamma
    for i in range(1, 7):
        assert np.array_equal(U[i], U[i].T)
        assert np.allclose(np.sort(np.linalg.eigvalsh(U[i])), sorted((a, b, g)), rtol=0, atol=1e-15)
    assert U[1][1, 1] == b and U[3][2, 2] == b and U[5][0, 0] == b
    L = abi.lib(6)
    m = abi.CubicMaterial()
    assert L.pfm_params_from_cubic(C.byref(m), 0.1, 7, C.byref(abi.PARAMS[6]())) == 1
    bad = (C.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 2)  # not orthogonal
    assert L.pfm_params_rotate(C.byref(P), bad) == 1
