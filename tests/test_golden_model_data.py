"""The model data used by both the oracle and the CUDA path against the values
the paper prints (no GPU): tests/golden/sec5_1_model_data.txt (Sec. 5.1) and
tests/golden/table1_elastic_constants.txt (Table 1), each line with its
citation. Unit conversions: 1 J/m^2 = 1 GPa nm, 1 MPa = 1e-3 GPa,
1 (MPa s)^-1 = 1e3 (GPa s)^-1. The variant stretches are checked as built by
the oracle and as handed to the C ABI, against the printed matrix patterns
filled with the printed alpha, beta, gamma (reading: '+' on the odd variant of
each pair)."""
import os

import numpy as np
import pytest

from oracle import qp
from paper_2011_08802_gb300 import abi, inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append(line.split())
    return rows


def _sec5_1():
    return {r[0]: (float(r[1]), r[2]) for r in _read("sec5_1_model_data.txt")}


TO_GPA_NM = {"J/m^2": 1.0, "MPa": 1e-3, "GPa": 1.0, "nm": 1.0, "1/(MPa*s)": 1e3, "-": 1.0}


@pytest.mark.parametrize("key, name", [
    ("alpha", "stretch_alpha"), ("beta", "stretch_beta"), ("gamma", "stretch_gamma"),
    ("gamma_am", "gamma_am"), ("gamma_mm", "gamma_mm"), ("F0_austenite", "F0_austenite"),
    ("F0_martensite", "F0_martensite"), ("mobility", "mobility"), ("ell", "ell"), ("eps_eta", "eps_eta"),
])
def test_sec5_1_constants(key, name):
    value, unit = _sec5_1()[key]
    assert inputs.MATERIAL[name] == pytest.approx(value * TO_GPA_NM[unit], rel=1e-15)


def test_every_fixture_line_is_checked():
    checked = {"alpha", "beta", "gamma", "gamma_am", "gamma_mm", "F0_austenite", "F0_martensite",
               "mobility", "ell", "eps_eta"}
    assert set(_sec5_1()) == checked


def test_table1_elastic_constants():
    rows = _read("table1_elastic_constants.txt")
    assert len(rows) == 12
    for phase, const, value in rows:
        assert inputs.ELASTIC_TABLE1[phase][const] == float(value), (phase, const)
    assert sum(len(v) for v in inputs.ELASTIC_TABLE1.values()) == 12


def _printed_stretches():
    g = _sec5_1()
    a, b, c = g["alpha"][0], g["beta"][0], g["gamma"][0]
    d, o = (a + c) / 2, (a - c) / 2
    U = []
    for s in (1.0, -1.0):  # U_1, U_2: (1,3) coupling, beta in the middle
        U.append([[d, 0, s * o], [0, b, 0], [s * o, 0, d]])
    for s in (1.0, -1.0):  # U_3, U_4: (1,2) coupling, beta last
        U.append([[d, s * o, 0], [s * o, d, 0], [0, 0, b]])
    for s in (1.0, -1.0):  # U_5, U_6: (2,3) coupling, beta first
        U.append([[b, 0, 0], [0, d, s * o], [0, s * o, d]])
    return np.array(U)


def test_variant_stretches_of_the_oracle():
    mat = qp.material_from(inputs.MATERIAL, tau=0.1)
    np.testing.assert_array_equal(mat.U[0], np.eye(3))
    np.testing.assert_allclose(mat.U[1:], _printed_stretches(), rtol=0, atol=1e-15)


def test_variant_stretches_given_to_the_c_abi():
    p = abi.params_from_material(inputs.MATERIAL, 0.1)
    Ut = np.array([[p.Ut[i][k] for k in range(9)] for i in range(7)]).reshape(7, 3, 3)
    np.testing.assert_array_equal(Ut[0], np.eye(3))
    np.testing.assert_allclose(Ut[1:], _printed_stretches(), rtol=0, atol=1e-15)
