"""Microstructure diagnostics of Sec. 5.3 (violation index, diffuseness
index, eta* and their per-plane mean and maximum) on the GPU against the
oracle (GPU tests): a ragged box, a one-column grid with many planes, and
every node of the 128^3 indentation state with a seeded perturbation that
makes some eta_i negative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import diagnostics as D  # noqa: E402
from paper_2011_08802_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _check(P, st, U=None):
    Uh = st.U if U is None else U
    out = P.diagnostics(None if U is None else torch.from_numpy(U).cuda())
    # eta* is one subtraction (bit-exact); I_v and I_d sum seven terms, and
    # I_d = 1 - sum eta^4 with eta_0 near 1 loses a few ulps of 1 to rounding order
    np.testing.assert_array_equal(out["eta_star"].cpu().numpy(), D.composite(Uh))
    for key, ref in (("Iv", D.violation_index(Uh)), ("Id", D.diffuseness_index(Uh))):
        got = out[key].cpu().numpy()
        assert np.abs(got - ref).max() <= 8 * 2.0 ** -52 * max(1.0, np.abs(ref).max()), key
    S = out["planes"].cpu().numpy()
    So = D.plane_statistics(st.mesh, Uh)
    assert np.abs(S[:, [1, 3]] - So[:, [1, 3]]).max() <= 8 * 2.0 ** -52
    assert np.abs(S[:, [0, 2]] - So[:, [0, 2]]).max() <= 1e-14
    return S


def test_ragged_box_with_violations(binding):
    st = inputs.config_random(7, 5, 3, seed=31, eta_lo=-0.04, eta_hi=0.32, Lx=14.0, Ly=10.0, Lz=6.0)
    P = binding.problem_from_state(st)
    S = _check(P, st)
    assert S[:, 1].max() > 0.0  # some constraint is violated
    P.close()


def test_one_column_many_planes(binding):
    st = inputs.config_random(1, 1, 300, seed=2, eta_lo=-0.05, eta_hi=0.3, Lx=1.0, Ly=1.0, Lz=300.0)
    P = binding.problem_from_state(st)
    _check(P, st)
    P.close()


def test_explicit_state_and_pure_phases(binding):
    st = inputs.config_random(4, 3, 2, seed=5)
    P = binding.problem_from_state(st)
    U = np.zeros_like(st.U)
    U[3 + 2] = 1.0  # variant 3 everywhere
    S = _check(P, st, U)
    assert np.all(S == 0.0)
    assert np.all(P.diagnostics(torch.from_numpy(U).cuda())["eta_star"].cpu().numpy() == 1.0)
    P.close()


def test_full_size_indentation_state(binding):
    st = inputs.config_indentation(128, seed=5, step=1)
    U = st.U.copy()
    U[3:9] += 0.02 * np.random.default_rng(17).standard_normal(U[3:9].shape)
    P = binding.problem_from_state(st)
    S = _check(P, st, U)
    assert S.shape == (129, 4) and S[:, 1].max() > 0.0
    P.close()
