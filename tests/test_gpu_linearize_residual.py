"""Residual formed by the linearisation pass (GPU tests): pfm_linearize_residual
(and the first residual of pfm_newton_solve) returns the residual and energy
of Sec. 3.4, Eq. FinalRes, from the same pass over the elements that computes
the Gauss-point Hessians (FP64 arithmetic; with double-float arithmetic in
either the call falls back to the two passes). Checked against the oracle
and the separate residual kernel, atomic and atomic-free, in both forms; the
tangent it leaves is the one pfm_linearize leaves (bitwise in the atomic-free
form)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

INVALID_ARG = 1  # pfm_status PFM_ERR_INVALID_ARG


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


@pytest.fixture(scope="module")
def ragged():
    # 9 x 7 x 6 elements: 378 elements = 94.5 warps of four, a ragged last block
    st = inputs.config_random(9, 7, 6, seed=161, eta_lo=-0.03, eta_hi=0.3, Lx=18.0, Ly=14.0, Lz=12.0)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    return st, fe.residual(disc, st, mat), fe.energy(disc, st, mat)


@pytest.mark.parametrize("det", [False, True])
@pytest.mark.parametrize("df", [False, True])
def test_fused_residual_matches_oracle_and_residual_kernel(binding, ragged, det, df):
    st, R, E = ragged
    P = binding.problem_from_state(st)
    P.set_deterministic(det)
    P.set_linearize_arithmetic(df)
    P.set_residual_arithmetic(df)
    Rf, Ef = P.linearize_residual(abi.PFM_F32, energy=True)
    assert np.abs(Rf.cpu().numpy() - R).max() <= 1e-11 * np.abs(R).max()
    assert abs(Ef - E) <= 1e-11 * abs(E)
    Rs, Es = P.residual(energy=True)
    assert float((Rf - Rs).abs().max()) <= 1e-13 * float(Rs.abs().max())
    assert abs(Ef - Es) <= 1e-13 * abs(Es)
    # Dirichlet rows are zero, as in the residual kernel
    m = torch.from_numpy(st.mask.astype(bool)).cuda()
    assert float(Rf[m].abs().max()) == 0.0
    # the tangent left behind is pfm_linearize's
    v = torch.from_numpy(np.random.default_rng(5).standard_normal(st.U.shape)).cuda()
    y1 = P.jacobian_apply(v)
    y1f = P.jacobian_apply(v.float())
    P.linearize(abi.PFM_F32)
    y2 = P.jacobian_apply(v)
    y2f = P.jacobian_apply(v.float())
    if det:
        assert torch.equal(y1, y2) and torch.equal(y1f, y2f)
    else:
        assert float((y1 - y2).abs().max()) <= 1e-13 * float(y2.abs().max())
        assert float((y1f - y2f).abs().max()) <= 1e-5 * float(y2f.abs().max())
    P.close()


def test_mixed_arithmetic_falls_back_to_two_passes(binding, ragged):
    st, R, E = ragged
    P = binding.problem_from_state(st)
    P.set_residual_arithmetic(True)  # double-float residual, FP64 linearisation
    Rf, Ef = P.linearize_residual(abi.PFM_F64, energy=True)
    Rs, Es = P.residual(energy=True)
    assert float((Rf - Rs).abs().max()) <= 1e-13 * float(Rs.abs().max())
    assert abs(Ef - E) <= 1e-11 * abs(E)
    P.close()


def test_newton_first_residual_comes_from_the_linearisation(binding, ragged):
    st, R, E = ragged
    P = binding.problem_from_state(st)
    r0 = float(torch.linalg.vector_norm(P.residual()))
    opts = abi.default_opts(abi.PFM_F32)
    opts.max_newton = 1
    U = torch.from_numpy(st.U.copy()).cuda()
    rep = P.newton_solve(U, opts)
    assert abs(rep.res0 - r0) <= 1e-13 * r0
    assert abs(rep.res0 - np.linalg.norm(R)) <= 1e-11 * np.linalg.norm(R)
    assert rep.newton_its == 1 and rep.ms_residual > 0.0 and rep.ms_linearize > 0.0
    P.close()


def test_argument_errors(binding, ragged):
    st, R, E = ragged
    P = binding.problem_from_state(st)
    lib = P._lib
    assert lib.pfm_linearize_residual(P.h, 7, None, None) == INVALID_ARG
    assert lib.pfm_linearize_residual(P.h, abi.PFM_F64, None, None) == INVALID_ARG
    assert lib.pfm_linearize_residual(None, abi.PFM_F64, None, None) == INVALID_ARG
    P.close()
