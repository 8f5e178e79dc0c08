"""Mixed-precision iterative refinement (GPU tests): opts.refine = 1 solves
the Newton system J dU = -R (Sec. 3.4, Eq. linAlgEq) by inner FGMRES cycles
with the FP32 tangent and the FP32 V-cycle, each followed by an FP64-class
true residual b - J x (double-float J x_hi plus FP32 J x_lo, or the FP64
kernel). The result meets the same tolerances against the oracle's direct
solve as the FGMRES whose every iteration applies the FP64-class operator."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _oracle(st):
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    K = fe.tangent(disc, st, mat, d)
    R = fe.residual(disc, st, mat, d)
    return K, R, fe.newton_correction(K, R)


@pytest.fixture(scope="module")
def ragged():
    st = inputs.config_random(9, 7, 6, seed=3, eta_lo=-0.03, eta_hi=0.3, Lx=18.0, Ly=14.0, Lz=12.0)
    return (st,) + _oracle(st)


@pytest.mark.parametrize("outer_df", [True, False])
@pytest.mark.parametrize("inner_rtol", [1e-2, 1e-4])
def test_refinement_matches_direct_solve(binding, ragged, outer_df, inner_rtol):
    st, K, R, dU = ragged
    P = binding.problem_from_state(st)
    P.set_outer_operator(outer_df)
    P.linearize(abi.PFM_F32)
    opts = abi.default_opts(abi.PFM_F32, lin_rtol=1e-10, refine=1, inner_rtol=inner_rtol, max_lin_it=300)
    x, rep = P.fgmres_solve(-P.residual(), opts)
    x = x.cpu().numpy()
    res = np.linalg.norm(K @ x.reshape(-1) + R.reshape(-1)) / np.linalg.norm(R)
    err = np.linalg.norm(x - dU) / np.linalg.norm(dU)
    assert res <= 1e-9 and err <= 1e-7, (res, err)
    # the reported relative residual is the FP64-class true residual
    assert rep.lin_res_final <= 1e-10
    assert rep.lin_res_final == pytest.approx(res, rel=1e-2, abs=1e-13)
    assert rep.lin_outer_last >= 2
    P.close()


def test_refinement_at_32_cubed_and_newton(binding):
    """The 32^3 indentation state, first load step: refinement and the plain
    mixed FGMRES both reach 1e-8 by the FP64 operator; a Newton solve with
    refinement converges like the plain one."""
    st = inputs.config_indentation(32, seed=2, step=1)
    P = binding.problem_from_state(st)
    R = P.residual()
    P.linearize(abi.PFM_F32)
    Rn = float(torch.linalg.norm(R))
    its = {}
    for refine in (0, 1):
        x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-8, max_lin_it=400, refine=refine))
        y = P.jacobian_apply(x)
        assert float(torch.linalg.norm(y + R)) <= 1e-8 * Rn
        its[refine] = rep.lin_its_last
    print("FGMRES iterations: plain", its[0], "refinement", its[1])
    assert its[1] <= 2 * its[0] + 10
    reps = []
    for refine in (0, 1):
        U = torch.from_numpy(st.U.copy()).cuda()
        reps.append(P.newton_solve(U, abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-8,
                                                       lin_rtol=1e-8, max_lin_it=400, refine=refine)))
    assert reps[1].res_final <= 1e-8 * reps[1].res0
    assert abs(reps[1].newton_its - reps[0].newton_its) <= 1
    P.close()


def test_refinement_options_are_checked(binding, ragged):
    st = ragged[0]
    P = binding.problem_from_state(st)
    P.linearize(abi.PFM_F32)
    R = P.residual()
    for bad in (0.0, 1.0, -1e-3):
        with pytest.raises(binding.PfmError) as exc:
            P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, refine=1, inner_rtol=bad))
        assert exc.value.status == 1
    P.close()
