"""Mixed-precision Krylov modes that apply the FP64-class outer operator
less often (GPU tests), for the Newton system J dU = -R (Sec. 3.4,
Eq. linAlgEq):
* opts.krylov = 1, relaxed products: FGMRES applies the FP64-class operator
  while its residual estimate is above switch_rtol ||b|| and the FP32
  operator after it; the FP64-class true residual b - J x (double-float
  J x_hi plus FP32 J x_lo, or the FP64 kernel) decides convergence;
* opts.krylov = 2, iterative refinement: inner FGMRES cycles with the FP32
  tangent and the FP32 V-cycle, each followed by that true residual.
Both meet the same tolerances against the oracle's direct solve as the
FGMRES whose every iteration applies the FP64-class operator."""
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
@pytest.mark.parametrize("mode, switch", [(1, 1e-2), (1, 1e-4), (2, 1e-2), (2, 1e-4)])
def test_modes_match_direct_solve(binding, ragged, outer_df, mode, switch):
    st, K, R, dU = ragged
    P = binding.problem_from_state(st)
    P.set_outer_operator(outer_df)
    P.linearize(abi.PFM_F32)
    opts = abi.default_opts(abi.PFM_F32, lin_rtol=1e-10, krylov=mode, switch_rtol=switch, max_lin_it=300)
    x, rep = P.fgmres_solve(-P.residual(), opts)
    x = x.cpu().numpy()
    res = np.linalg.norm(K @ x.reshape(-1) + R.reshape(-1)) / np.linalg.norm(R)
    err = np.linalg.norm(x - dU) / np.linalg.norm(dU)
    assert res <= 1e-9 and err <= 1e-7, (res, err)
    # the reported relative residual is the FP64-class true residual
    assert rep.lin_res_final <= 1e-10
    assert rep.lin_res_final == pytest.approx(res, rel=1e-2, abs=1e-13)
    assert rep.lin_outer_last >= (2 if mode == 2 else 1)
    P.close()


def test_modes_at_32_cubed_and_newton(binding):
    """The 32^3 indentation state, first load step: every mode reaches 1e-8
    by the FP64 operator; Newton solves in each mode converge alike."""
    st = inputs.config_indentation(32, seed=2, step=1)
    P = binding.problem_from_state(st)
    R = P.residual()
    P.linearize(abi.PFM_F32)
    Rn = float(torch.linalg.norm(R))
    its = {}
    modes = ((0, 1e-3), (1, 1e-3), (2, 1e-4))
    for mode, sw in modes:
        x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-8, max_lin_it=400, krylov=mode,
                                                      switch_rtol=sw))
        y = P.jacobian_apply(x)
        assert float(torch.linalg.norm(y + R)) <= 1e-8 * Rn
        its[mode] = rep.lin_its_last
    print("FGMRES iterations by mode:", its)
    assert its[1] <= its[0] + 5 and its[2] <= 2 * its[0] + 10
    reps = []
    for mode, sw in modes:
        U = torch.from_numpy(st.U.copy()).cuda()
        reps.append(P.newton_solve(U, abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-8,
                                                       lin_rtol=1e-8, max_lin_it=400, krylov=mode,
                                                       switch_rtol=sw)))
    for r in reps[1:]:
        assert r.res_final <= 1e-8 * r.res0
        assert abs(r.newton_its - reps[0].newton_its) <= 1
    P.close()


def test_mode_options_are_checked(binding, ragged):
    st = ragged[0]
    P = binding.problem_from_state(st)
    P.linearize(abi.PFM_F32)
    R = P.residual()
    for mode, bad in ((1, 0.0), (2, 1.0), (1, -1e-3), (3, 1e-3)):
        with pytest.raises(binding.PfmError) as exc:
            P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, krylov=mode, switch_rtol=bad))
        assert exc.value.status == 1
    P.close()
