"""Parity of the multigrid-preconditioned FGMRES and of the Newton step with
the oracle's sparse direct solve (GPU tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

RES_TOL = 1e-8   # relative residual ||K x + R|| / ||R|| against the oracle's K
ERR_TOL = 1e-7   # relative error against the oracle's direct solution


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
def smooth8():
    st = inputs.config_smooth(8, seed=1)
    return (st,) + _oracle(st)


@pytest.fixture(scope="module")
def ragged_box():
    st = inputs.config_random(9, 7, 6, seed=3, eta_lo=-0.03, eta_hi=0.3, Lx=18.0, Ly=14.0, Lz=12.0)
    return (st,) + _oracle(st)


def _check_solution(K, R, x, dU):
    res = np.linalg.norm(K @ x.reshape(-1) + R.reshape(-1)) / np.linalg.norm(R)
    err = np.linalg.norm(x - dU) / np.linalg.norm(dU)
    assert res <= RES_TOL, res
    assert err <= ERR_TOL, err
    return res, err


@pytest.mark.parametrize("prec", [abi.PFM_F64, abi.PFM_F32])
def test_fgmres_matches_direct_solve(binding, smooth8, prec):
    st, K, R, dU = smooth8
    P = binding.problem_from_state(st)
    assert P.n_levels == 2
    P.linearize(prec)
    Rg = P.residual()
    x, rep = P.fgmres_solve(-Rg, abi.default_opts(prec, lin_rtol=1e-10))
    _check_solution(K, R, x.cpu().numpy(), dU)
    assert rep.lin_its_last < 60


@pytest.mark.parametrize("prec", [abi.PFM_F64, abi.PFM_F32])
def test_fgmres_non_nested_levels(binding, ragged_box, prec):
    st, K, R, dU = ragged_box
    P = binding.problem_from_state(st)
    assert P.n_levels == 3  # 9x7x6 -> 5x4x3 -> 3x2x2
    P.linearize(prec)
    x, rep = P.fgmres_solve(-P.residual(), abi.default_opts(prec, lin_rtol=1e-10))
    _check_solution(K, R, x.cpu().numpy(), dU)


@pytest.mark.parametrize("prec", [abi.PFM_F64, abi.PFM_F32])
def test_vcycle_reduces_residual(binding, smooth8, prec):
    st, K, R, dU = smooth8
    P = binding.problem_from_state(st)
    P.linearize(prec)
    dt = torch.float32 if prec == abi.PFM_F32 else torch.float64
    r = torch.from_numpy(-R).to(dt).cuda()
    z = P.vcycle(r).double().cpu().numpy()
    rz = (-R).reshape(-1) - K @ z.reshape(-1)
    assert np.linalg.norm(rz) < 0.5 * np.linalg.norm(R)
    assert np.all(z[st.mask.astype(bool)] == 0.0)


def test_newton_step_matches_oracle(binding, smooth8):
    st, K, R, dU = smooth8
    P = binding.problem_from_state(st)
    U = torch.from_numpy(st.U.copy()).cuda()
    rep = P.newton_solve(U, abi.default_opts(abi.PFM_F32, max_newton=1, lin_rtol=1e-10))
    assert rep.newton_its == 1
    Unew = U.cpu().numpy()
    assert np.linalg.norm(Unew - (st.U + dU)) <= ERR_TOL * np.linalg.norm(dU)
    assert abs(rep.res0 - np.linalg.norm(R)) <= 1e-10 * np.linalg.norm(R)


def test_newton_converges_quadratically(binding):
    """Newton's method (Eq. linAlgEq) on the first indentation load step.
    With linear solves to a relative residual eta = 1e-10 (inexact Newton),
    the relative residuals rho_k = ||R_k|| / ||R_0|| obey
    rho_{k+1} <= eta rho_k + C rho_k^2: quadratic once in the basin, until
    the eta rho_k and FP64 rounding floors. Asserted: 1e-9 within five
    corrections, and every step taken from 1e-7 < rho_k <= 1e-2 lands at or
    below 10 rho_k^2 (plus a 1e-12 floor), with at least one such step."""
    st = inputs.config_indentation(8, seed=5, step=1)
    P = binding.problem_from_state(st)
    U = torch.from_numpy(st.U.copy()).cuda()
    norms = []
    for _ in range(5):
        rep = P.newton_solve(U, abi.default_opts(abi.PFM_F32, max_newton=1, lin_rtol=1e-10, max_lin_it=600))
        norms.append(rep.res0)
    norms.append(rep.res_final)
    rho = [x / norms[0] for x in norms]
    print("relative Newton residuals:", " ".join(f"{r:.3e}" for r in rho))
    assert rho[-1] < 1e-9, rho
    basin = [k for k in range(1, len(rho) - 1) if 1e-7 < rho[k] <= 1e-2]
    assert basin, rho
    for k in basin:
        assert rho[k + 1] <= 10.0 * rho[k] ** 2 + 1e-12, (k, rho)


@pytest.mark.parametrize("prec", [abi.PFM_F32, abi.PFM_F64])
def test_single_level_grid(binding, prec):
    """A 4^3 grid is its own coarsest level: the preconditioner is the dense
    coarse solve, and the mixed solve's double-float outer operator still has
    its FP32 Hessian pair on that level."""
    st = inputs.config_indentation(4, seed=11, step=1)
    K, R, dU = _oracle(st)
    P = binding.problem_from_state(st)
    assert P.n_levels == 1
    P.linearize(prec)
    x, rep = P.fgmres_solve(-P.residual(), abi.default_opts(prec, lin_rtol=1e-10))
    _check_solution(K, R, x.cpu().numpy(), dU)
    assert rep.lin_its_last <= 3
