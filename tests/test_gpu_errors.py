"""Failure detection through status codes (GPU tests). Every failure is made
on the host (a bad input, an iteration cap, a call out of order); nothing
faults, traps or hangs the GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

INVALID_ARG, NONFINITE, NOT_CONVERGED, STATE = 1, 4, 5, 8


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


@pytest.fixture()
def st():
    return inputs.config_random(5, 4, 4, seed=81, eta_lo=0.0, eta_hi=0.3, Lx=10.0, Ly=8.0, Lz=8.0)


def test_nonfinite_state_is_reported(binding, st):
    U = st.U.copy()
    U[4, 7] = np.nan
    P = binding.problem_from_state(st)
    Ut = torch.from_numpy(U).cuda()
    rep = P.newton_solve(Ut, abi.default_opts(), check=False)
    assert rep.status == NONFINITE


def test_iteration_cap_is_reported(binding, st):
    P = binding.problem_from_state(st)
    P.linearize(abi.PFM_F32)
    R = P.residual()
    x, rep = P.fgmres_solve(-R, abi.default_opts(max_lin_it=1, lin_rtol=1e-14), check=False)
    assert rep.status == NOT_CONVERGED and rep.lin_its_last == 1
    with pytest.raises(binding.PfmError) as e:
        P.fgmres_solve(-R, abi.default_opts(max_lin_it=1, lin_rtol=1e-14))
    assert e.value.status == NOT_CONVERGED


def test_prescribed_order_parameter_is_rejected(binding, st):
    P = binding.problem_from_state(st)
    m = st.mask.copy()
    m[5, 3] = 1
    with pytest.raises(binding.PfmError) as e:
        P.set_dirichlet(torch.from_numpy(m).cuda())
    assert e.value.status == INVALID_ARG


def test_calls_out_of_order_and_bad_options(binding, st):
    P = binding.Problem(st.mesh.nx, st.mesh.ny, st.mesh.nz, st.mesh.Lx, st.mesh.Ly, st.mesh.Lz,
                        abi.params_from_material(st.material, st.tau))
    with pytest.raises(binding.PfmError) as e:
        P.residual()
    assert e.value.status == STATE
    P.set_state(torch.from_numpy(st.U).cuda(), torch.from_numpy(st.Un).cuda())
    with pytest.raises(binding.PfmError) as e:
        P.jacobian_apply(torch.zeros(P.shape, dtype=torch.float64, device="cuda"))
    assert e.value.status == STATE
    P.linearize(abi.PFM_F64)
    with pytest.raises(binding.PfmError) as e:
        P.fgmres_solve(torch.zeros(P.shape, dtype=torch.float64, device="cuda"), abi.default_opts(restart=0))
    assert e.value.status == INVALID_ARG


def test_oversized_coarse_level_is_rejected(binding, st):
    with pytest.raises(binding.PfmError) as e:
        binding.Problem(16, 16, 16, 64.0, 64.0, 64.0, abi.params_from_material(st.material, st.tau), n_levels=1)
    assert e.value.status == INVALID_ARG


@pytest.mark.parametrize("dims, lengths, n_levels, tau", [
    ((0, 4, 4), (8.0, 8.0, 8.0), 0, 0.1),   # empty grid
    ((4, 4, 0), (8.0, 8.0, 8.0), 0, 0.1),
    ((4, 4, 4), (8.0, 0.0, 8.0), 0, 0.1),   # degenerate box
    ((4, 4, 4), (8.0, 8.0, 8.0), -1, 0.1),  # negative level count
    ((4, 4, 4), (8.0, 8.0, 8.0), 0, 0.0),   # no time increment
])
def test_empty_and_degenerate_problems_are_rejected(binding, st, dims, lengths, n_levels, tau):
    params = abi.params_from_material(st.material, tau if tau > 0 else 0.1)
    params.tau = tau
    with pytest.raises(binding.PfmError) as e:
        binding.Problem(*dims, *lengths, params, n_levels=n_levels)
    assert e.value.status == INVALID_ARG
