"""Deterministic mode (GPU tests): with pfm_set_deterministic(h, 1) (or
opts.deterministic) every element kernel adds its contributions without
atomics, so repeated runs on the same data are bitwise equal: the residual
and energy, the FP32, FP64, binary16 and double-float tangent applications
(the tangent of Sec. 3.4, Eq. linAlgEq), and a whole mixed-precision Newton
correction. Parity with the oracle is unchanged."""
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


@pytest.fixture(scope="module")
def ragged():
    st = inputs.config_random(9, 7, 6, seed=81, eta_lo=-0.03, eta_hi=0.3, Lx=18.0, Ly=14.0, Lz=12.0)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    K = fe.tangent(disc, st, mat, d)
    R = fe.residual(disc, st, mat, d)
    return st, K, R, fe.newton_correction(K, R), fe.energy(disc, st, mat)


def test_residual_and_energy_bitwise_and_oracle(binding, ragged):
    st, K, R, dU, E = ragged
    P = binding.problem_from_state(st)
    P.set_deterministic(True)
    R1, E1 = P.residual(energy=True)
    R2, E2 = P.residual(energy=True)
    assert torch.equal(R1, R2) and E1 == E2
    assert np.abs(R1.cpu().numpy() - R).max() <= 1e-11 * np.abs(R).max()
    assert abs(E1 - E) <= 1e-11 * abs(E)
    # the atomic form gives the same values up to rounding
    P.set_deterministic(False)
    R3, E3 = P.residual(energy=True)
    assert float((R3 - R1).abs().max()) <= 1e-13 * float(R1.abs().max())
    P.close()


@pytest.mark.parametrize("half", [False, True])
def test_tangent_applications_bitwise_and_oracle(binding, ragged, half):
    st, K, R, dU, E = ragged
    P = binding.problem_from_state(st)
    P.set_deterministic(True)
    P.set_preconditioner_store(half)
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(3).standard_normal(st.U.shape)
    v32 = torch.from_numpy(v.astype(np.float32)).cuda()
    v64 = torch.from_numpy(v).cuda()
    outs = {}
    for name, fn, arg in (("f32", P.jacobian_apply, v32), ("f64", P.jacobian_apply, v64),
                          ("df", P.jacobian_apply_mixed, v32)):
        a, b = fn(arg), fn(arg)
        assert torch.equal(a, b), name
        outs[name] = a.double().cpu().numpy()
    Kv = (K @ v.reshape(-1)).reshape(v.shape)
    Kv32 = (K @ v.astype(np.float32).astype(np.float64).reshape(-1)).reshape(v.shape)

    def err(y, yo):  # worst per-field error relative to the field's largest entry
        return max(np.abs(y[f] - yo[f]).max() / np.abs(yo[f]).max() for f in range(9))

    assert err(outs["f64"], Kv) <= 1e-11
    assert err(outs["df"], Kv32) <= 1e-11
    # binary16 store: 11-bit entries; FP32 store: FP32 rounding
    assert err(outs["f32"], Kv32) <= (2e-3 if half else 2e-5)
    P.close()


def test_newton_correction_bitwise_and_oracle(binding, ragged):
    """A whole mixed-precision Newton correction (residual, linearisation of
    every level, FGMRES with the FP32 V-cycle and the double-float outer
    operator, update) twice with opts.deterministic: bitwise equal iterates;
    the correction equals the oracle's direct solve."""
    st, K, R, dU, E = ragged
    P = binding.problem_from_state(st)
    opts = abi.default_opts(abi.PFM_F32, max_newton=1, lin_rtol=1e-10, deterministic=1)
    outs = []
    for _ in range(2):
        U = torch.from_numpy(st.U.copy()).cuda()
        rep = P.newton_solve(U, opts)
        assert rep.newton_its == 1
        outs.append(U)
    assert torch.equal(outs[0], outs[1])
    x = outs[0].cpu().numpy() - st.U
    assert np.linalg.norm(K @ x.reshape(-1) + R.reshape(-1)) <= 1e-8 * np.linalg.norm(R)
    assert np.linalg.norm(x - dU) <= 1e-7 * np.linalg.norm(dU)
    P.close()


def test_contact_is_rejected_in_deterministic_mode(binding):
    st = inputs.config_indentation(6, seed=82, step=1)
    P = binding.problem_from_state(st)
    P.set_contact(np.array([32.0, 32.0, 64.0 + 30.0]), 30.5, 100.0)
    P.set_deterministic(True)
    with pytest.raises(binding.PfmError) as exc:
        P.residual()
    assert exc.value.status == 1 and "contact" in str(exc.value)
    P.close()
