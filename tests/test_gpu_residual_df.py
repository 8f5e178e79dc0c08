"""Residual point physics in double-float arithmetic (GPU tests):
pfm_set_residual_arithmetic(h, 1) evaluates the residual (Sec. 3.4,
Eq. FinalRes) and energy with pairs of FP32 numbers (about 48 bits) on the
FP32 pipes; against the oracle it meets the FP64 residual's tolerance, and a
mixed Newton solve with it converges as with the FP64 residual."""
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


@pytest.mark.parametrize("hencky", ["log", "pade22"])
def test_double_float_residual_matches_oracle(binding, hencky):
    st = inputs.config_random(7, 5, 4, seed=141, eta_lo=-0.03, eta_hi=0.32, Lx=14.0, Ly=10.0, Lz=8.0)
    mat = qp.material_from(st.material, st.tau, hencky=hencky)
    disc = fe.Discretisation(st.mesh)
    R = fe.residual(disc, st, mat)
    E = fe.energy(disc, st, mat)
    P = binding.problem_from_state(st, params=abi.params_from_material(st.material, st.tau, hencky=hencky))
    P.set_residual_arithmetic(True)
    Rg, Eg = P.residual(energy=True)
    assert np.abs(Rg.cpu().numpy() - R).max() <= 1e-11 * np.abs(R).max()
    assert abs(Eg - E) <= 1e-11 * abs(E)
    P.set_residual_arithmetic(False)
    R64 = P.residual()
    assert float((R64 - Rg).abs().max()) <= 1e-12 * float(R64.abs().max())
    P.close()


def test_newton_with_double_float_residual(binding):
    st = inputs.config_indentation(16, seed=8, step=1)
    P = binding.problem_from_state(st)
    opts = abi.default_opts(abi.PFM_F32, max_newton=8, newton_rtol=1e-8, lin_rtol=1e-8, max_lin_it=300, krylov=1,
                            switch_rtol=1e-4)
    reps = []
    for df in (False, True):
        P.set_residual_arithmetic(df)
        U = torch.from_numpy(st.U.copy()).cuda()
        reps.append((P.newton_solve(U, opts), U.cpu().numpy()))
    (r64, U64), (rdf, Udf) = reps
    assert rdf.res_final <= 1e-8 * rdf.res0 and rdf.newton_its == r64.newton_its
    assert np.linalg.norm(Udf - U64) <= 1e-7 * np.linalg.norm(U64 - st.U)
    P.close()
