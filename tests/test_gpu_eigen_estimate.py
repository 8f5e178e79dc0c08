"""The smoother's eigenvalue estimate (Lanczos steps for J D^-1 in the D^-1
inner product, pfm_linearize) against the exact largest eigenvalue of
D^-1 J (GPU tests): J assembled column by column from the library's FP64
tangent application on a ragged grid, D its 9 x 9 nodal diagonal blocks, and
the generalised symmetric eigenproblem J x = lambda D x solved by LAPACK. The
Ritz value lies below lambda_max and close to it; more steps bring it closer."""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")

from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _dense_tangent(P):
    shape = P.shape
    n = shape[0] * shape[1]
    J = np.empty((n, n))
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    for i in range(n):
        e.zero_()
        e[i] = 1.0
        J[:, i] = P.jacobian_apply(e.view(shape)).reshape(-1).cpu().numpy()
    return J


@pytest.mark.parametrize("steps", [10, 30])
def test_lanczos_estimate_below_and_near_lambda_max(binding, steps):
    st = inputs.config_random(6, 5, 4, seed=17, eta_lo=-0.02, eta_hi=0.3, Lx=12.0, Ly=10.0, Lz=8.0)
    P = binding.problem_from_state(st, n_levels=2)
    P.set_power_iterations(steps)
    P.linearize(abi.PFM_F64)
    lam = P.get_level(0)[3]
    J = _dense_tangent(P)
    P.close()
    nn = st.U.shape[1]
    D = np.zeros_like(J)
    for node in range(nn):
        idx = node + nn * np.arange(9)
        D[np.ix_(idx, idx)] = J[np.ix_(idx, idx)]
    J = 0.5 * (J + J.T)
    exact = sla.eigh(J, D, eigvals_only=True).max()
    print(f"{steps} Lanczos steps: {lam:.6f}, lambda_max {exact:.6f}")
    assert lam <= exact * (1 + 1e-10)
    assert lam >= (0.97 if steps == 10 else 0.999) * exact
