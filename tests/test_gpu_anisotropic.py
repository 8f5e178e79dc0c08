"""Anisotropic CuAlNi stiffness (Table 1: cubic austenite, orthorhombic
martensite in each variant's principal axes) in the [011] orientation of
Sec. 5.1, on the GPU against the oracle (GPU tests). The binding builds the
per-phase Voigt matrices with Bond-matrix rotations, the oracle rotates the
fourth-order tensors directly; the kernels take the per-phase stiffness
path (L(eta) = sum eta_i L_i with distinct L_i)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

T1 = inputs.ELASTIC_TABLE1
R011 = inputs.ORIENTATION_011


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _params(st):
    return abi.params_anisotropic(st.material, T1, st.tau, R011)


def test_qp_physics(binding):
    rng = np.random.default_rng(51)
    st = inputs.config_random(2, 2, 2, seed=1)
    mat = qp.material_anisotropic(st.material, T1, st.tau, R011)
    B = 64
    F = np.eye(3) + 0.06 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(-0.05, 0.4, (B, 6))
    ehn = eh + 0.02 * rng.standard_normal((B, 6))
    for k in range(6):  # pure variants (C^e = I)
        e = np.zeros(6); e[k] = 1.0
        F[k] = mat.U[k + 1]
        eh[k] = e
    W = qp.local_energy(F, eh, ehn, mat, order=2)
    P = binding.problem_from_state(st, params=_params(st))
    Wg, gg, Hg = P.qp_eval(torch.from_numpy(F.reshape(B, 9)).cuda(), torch.from_numpy(eh).cuda(),
                           torch.from_numpy(ehn).cuda())
    P.close()
    iu = np.triu_indices(15)
    assert _relerr(Wg.cpu().numpy(), W.v) < 1e-13
    assert _relerr(gg.cpu().numpy(), W.g) < 1e-13
    assert _relerr(Hg.cpu().numpy(), W.H[:, iu[0], iu[1]]) < 1e-12


@pytest.fixture(scope="module")
def ragged(binding):
    st = inputs.config_random(6, 5, 4, seed=35, eta_lo=-0.03, eta_hi=0.32, Lx=12.0, Ly=10.0, Lz=8.0)
    mat = qp.material_anisotropic(st.material, T1, st.tau, R011)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    K = fe.tangent(disc, st, mat, d)
    P = binding.problem_from_state(st, params=_params(st))
    yield dict(st=st, mat=mat, disc=disc, d=d, K=K, P=P)
    P.close()


def test_residual_hessians_tangent(ragged):
    P, st, mat, disc, d, K = (ragged[k] for k in ("P", "st", "mat", "disc", "d", "K"))
    R, E = P.residual(energy=True)
    assert _relerr(R.cpu().numpy(), fe.residual(disc, st, mat, d)) < 1e-11
    assert abs(E - fe.energy(disc, st, mat)) < 1e-12 * abs(E)
    P.linearize(abi.PFM_F32)
    iu = np.triu_indices(15)
    assert _relerr(P.get_hessians(0, P.n_elems), d["H"][:, :, iu[0], iu[1]]) < 1e-12
    v = np.random.default_rng(2).standard_normal(st.U.shape)
    y = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _relerr(y, (K @ v.reshape(-1)).reshape(v.shape)) < 1e-11


def test_newton_correction(ragged):
    P, st, mat, disc, d, K = (ragged[k] for k in ("P", "st", "mat", "disc", "d", "K"))
    R = P.residual()
    P.linearize(abi.PFM_F32)
    x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-12, max_lin_it=300))
    Ro = fe.residual(disc, st, mat, d)
    xo = fe.newton_correction(K, Ro)
    xg = x.cpu().numpy()
    assert np.linalg.norm(K @ xg.reshape(-1) + Ro.reshape(-1)) <= 1e-10 * np.linalg.norm(Ro)
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)
