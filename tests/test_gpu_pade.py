"""Pade Hencky modes (Sec. 2.4, Eqs. pade11, pade22, pade33) on the GPU
against the oracle, which evaluates the paper's explicit matrix formulas
(GPU tests): Gauss-point physics including nearly repeated eigenvalues,
residual and energy, stored Hessians, FP64 tangent application and the
Newton correction of a mixed-precision solve, for each order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

MODES = ("pade11", "pade22", "pade33")


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module", params=MODES)
def ragged(binding, request):
    """6x5x3 hexes, eta_hat in [-0.04, 0.32] (penalty branch active)."""
    mode = request.param
    st = inputs.config_random(6, 5, 3, seed=33, eta_lo=-0.04, eta_hi=0.32, Lx=12.0, Ly=10.0, Lz=6.0)
    mat = qp.material_from(st.material, st.tau, hencky=mode)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    K = fe.tangent(disc, st, mat, d)
    P = binding.problem_from_state(st, params=abi.params_from_material(st.material, st.tau, hencky=mode))
    yield dict(mode=mode, st=st, mat=mat, disc=disc, d=d, K=K, P=P)
    P.close()


@pytest.mark.parametrize("mode", MODES)
def test_qp_physics(binding, mode):
    rng = np.random.default_rng(41)
    st = inputs.config_random(2, 2, 2, seed=1)
    mat = qp.material_from(st.material, st.tau, hencky=mode)
    B = 64
    F = np.eye(3) + 0.06 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(-0.05, 0.4, (B, 6))
    ehn = eh + 0.02 * rng.standard_normal((B, 6))
    for k in range(8):  # C^e = I exactly and nearly (F = F^t)
        e = np.zeros(6); e[k % 6] = 0.3 * (k + 1) / 8
        F[k] = np.einsum("i,ijk->jk", np.concatenate([[1 - e.sum()], e]), mat.U)
        eh[k] = e
        if k >= 4:
            F[k] = F[k] @ (np.eye(3) + 1e-7 * rng.standard_normal((3, 3)))
    F[8] = np.diag([1.02, 1.02, 0.97]); eh[8] = 0
    F[9] = np.diag([1.3, 0.8, 1.1]); eh[9] = 0   # large stretches
    W = qp.local_energy(F, eh, ehn, mat, order=2)
    P = binding.problem_from_state(st, params=abi.params_from_material(st.material, st.tau, hencky=mode))
    Wg, gg, Hg = P.qp_eval(torch.from_numpy(F.reshape(B, 9)).cuda(), torch.from_numpy(eh).cuda(),
                           torch.from_numpy(ehn).cuda())
    P.close()
    iu = np.triu_indices(15)
    assert _relerr(Wg.cpu().numpy(), W.v) < 1e-13
    assert _relerr(gg.cpu().numpy(), W.g) < 1e-13
    assert _relerr(Hg.cpu().numpy(), W.H[:, iu[0], iu[1]]) < 1e-12


def test_residual_and_energy(ragged):
    st, mat, disc, P = ragged["st"], ragged["mat"], ragged["disc"], ragged["P"]
    R, E = P.residual(energy=True)
    assert _relerr(R.cpu().numpy(), fe.residual(disc, st, mat, ragged["d"])) < 1e-11
    assert abs(E - fe.energy(disc, st, mat)) < 1e-12 * abs(E)


def test_stored_hessians_and_tangent(ragged):
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.linearize(abi.PFM_F32)
    iu = np.triu_indices(15)
    assert _relerr(P.get_hessians(0, P.n_elems), ragged["d"]["H"][:, :, iu[0], iu[1]]) < 1e-12
    v = np.random.default_rng(2).standard_normal(st.U.shape)
    y = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _relerr(y, (K @ v.reshape(-1)).reshape(v.shape)) < 1e-11


def test_newton_correction(ragged):
    P, K, st, disc, mat = ragged["P"], ragged["K"], ragged["st"], ragged["disc"], ragged["mat"]
    R = P.residual()
    P.linearize(abi.PFM_F32)
    # rtol 1e-12: this ragged state has cond(K) ~ 1e3, so 1e-10 leaves ~1e-7 of error
    x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-12, max_lin_it=300))
    Ro = fe.residual(disc, st, mat, ragged["d"])
    xo = fe.newton_correction(K, Ro)
    xg = x.cpu().numpy()
    assert np.linalg.norm(K @ xg.reshape(-1) + Ro.reshape(-1)) <= 1e-10 * np.linalg.norm(Ro)
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_modes_differ_as_the_approximation_order_predicts(binding):
    """At a finite-strain state the residuals of the four modes approach the
    exact-log residual as the order grows (Sec. 5.4: (2,2) and (3,3) close,
    (1,1) visibly off)."""
    st = inputs.config_random(4, 4, 4, seed=9, eta_lo=0.0, eta_hi=0.3)
    out = {}
    for mode in ("log",) + MODES:
        P = binding.problem_from_state(st, params=abi.params_from_material(st.material, st.tau, hencky=mode))
        out[mode] = P.residual().cpu().numpy()
        P.close()
    d = [np.abs(out[m] - out["log"]).max() for m in MODES]
    assert d[0] > d[1] > d[2] > 0.0


def test_invalid_mode_rejected(binding):
    st = inputs.config_random(2, 2, 2, seed=1)
    p = abi.params_from_material(st.material, st.tau)
    p.hencky = 4
    with pytest.raises(binding.PfmError):
        binding.problem_from_state(st, params=p)
