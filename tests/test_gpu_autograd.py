"""Differentiation (GPU tests): forward-mode J v and reverse-mode J^T w of
the residual behind torch.autograd, derivatives with respect to the material
parameters theta = (C11, C12, C44, s_gamma), checked against the oracle and
against central finite differences; the adjoint gradient of a linear
functional of the Newton solution checked against finite differences."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

THETA0 = np.array([141.0, 126.0, 34.0, 1.0])


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import autograd, binding
    return autograd, binding


@pytest.fixture(scope="module")
def case(mods):
    autograd, binding = mods
    st = inputs.config_random(5, 4, 3, seed=51, eta_lo=-0.03, eta_hi=0.3, Lx=10.0, Ly=8.0, Lz=6.0)
    P = binding.problem_from_state(st)
    disc = fe.Discretisation(st.mesh)
    return st, P, disc


def _oracle_mat(st, theta):
    return qp.material_from(st.material, st.tau, C=tuple(theta[:3]), gamma_scale=theta[3])


def test_energy_and_residual_parameter_derivatives(case):
    st, P, disc = case
    P.set_state(torch.from_numpy(st.U).cuda(), torch.from_numpy(st.Un).cuda())
    w = np.random.default_rng(3).standard_normal(st.U.shape)
    dPi, wdR = P.param_grad(torch.from_numpy(w).cuda())
    E0 = fe.energy(disc, st, _oracle_mat(st, THETA0))
    R0 = fe.residual(disc, st, _oracle_mat(st, THETA0))
    for k in range(4):
        th = THETA0.copy()
        th[k] += 1.0  # Pi and R are affine in theta_k: the unit difference is the derivative
        dE = fe.energy(disc, st, _oracle_mat(st, th)) - E0
        dR = fe.residual(disc, st, _oracle_mat(st, th)) - R0
        assert abs(dPi[k] - dE) <= 1e-9 * abs(dE) + 1e-12, k
        assert abs(wdR[k] - (w * dR).sum()) <= 1e-9 * np.abs(w * dR).sum(), k


def test_autograd_backward_and_jvp(case, mods):
    autograd, _ = mods
    st, P, disc = case
    U = torch.from_numpy(st.U).cuda().requires_grad_(True)
    theta = torch.tensor(THETA0, dtype=torch.float64, device="cuda", requires_grad=True)
    Un = torch.from_numpy(st.Un).cuda()
    R = autograd.PFMResidual.apply(U, theta, P, Un, st.material, st.tau)
    mat = _oracle_mat(st, THETA0)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    assert np.abs(R.detach().cpu().numpy() - fe.residual(disc, st, mat, d)).max() < 1e-10 * np.abs(R.detach().cpu().numpy()).max()
    w = torch.from_numpy(np.random.default_rng(4).standard_normal(st.U.shape)).cuda()
    gU, gth = torch.autograd.grad((R * w).sum(), (U, theta))
    K = fe.tangent(disc, st, mat, d)
    gU_o = (K.T @ w.cpu().numpy().reshape(-1)).reshape(st.U.shape)
    # the tangent has identity rows/columns at Dirichlet DOFs; R is 0 there
    free = ~st.mask.astype(bool)
    assert np.abs(gU.cpu().numpy()[free] - gU_o[free]).max() < 1e-10 * np.abs(gU_o).max()
    _, wdR = P.param_grad(w)
    assert np.allclose(gth.cpu().numpy(), wdR, rtol=1e-12)
    # forward mode: J v through torch.func.jvp semantics of the Function
    v = torch.from_numpy(np.random.default_rng(5).standard_normal(st.U.shape)).cuda()
    P.set_state(U.detach(), Un)
    P.linearize(abi.PFM_F64)
    Jv = P.jacobian_apply(v).cpu().numpy()
    assert np.abs(Jv - (K @ v.cpu().numpy().reshape(-1)).reshape(Jv.shape)).max() < 1e-10 * np.abs(Jv).max()


def test_jvp_against_central_differences(case):
    """J v vs (R(U + h v) - R(U - h v)) / 2h, h = 1e-6, for 16 seeded
    directions with Dirichlet entries zeroed (the penalty kink is avoided by
    the smooth eta field away from zero)."""
    st0, P, disc = case
    st = inputs.config_random(5, 4, 3, seed=52, eta_lo=0.05, eta_hi=0.3, Lx=10.0, Ly=8.0, Lz=6.0)
    Ut = torch.from_numpy(st.U).cuda()
    Un = torch.from_numpy(st.Un).cuda()
    P.set_params(abi.params_from_material(st.material, st.tau))
    P.set_state(Ut, Un)
    P.linearize(abi.PFM_F64)
    V = inputs.direction_vectors(st, 16, seed=3)
    h = 1e-6
    for v in V:
        vt = torch.from_numpy(v).cuda()
        Jv = P.jacobian_apply(vt)
        P.set_state(Ut + h * vt, Un)
        Rp = P.residual().clone()
        P.set_state(Ut - h * vt, Un)
        Rm = P.residual().clone()
        P.set_state(Ut, Un)
        P.linearize(abi.PFM_F64)
        fd = (Rp - Rm) / (2 * h)
        free = torch.from_numpy(~st.mask.astype(bool)).cuda()
        err = (Jv - fd)[free].abs().max() / Jv.abs().max()
        assert err < 1e-6, float(err)


def test_adjoint_gradient_matches_finite_differences(mods):
    """g(theta) = w . U*(theta) with R(U*, theta) = 0: the adjoint gradient
    -lam . dR/dtheta (J^T lam = w) equals central differences of g."""
    autograd, binding = mods
    st = inputs.config_random(6, 5, 4, seed=61, eta_lo=0.02, eta_hi=0.3, Lx=12.0, Ly=10.0, Lz=8.0)
    w = torch.from_numpy(inputs.direction_vectors(st, 1, seed=7)[0]).cuda()
    Un = torch.from_numpy(st.Un).cuda()
    opts = abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-12, lin_rtol=1e-10, max_lin_it=600)

    def solve(theta):
        P = binding.problem_from_state(st, params=autograd.params_for(st.material, st.tau, theta))
        U = torch.from_numpy(st.U.copy()).cuda()
        P.newton_solve(U, opts, check=False)
        return P, U

    P, U = solve(THETA0)
    P.set_state(U, Un)
    g, lam, rep = autograd.adjoint_gradient(P, w)
    for k, step in ((0, 0.05), (2, 0.02), (3, 1e-4)):
        tp, tm = THETA0.copy(), THETA0.copy()
        tp[k] += step
        tm[k] -= step
        gp = float((w * solve(tp)[1]).sum())
        gm = float((w * solve(tm)[1]).sum())
        fd = (gp - gm) / (2 * step)
        assert abs(float(g[k]) - fd) <= 3e-5 * abs(fd) + 1e-9, (k, float(g[k]), fd)
