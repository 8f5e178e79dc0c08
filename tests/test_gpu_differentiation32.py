"""Differentiation at 32^3 (GPU tests): the state after five load steps of the
indentation ramp, 16 seeded direction vectors (Dirichlet entries zeroed).
Forward products J v against central differences of the residual
(h = 1e-6, FP64) and against the oracle's rows at sampled nodes, reverse
products against <w, J v> = <J^T w, v>, parameter derivatives of the energy
against exact differences (the energy is affine in each parameter), and 16
adjoint solves J^T lam = w checked through lam . J v = w . v."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

N = 32


@pytest.fixture(scope="module")
def loaded():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding, driver
    st = inputs.config_indentation(N, seed=2, step=1)
    P = binding.problem_from_state(st)
    U, reps = driver.load_ramp(P, st, upto=5)
    assert all(r.status == 0 for r in reps)
    Un = U.clone()
    mask, values = inputs.indentation_dirichlet(st.mesh, 5)
    st5 = inputs.State(st.mesh, U.cpu().numpy(), Un.cpu().numpy(), mask, st.tau, st.material)
    P.set_state(U, Un)
    P.linearize(abi.PFM_F32)
    V = inputs.direction_vectors(st5, 16, seed=3)
    yield dict(P=P, st=st5, U=U, Un=Un, V=V)
    P.close()


def test_jvp_central_differences(loaded):
    P, U, Un, V, st = loaded["P"], loaded["U"], loaded["Un"], loaded["V"], loaded["st"]
    free = torch.from_numpy(~st.mask.astype(bool)).cuda()
    h = 1e-6
    errs = []
    for v in V:
        vt = torch.from_numpy(v).cuda()
        P.set_state(U, Un)
        P.linearize(abi.PFM_F64)
        Jv = P.jacobian_apply(vt)
        P.set_state(U + h * vt, Un)
        Rp = P.residual().clone()
        P.set_state(U - h * vt, Un)
        Rm = P.residual().clone()
        fd = (Rp - Rm) / (2 * h)
        errs.append(float((Jv - fd)[free].abs().max() / Jv.abs().max()))
    P.set_state(U, Un)
    # the strict penalty kink can sit inside +-h v at a few points; all but at most one direction clean
    errs.sort()
    assert errs[-2] < 1e-6, errs


def test_jvp_rows_against_oracle(loaded):
    P, st, V = loaded["P"], loaded["st"], loaded["V"]
    P.set_state(loaded["U"], loaded["Un"])
    P.linearize(abi.PFM_F64)
    mat = qp.material_from(st.material, st.tau)
    m = st.mesh
    v = V[0]
    y = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
    for (i, j, k) in ((16, 16, 32), (16 + 9, 16, 32), (5, 7, 3), (31, 2, 20)):
        n = i + (m.nx + 1) * (j + (m.ny + 1) * k)
        ids = [a + m.nx * (b + m.ny * c) for c in range(max(k - 1, 0), min(k, m.nz - 1) + 1)
               for b in range(max(j - 1, 0), min(j, m.ny - 1) + 1)
               for a in range(max(i - 1, 0), min(i, m.nx - 1) + 1)]
        disc = fe.Discretisation(m, elements=ids)
        d = fe.qp_derivatives(disc, st, mat, order=2)
        yo = fe.jvp(disc, st, v, d)[:, n]
        assert np.abs(y[:, n] - yo).max() <= 1e-11 * np.abs(y).max()


def test_vjp_consistency(loaded):
    P, V = loaded["P"], loaded["V"]
    P.set_state(loaded["U"], loaded["Un"])
    P.linearize(abi.PFM_F64)
    for a in range(0, 16, 2):
        v, w = torch.from_numpy(V[a]).cuda(), torch.from_numpy(V[a + 1]).cuda()
        lhs = float((w * P.jacobian_apply(v)).sum())
        rhs = float((P.jacobian_transpose_apply(w) * v).sum())
        assert abs(lhs - rhs) <= 1e-11 * float((w * P.jacobian_apply(v)).abs().sum())


def test_energy_parameter_gradient(loaded):
    from paper_2011_08802_gb300 import autograd
    P, st = loaded["P"], loaded["st"]
    theta = np.array([141.0, 126.0, 34.0, 1.0])
    P.set_state(loaded["U"], loaded["Un"])
    dPi, _ = P.param_grad(None)
    for k in range(4):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += 1.0
        tm[k] -= 1.0
        P.set_params(autograd.params_for(st.material, st.tau, tp))
        _, Ep = P.residual(energy=True)
        P.set_params(autograd.params_for(st.material, st.tau, tm))
        _, Em = P.residual(energy=True)
        assert abs(dPi[k] - (Ep - Em) / 2.0) <= 1e-9 * abs(dPi[k]) + 1e-12, k
    P.set_params(autograd.params_for(st.material, st.tau, theta))


def test_adjoint_solves_for_sixteen_directions(loaded):
    from paper_2011_08802_gb300 import autograd
    P, V = loaded["P"], loaded["V"]
    P.set_state(loaded["U"], loaded["Un"])
    v = torch.from_numpy(np.random.default_rng(11).standard_normal(V[0].shape)).cuda()
    v[torch.from_numpy(loaded["st"].mask.astype(bool)).cuda()] = 0.0
    for w in V:
        wt = torch.from_numpy(w).cuda()
        g, lam, rep = autograd.adjoint_gradient(P, wt)
        assert rep.lin_res_final <= 1e-10
        P.linearize(abi.PFM_F64)
        lhs = float((lam * P.jacobian_apply(v)).sum())
        rhs = float((wt * v).sum())
        assert abs(lhs - rhs) <= 1e-7 * abs(rhs) + 1e-9 * float((wt * v).abs().sum())
        assert np.all(np.isfinite(g.numpy()))
