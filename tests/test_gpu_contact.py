"""Penalty contact with a rigid sphere (Sec. 2.5, Eq. PenPot) on the GPU
against the oracle (GPU tests): residual, energy and indenter load, tangent
applications in FP64, FP32 and double-float, the Newton correction of the
mixed solve against the direct solve of the assembled (volume + contact)
tangent, and contact on non-nested coarse levels."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import contact as C  # noqa: E402
from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _case(nx, ny, nz, seed, depth=0.6, radius=6.0, eps=100.0):
    """Top face free (only the bottom clamped), a sphere pressing its centre."""
    st = inputs.config_random(nx, ny, nz, seed=seed, Lx=2.0 * nx, Ly=2.0 * ny, Lz=2.0 * nz, top=False)
    sph = C.indenter(st.mesh, depth, radius, eps)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    Ec, Rc, Kc, load = C.contact(st.mesh, st.U, sph)
    keep = sp.diags((~st.mask.reshape(-1).astype(bool)).astype(np.float64))
    K = (fe.tangent(disc, st, mat, d) + keep @ Kc @ keep).tocsr()
    R = fe.residual(disc, st, mat, d) + Rc * (~st.mask.astype(bool))
    E = fe.energy(disc, st, mat) + Ec
    return dict(st=st, sph=sph, K=K, R=R, E=E, load=load, Ec=Ec)


@pytest.fixture(scope="module")
def case(binding):
    c = _case(7, 6, 4, seed=21)
    P = binding.problem_from_state(c["st"])
    P.set_contact(c["sph"].center, c["sph"].radius, c["sph"].eps_N)
    c["P"] = P
    yield c
    P.close()


def test_residual_energy_and_load(case):
    P = case["P"]
    R, E = P.residual(energy=True)
    assert _relerr(R.cpu().numpy(), case["R"]) < 1e-11
    assert abs(E - case["E"]) < 1e-12 * abs(case["E"])
    load, Ec = P.contact_load()
    assert case["load"] > 0.0
    assert abs(load - case["load"]) < 1e-11 * case["load"]
    assert abs(Ec - case["Ec"]) < 1e-11 * case["Ec"]


def test_tangent_applications(case):
    P, K, st = case["P"], case["K"], case["st"]
    P.linearize(abi.PFM_F32)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(st.U.shape)
    yo = (K @ v.reshape(-1)).reshape(v.shape)
    assert _relerr(P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy(), yo) < 1e-11
    v32 = v.astype(np.float32)
    yo32 = (K @ v32.astype(np.float64).reshape(-1)).reshape(v.shape)
    assert _relerr(P.jacobian_apply_mixed(torch.from_numpy(v32).cuda()).cpu().numpy(), yo32) < 1e-11
    y32 = P.jacobian_apply(torch.from_numpy(v32).cuda()).cpu().numpy()
    for f in range(9):
        assert np.abs(y32[f] - yo32[f]).max() <= 2e-5 * np.abs(yo32[f]).max()


@pytest.mark.parametrize("prec", [abi.PFM_F32, abi.PFM_F64])
def test_newton_correction_matches_direct_solve(case, prec):
    P, K = case["P"], case["K"]
    R = P.residual()
    P.linearize(prec)
    x, rep = P.fgmres_solve(-R, abi.default_opts(prec, lin_rtol=1e-12, max_lin_it=400))
    import scipy.sparse.linalg as spla
    xo = -spla.splu(K.tocsc()).solve(case["R"].reshape(-1))
    xg = x.cpu().numpy().reshape(-1)
    assert np.linalg.norm(K @ xg + case["R"].reshape(-1)) <= 1e-10 * np.linalg.norm(case["R"])
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_contact_on_non_nested_levels(binding):
    """9x7x6 hexes -> 5x4x3 -> 3x2x2: the contact term is re-discretised on
    every level; the preconditioned solve still reaches the direct solution."""
    c = _case(9, 7, 6, seed=8, depth=0.8, radius=7.0)
    P = binding.problem_from_state(c["st"])
    assert P.n_levels == 3
    P.set_contact(c["sph"].center, c["sph"].radius, c["sph"].eps_N)
    R = P.residual()
    assert _relerr(R.cpu().numpy(), c["R"]) < 1e-11
    P.linearize(abi.PFM_F32)
    x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-12, max_lin_it=400))
    xg = x.cpu().numpy().reshape(-1)
    assert np.linalg.norm(c["K"] @ xg + c["R"].reshape(-1)) <= 1e-10 * np.linalg.norm(c["R"])
    P.set_contact([0, 0, 0], 0.0, 1.0)  # off again: the plain residual
    st = c["st"]
    mat = qp.material_from(st.material, st.tau)
    assert _relerr(P.residual().cpu().numpy(), fe.residual(fe.Discretisation(st.mesh), st, mat)) < 1e-11
    P.close()
