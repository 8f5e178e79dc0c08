"""Binary16 Hessian store of the FP32 preconditioner (pfm_set_preconditioner_store)
against the oracle (GPU tests). The preconditioner's tangent application
reads per-level binary16 copies of s H (s a power of two), so it agrees with
the oracle's assembled tangent (Sec. 3.4) to the 11-bit rounding of the
entries; the Newton correction of the mixed solve, whose outer operator keeps
FP64-class accuracy, still equals the direct solve of the oracle's system."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import contact as C  # noqa: E402
from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

# binary16 keeps 11 significant bits: entries carry a relative rounding error
# of at most 2^-12; summed over the element contributions of one node the
# product then stays within a few 2^-12 of max |J v| per field
F16_TOL = 2e-3


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _oracle(st, constants=None):
    mat = qp.material_from(constants or st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    return fe.tangent(disc, st, mat, d), fe.residual(disc, st, mat, d)


def _field_errors(y, yo):
    return [np.abs(y[f] - yo[f]).max() / np.abs(yo[f]).max() for f in range(9)]


def _apply(P, v):
    return P.jacobian_apply(torch.from_numpy(v.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)


def test_application_from_binary16_store(binding):
    """6x5x3 hexes with the penalty branch active: the application from the
    binary16 copy is within the 11-bit rounding of the oracle's J v, visibly
    coarser than the FP32 store, and switching back restores the FP32 one."""
    st = inputs.config_random(6, 5, 3, seed=33, eta_lo=-0.04, eta_hi=0.32, Lx=12.0, Ly=10.0, Lz=6.0)
    K, _ = _oracle(st)
    P = binding.problem_from_state(st)
    v = np.random.default_rng(2).standard_normal(st.U.shape).astype(np.float32).astype(np.float64)
    yo = (K @ v.reshape(-1)).reshape(v.shape)
    P.linearize(abi.PFM_F32)
    e32 = max(_field_errors(_apply(P, v), yo))
    P.set_preconditioner_store(True)
    P.linearize(abi.PFM_F32)
    e16 = max(_field_errors(_apply(P, v), yo))
    P.set_preconditioner_store(False)
    P.linearize(abi.PFM_F32)
    e32b = max(_field_errors(_apply(P, v), yo))
    P.close()
    # the element contributions are added with atomics: same bound, not the same bits
    assert e32 < 2e-5 and e32b < 2e-5
    assert 10 * e32 < e16 < F16_TOL


def test_large_penalty_is_scaled_into_range(binding):
    """eps_eta = 1e6 GPa puts Hessian entries near 1e6, far above the binary16
    maximum (65504) unscaled; the per-level power-of-two scale keeps them."""
    st = inputs.config_random(5, 4, 3, seed=12, eta_lo=-0.05, eta_hi=0.3, Lx=10.0, Ly=8.0, Lz=6.0)
    constants = dict(st.material, eps_eta=1.0e6)
    K, _ = _oracle(st, constants)
    P = binding.problem_from_state(st, params=abi.params_from_material(constants, st.tau))
    P.set_preconditioner_store(True)
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(5).standard_normal(st.U.shape).astype(np.float32).astype(np.float64)
    yo = (K @ v.reshape(-1)).reshape(v.shape)
    y = _apply(P, v)
    P.close()
    assert np.all(np.isfinite(y))
    assert max(_field_errors(y, yo)) < F16_TOL


def test_newton_correction_matches_direct_solve(binding):
    st = inputs.config_random(6, 5, 3, seed=33, eta_lo=-0.04, eta_hi=0.32, Lx=12.0, Ly=10.0, Lz=6.0)
    K, Ro = _oracle(st)
    P = binding.problem_from_state(st)
    P.set_preconditioner_store(True)
    R = P.residual()
    P.linearize(abi.PFM_F32)
    x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-12, max_lin_it=300))
    P.close()
    xo = fe.newton_correction(K, Ro)
    xg = x.cpu().numpy()
    assert np.linalg.norm(K @ xg.reshape(-1) + Ro.reshape(-1)) <= 1e-10 * np.linalg.norm(Ro)
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_contact_on_non_nested_levels(binding):
    """9x7x6 hexes -> 5x4x3 -> 3x2x2 with a sphere pressing the free top
    face: binary16 copies on the two preconditioner levels, contact terms in
    FP32 beside them; the solve reaches the oracle's direct solution."""
    st = inputs.config_random(9, 7, 6, seed=8, Lx=18.0, Ly=14.0, Lz=12.0, top=False)
    sph = C.indenter(st.mesh, 0.8, 7.0, 100.0)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    _, Rc, Kc, _ = C.contact(st.mesh, st.U, sph)
    keep = sp.diags((~st.mask.reshape(-1).astype(bool)).astype(np.float64))
    K = (fe.tangent(disc, st, mat, d) + keep @ Kc @ keep).tocsr()
    Ro = fe.residual(disc, st, mat, d) + Rc * (~st.mask.astype(bool))
    P = binding.problem_from_state(st)
    assert P.n_levels == 3
    P.set_contact(sph.center, sph.radius, sph.eps_N)
    P.set_preconditioner_store(True)
    R = P.residual()
    P.linearize(abi.PFM_F32)
    x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, lin_rtol=1e-12, max_lin_it=400))
    P.close()
    xg = x.cpu().numpy().reshape(-1)
    assert np.linalg.norm(K @ xg + Ro.reshape(-1)) <= 1e-10 * np.linalg.norm(Ro)
    xo = -spla.splu(K.tocsc()).solve(Ro.reshape(-1))
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_invalid_value_rejected(binding):
    st = inputs.config_random(2, 2, 2, seed=1)
    P = binding.problem_from_state(st)
    with pytest.raises(binding.PfmError):
        P._check(P._lib.pfm_set_preconditioner_store(P.h, 2))
    P.close()
