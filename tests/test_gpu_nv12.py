"""Twelve variants on the GPU (GPU tests): the library built with N = 12
(libpfm_nv12.so; 15 unknowns per node, 21 at a Gauss point, 231 Hessian
entries) against the oracle with the same twelve-variant material: the
Gauss-point physics, the residual (Sec. 3.4, Eq. FinalRes), the stored
Hessians, the FP64 / FP32 / double-float tangent applications (Eq. linAlgEq)
on a ragged grid with the penalty branch active, and the mixed-precision
Newton correction against the oracle's sparse direct solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

NV = 12


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


@pytest.fixture(scope="module")
def ragged():
    st = inputs.config_random(6, 5, 4, seed=121, eta_lo=-0.01, eta_hi=0.07, Lx=12.0, Ly=10.0, Lz=8.0, n_var=NV)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh, n_var=NV)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    return dict(st=st, mat=mat, disc=disc, d=d, K=fe.tangent(disc, st, mat, d), R=fe.residual(disc, st, mat, d))


def test_both_libraries_in_one_process(binding, ragged):
    """A six-variant problem linearised first, then a twelve-variant one on two
    levels: each library keeps its own launch settings (the diagonal-block
    kernel's shared-memory size differs between them)."""
    st6 = inputs.config_random(6, 5, 4, seed=123, eta_lo=0.0, eta_hi=0.3, Lx=12.0, Ly=10.0, Lz=8.0)
    P6 = binding.problem_from_state(st6)
    P6.linearize(abi.PFM_F32)
    P6.linearize(abi.PFM_F64)
    P12 = binding.problem_from_state(ragged["st"])
    assert P12.n_levels == 2
    P12.linearize(abi.PFM_F32)
    P12.linearize(abi.PFM_F64)
    P6.linearize(abi.PFM_F32)
    P6.close()
    P12.close()


def test_library_has_twelve_variants(binding, ragged):
    P = binding.problem_from_state(ragged["st"])
    assert P.n_var == NV and P.shape == (15, ragged["st"].mesh.n_nodes)
    assert abi.lib(NV).pfm_variants() == NV
    P.close()


def test_point_physics(binding, ragged):
    st, mat = ragged["st"], ragged["mat"]
    rng = np.random.default_rng(5)
    n = 64
    F = np.eye(3) + 0.06 * rng.standard_normal((n, 3, 3))
    eh = rng.uniform(0.0, 0.08, (n, NV))
    eh[::7, 2] = -0.02  # penalty branch
    ehn = eh - 0.004
    P = binding.problem_from_state(st)
    W, g, H = P.qp_eval(torch.from_numpy(F.reshape(n, 9)).cuda(), torch.from_numpy(eh).cuda(),
                        torch.from_numpy(ehn).cuda())
    Wo = qp.local_energy(F, eh, ehn, mat, order=2)
    iu = np.triu_indices(9 + NV)
    Ho = Wo.H[:, iu[0], iu[1]]
    assert np.abs(W.cpu().numpy() - Wo.v).max() <= 1e-12 * np.abs(Wo.v).max()
    assert np.abs(g.cpu().numpy() - Wo.g).max() <= 1e-12 * np.abs(Wo.g).max()
    assert np.abs(H.cpu().numpy() - Ho).max() <= 1e-12 * np.abs(Ho).max()
    P.close()


def test_residual_hessians_and_tangent(binding, ragged):
    st, K, R, d = ragged["st"], ragged["K"], ragged["R"], ragged["d"]
    P = binding.problem_from_state(st)
    Rg, E = P.residual(energy=True)
    assert np.abs(Rg.cpu().numpy() - R).max() <= 1e-11 * np.abs(R).max()
    Eo = fe.energy(ragged["disc"], st, ragged["mat"])
    assert abs(E - Eo) <= 1e-11 * abs(Eo)
    P.linearize(abi.PFM_F32)
    iu = np.triu_indices(9 + NV)
    Hg = P.get_hessians(0, st.mesh.n_elems)
    Ho = d["H"][:, :, iu[0], iu[1]]
    assert np.abs(Hg - Ho).max() <= 1e-12 * np.abs(Ho).max()
    v = np.random.default_rng(6).standard_normal(st.U.shape)
    v32 = v.astype(np.float32)
    Kv = (K @ v.reshape(-1)).reshape(v.shape)
    Kv32 = (K @ v32.astype(np.float64).reshape(-1)).reshape(v.shape)

    def err(y, yo):
        return max(np.abs(y[f] - yo[f]).max() / np.abs(yo[f]).max() for f in range(15))

    assert err(P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy(), Kv) <= 1e-11
    assert err(P.jacobian_apply_mixed(torch.from_numpy(v32).cuda()).cpu().numpy(), Kv32) <= 1e-11
    assert err(P.jacobian_apply(torch.from_numpy(v32).cuda()).double().cpu().numpy(), Kv32) <= 2e-5
    P.close()


@pytest.fixture(scope="module")
def ragged_simplex():
    """The ragged grid with every eta_i in the admissible simplex (the
    penalty branch, which makes this small system hard for any variant count,
    is covered by the tangent tests above)."""
    st = inputs.config_random(6, 5, 4, seed=122, eta_lo=0.0, eta_hi=0.05, Lx=12.0, Ly=10.0, Lz=8.0, n_var=NV)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh, n_var=NV)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    return dict(st=st, K=fe.tangent(disc, st, mat, d), R=fe.residual(disc, st, mat, d))


@pytest.mark.parametrize("prec", [abi.PFM_F32, abi.PFM_F64])
def test_newton_correction_matches_direct_solve(binding, ragged_simplex, prec):
    st, K, R = ragged_simplex["st"], ragged_simplex["K"], ragged_simplex["R"]
    dU = fe.newton_correction(K, R)
    P = binding.problem_from_state(st)
    assert P.n_levels == 2
    P.linearize(prec)
    x, rep = P.fgmres_solve(-P.residual(), abi.default_opts(prec, lin_rtol=1e-10, max_lin_it=300))
    x = x.cpu().numpy()
    assert np.linalg.norm(K @ x.reshape(-1) + R.reshape(-1)) <= 1e-9 * np.linalg.norm(R)
    assert np.linalg.norm(x - dU) <= 1e-7 * np.linalg.norm(dU)
    P.close()


def test_indentation_newton_at_16_cubed(binding):
    """The indentation load on a 16^3 cube with twelve variants: a full
    Newton solve of the first load step converges, and the oracle's residual
    of the end state confirms it."""
    st = inputs.config_indentation(16, seed=7, step=1, n_var=NV)
    P = binding.problem_from_state(st)
    U = torch.from_numpy(st.U.copy()).cuda()
    rep = P.newton_solve(U, abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-8, lin_rtol=1e-8,
                                             max_lin_it=400))
    assert rep.res_final <= 1e-8 * rep.res0
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh, n_var=NV)
    Uh = U.cpu().numpy()
    R1 = fe.residual(disc, inputs.State(st.mesh, Uh, st.Un, st.mask, st.tau, st.material), mat)
    R0 = fe.residual(disc, st, mat)
    assert np.linalg.norm(R1) <= 1e-7 * np.linalg.norm(R0)
    assert abs(rep.res0 - np.linalg.norm(R0)) <= 1e-10 * np.linalg.norm(R0)
    P.close()


def test_batched_engine_with_twelve_variants(binding):
    """Three twelve-variant indentation problems of uneven size (a non-nested
    hierarchy among them) in one batch: the batched engine (one launch per
    phase over all problems) and the per-problem lockstep driver give the same
    Newton corrections to the solve tolerance, and each meets it against the
    FP64 operator of its own problem."""
    sts = [inputs.config_indentation(n, seed=300 + n, step=1, n_var=NV) for n in (5, 8, 9)]
    opts = abi.default_opts(abi.PFM_F32, max_newton=1, lin_rtol=1e-10, max_lin_it=600)
    out = []
    for mode in (0, 1):
        probs = [binding.problem_from_state(st) for st in sts]
        B = binding.Batch(probs)
        B.set_mode(mode)
        Us = [torch.from_numpy(st.U.copy()).cuda() for st in sts]
        reps = B.newton_solve(Us, opts, check=False)
        assert all(r.newton_its == 1 and r.lin_res_final <= 1e-10 for r in reps), \
            [(r.newton_its, r.lin_res_final) for r in reps]
        out.append([u.cpu().numpy() for u in Us])
        if mode == 0:
            for P, st, U1 in zip(probs, sts, Us):
                U0 = torch.from_numpy(st.U).cuda()
                P.set_state(U0, torch.from_numpy(st.Un).cuda())
                R = P.residual()
                P.linearize(abi.PFM_F64)
                y = P.jacobian_apply(U1 - U0)
                assert float(torch.linalg.norm(y + R) / torch.linalg.norm(R)) <= 1e-9
        B.close()
        for P in probs:
            P.close()
    for k, st in enumerate(sts):
        d0, d1 = out[0][k] - st.U, out[1][k] - st.U
        assert np.linalg.norm(d0 - d1) <= 1e-6 * np.linalg.norm(d1), k
