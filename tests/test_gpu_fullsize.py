"""Parity at the benchmark size (GPU tests): the 128^3 nano-indentation state
(19,320,201 DOFs, 6 levels) in the launch configuration bench.py times,
checked on sampled outputs the oracle computes one by one: each sampled node
needs only its (at most eight) adjacent elements, each sampled element only
its own Gauss points."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

N = 128


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding
    st = inputs.config_indentation(N, seed=5, step=1)
    P = binding.problem_from_state(st)
    mat = qp.material_from(st.material, st.tau)
    rng = np.random.default_rng(123)
    m = st.mesh
    # sampled nodes: under the cap, at the cap rim, interior, near the clamped bottom, on a lateral face
    ijk = [(64, 64, 128), (64 + 38, 64, 128), (64, 64, 127), (10, 20, 1), (0, 50, 60), (127, 127, 64)]
    ijk += [tuple(int(x) for x in rng.integers(0, N + 1, 3)) for _ in range(6)]
    nodes = [i + (m.nx + 1) * (j + (m.ny + 1) * k) for i, j, k in ijk]
    yield dict(st=st, P=P, mat=mat, ijk=ijk, nodes=nodes)
    P.close()


def _adjacent(m, i, j, k):
    ids = []
    for c in range(max(k - 1, 0), min(k, m.nz - 1) + 1):
        for b in range(max(j - 1, 0), min(j, m.ny - 1) + 1):
            for a in range(max(i - 1, 0), min(i, m.nx - 1) + 1):
                ids.append(a + m.nx * (b + m.ny * c))
    return ids


def _rows(big, node_vals_fn):
    """Evaluate an oracle quantity at each sampled node from its adjacent elements."""
    st, out = big["st"], []
    for (i, j, k), n in zip(big["ijk"], big["nodes"]):
        disc = fe.Discretisation(st.mesh, elements=_adjacent(st.mesh, i, j, k))
        out.append(node_vals_fn(disc)[:, n])
    return np.array(out)


def test_residual_rows(big):
    st, P, mat = big["st"], big["P"], big["mat"]
    R = P.residual().cpu().numpy()
    Ro = _rows(big, lambda disc: fe.residual(disc, st, mat))
    Rg = R[:, big["nodes"]].T
    scale = np.abs(R).max()
    assert np.abs(Rg - Ro).max() <= 1e-11 * scale


def test_hessians_of_sampled_elements(big):
    st, P, mat = big["st"], big["P"], big["mat"]
    P.linearize(abi.PFM_F32)
    iu = np.triu_indices(15)
    for (i, j, k) in big["ijk"][:6]:
        e = min(i, N - 1) + N * (min(j, N - 1) + N * min(k, N - 1))
        Hg = P.get_hessians(e, 1)[0]
        d = fe.qp_derivatives(fe.Discretisation(st.mesh, elements=[e]), st, mat, order=2)
        Ho = d["H"][0][:, iu[0], iu[1]]
        assert np.abs(Hg - Ho).max() <= 1e-12 * np.abs(Ho).max()


@pytest.mark.parametrize("mode", ["pade11", "pade22", "pade33"])
def test_pade_hessians_under_the_cap(big, mode):
    """Pade modes at the benchmark state, where the top element layer under
    the cap is compressed by up to ~25 %: Hessians of elements along a radius
    of the cap, from the centre to past the rim, against the oracle."""
    from paper_2011_08802_gb300 import binding
    st = big["st"]
    mat = qp.material_from(st.material, st.tau, hencky=mode)
    P = binding.problem_from_state(st, params=abi.params_from_material(st.material, st.tau, hencky=mode))
    P.linearize(abi.PFM_F32)
    iu = np.triu_indices(15)
    for i in range(N // 2, N // 2 + 45, 11):
        e = i + N * (N // 2 + N * (N - 1))
        Hg = P.get_hessians(e, 1)[0]
        d = fe.qp_derivatives(fe.Discretisation(st.mesh, elements=[e]), st, mat, order=2)
        Ho = d["H"][0][:, iu[0], iu[1]]
        assert np.abs(Hg - Ho).max() <= 1e-12 * np.abs(Ho).max()
    P.close()


def test_tangent_rows_fp64_and_fp32(big):
    st, P, mat = big["st"], big["P"], big["mat"]
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(7).standard_normal(st.U.shape)
    y64 = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
    v32 = v.astype(np.float32)
    y32 = P.jacobian_apply(torch.from_numpy(v32).cuda()).cpu().numpy()
    ydf = P.jacobian_apply_mixed(torch.from_numpy(v32).cuda()).cpu().numpy()
    for (i, j, k), n in zip(big["ijk"], big["nodes"]):
        disc = fe.Discretisation(st.mesh, elements=_adjacent(st.mesh, i, j, k))
        d = fe.qp_derivatives(disc, st, mat, order=2)
        yo = fe.jvp(disc, st, v, d)[:, n]
        yo32 = fe.jvp(disc, st, v32.astype(np.float64), d)[:, n]
        # FP32 bound: a few hundred rounding errors of the absolute row sum |K| |v|
        Ke = fe.element_matrices(disc, d)
        vabs = np.abs(v32.astype(np.float64)).reshape(-1)
        yabs = np.zeros(v.size)
        np.add.at(yabs, disc.edofs[disc.elements].ravel(),
                  np.einsum("elm,em->el", np.abs(Ke), vabs[disc.edofs[disc.elements]]).ravel())
        yabs = yabs.reshape(v.shape)[:, n]
        free = ~st.mask[:, n].astype(bool)
        assert np.all(np.abs(y64[:, n] - yo)[free] <= 1e-11 * (yabs[free] + 1e-300))
        assert np.all(np.abs(ydf[:, n] - yo32)[free] <= 1e-11 * (yabs[free] + 1e-300))
        assert np.all(np.abs(y32[:, n] - yo32)[free] <= 2e-5 * (yabs[free] + 1e-300))


def test_newton_correction_rows(big):
    """The mixed-precision Newton correction of the benchmark: global true
    residual (FP64 operator) below 1e-8, and the oracle's residual rows
    K x + R at the sampled nodes below 1e-8 ||R||."""
    st, P, mat = big["st"], big["P"], big["mat"]
    P.set_state(torch.from_numpy(st.U).cuda(), torch.from_numpy(st.Un).cuda())
    R = P.residual()
    P.linearize(abi.PFM_F32)
    x, rep = P.fgmres_solve(-R, abi.default_opts(abi.PFM_F32, max_lin_it=400, lin_rtol=1e-8))
    y = P.jacobian_apply(x)
    Rn = float(torch.linalg.norm(R))
    assert float(torch.linalg.norm(y + R)) <= 1e-8 * Rn
    xh = x.cpu().numpy()
    for (i, j, k), n in zip(big["ijk"], big["nodes"]):
        disc = fe.Discretisation(st.mesh, elements=_adjacent(st.mesh, i, j, k))
        d = fe.qp_derivatives(disc, st, mat, order=2)
        row = fe.jvp(disc, st, xh, d)[:, n] + fe.residual(disc, st, mat, d)[:, n]
        assert np.abs(row).max() <= 1e-8 * Rn
