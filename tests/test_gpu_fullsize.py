"""Parity at the benchmark size (GPU tests): the 128^3 nano-indentation state
(19,320,201 DOFs, 6 levels) in the launch configuration bench.py times,
checked on sampled outputs the oracle computes one by one: each sampled node
needs only its (at most eight) adjacent elements, each sampled element only
its own Gauss points. The Newton correction is also checked by the oracle's
rows of K x + R over the whole cap footprint of the top element layer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from oracle_pool import OraclePool  # noqa: E402
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


def _top_layer_box(st, x, i0, i1):
    """The top element layer restricted to elements i, j in [i0, i1) as a
    state of its own (node planes nz-1 and nz), with x restricted alike."""
    m = st.mesh
    ii, jj, kk = np.meshgrid(np.arange(i0, i1 + 1), np.arange(i0, i1 + 1), np.arange(m.nz - 1, m.nz + 1),
                             indexing="ij")
    nodes = (ii + (m.nx + 1) * (jj + (m.ny + 1) * kk)).transpose(2, 1, 0).reshape(-1)
    hx, hy, hz = m.h
    e = i1 - i0
    sub = inputs.Mesh(e, e, 1, e * hx, e * hy, hz)
    box = inputs.State(sub, st.U[:, nodes].copy(), st.Un[:, nodes].copy(), st.mask[:, nodes].copy(), st.tau,
                       st.material)
    return box, x[:, nodes].copy()


def test_newton_correction_rows(big):
    """The mixed-precision Newton correction of the benchmark: global true
    residual (FP64 operator) below 1e-8, and the oracle's residual rows
    K x + R below 1e-8 ||R|| at the sampled nodes and at every top-face node
    over the cap footprint (the cap of radius 0.3 L = 38.4 elements: a box of
    80 x 80 top-layer elements around it, rows of its 79 x 79 inner top-face
    nodes, whose adjacent elements all lie in the box)."""
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
    i0, i1 = N // 2 - 40, N // 2 + 40
    box, xb = _top_layer_box(st, xh, i0, i1)
    e = i1 - i0
    inner = [a + (e + 1) * (b + (e + 1) * 1) for b in range(1, e) for a in range(1, e)]
    with OraclePool() as pool:
        rows = pool.rows_Kx_plus_R(box, xb, np.arange(box.mesh.n_elems), inner)
    worst = float(np.abs(rows).max()) / Rn
    print(f"cap footprint: {len(inner)} top-face nodes, max |K x + R| / ||R|| = {worst:.3e}")
    assert worst <= 1e-8
