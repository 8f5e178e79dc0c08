"""Adaptive loading-unloading history on the GPU (GPU tests): every accepted
step is a converged Newton solve whose end state the oracle's residual
confirms, the history ends unloaded, and the diagnostics are recorded."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def test_loading_unloading_history(binding):
    from paper_2011_08802_gb300 import driver
    n = 12
    st = inputs.config_indentation(n, seed=3, step=0)
    P = binding.problem_from_state(st)
    depth_max = 0.03 * st.mesh.Lz
    pairs = []
    U, recs = driver.indentation_history(P, st, depth_max=depth_max, speed=1.0, tau0=0.2,
                                         on_accept=lambda r, Un, U: pairs.append((r, Un.cpu().numpy(),
                                                                                  U.cpu().numpy())))
    acc = [r for r in recs if r.accepted]
    assert acc[-1].t == pytest.approx(2 * depth_max) and acc[-1].depth == pytest.approx(0.0, abs=1e-12)
    assert max(r.depth for r in acc) == pytest.approx(depth_max)
    assert all(r.newton_its <= 12 for r in acc)
    assert all(np.isfinite(r.max_Iv) and np.isfinite(r.mean_Id) for r in acc)
    assert len(pairs) == len(acc)
    # the step at the deepest load and the last step solve their equations by the oracle's residual
    disc = fe.Discretisation(st.mesh)
    for rec, Un, Uk in (max(pairs, key=lambda p: p[0].depth), pairs[-1]):
        mask, values = inputs.indentation_dirichlet_depth(st.mesh, rec.depth)
        mat = qp.material_from(st.material, rec.tau)
        R = fe.residual(disc, inputs.State(st.mesh, Uk, Un, mask, rec.tau, st.material), mat)
        U0 = Un.copy()
        U0[mask.astype(bool)] = values[mask.astype(bool)]
        R0 = fe.residual(disc, inputs.State(st.mesh, U0, Un, mask, rec.tau, st.material), mat)
        assert np.all(Uk[mask.astype(bool)] == values[mask.astype(bool)])
        assert np.linalg.norm(R) <= 1e-7 * np.linalg.norm(R0)
    np.testing.assert_array_equal(U.cpu().numpy(), pairs[-1][2])
    P.close()


def test_contact_loading_unloading(binding):
    """The same history with a rigid spherical indenter and penalty contact:
    the load grows during loading, the deepest step solves its equations by
    the oracle's residual (volume + contact), and the load there equals the
    oracle's."""
    from oracle import contact as C
    from paper_2011_08802_gb300 import driver
    n = 12
    st = inputs.config_indentation(n, seed=4, step=0)
    st.mask[:] = inputs.face_mask(st.mesh, bottom=True, top=False)
    L = st.mesh.Lx
    radius, eps = 0.57 * L, 100.0
    depth_max = 0.03 * L
    P = binding.problem_from_state(st)
    pairs = []
    U, recs = driver.indentation_history(P, st, depth_max=depth_max, speed=1.0, tau0=0.2,
                                         contact=(radius, eps),
                                         on_accept=lambda r, Un, U: pairs.append((r, Un.cpu().numpy(),
                                                                                  U.cpu().numpy())))
    acc = [r for r in recs if r.accepted]
    assert acc[-1].depth == pytest.approx(0.0, abs=1e-12)
    loading = [r for r in acc if r.t <= depth_max + 1e-12]
    assert all(b.load > a.load for a, b in zip(loading, loading[1:]))
    rec, Un, Uk = max(pairs, key=lambda p: p[0].depth)
    assert rec.depth == pytest.approx(depth_max)
    sph = C.indenter(st.mesh, rec.depth, radius, eps)
    mask = inputs.face_mask(st.mesh, bottom=True, top=False)
    mat = qp.material_from(st.material, rec.tau)
    disc = fe.Discretisation(st.mesh)
    s_k = inputs.State(st.mesh, Uk, Un, mask, rec.tau, st.material)
    Ec, Rc, Kc, load = C.contact(st.mesh, Uk, sph)
    R = fe.residual(disc, s_k, mat) + Rc * (~mask.astype(bool))
    s_0 = inputs.State(st.mesh, Un, Un, mask, rec.tau, st.material)
    R0 = fe.residual(disc, s_0, mat) + C.contact(st.mesh, Un, sph)[1] * (~mask.astype(bool))
    assert np.linalg.norm(R) <= 1e-7 * np.linalg.norm(R0)
    assert abs(rec.load - load) <= 1e-9 * load
    P.close()
