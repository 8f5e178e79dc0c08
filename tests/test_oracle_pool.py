"""The chunked oracle pool (test infrastructure, no GPU): the residual summed
over element chunks equals the oracle's one-process residual, and the rows of
K x + R from a subset of elements equal the assembled tangent's rows at nodes
whose adjacent elements are all in the subset."""
import numpy as np

from oracle import fe, qp
from oracle_pool import OraclePool
from paper_2011_08802_gb300 import inputs


def test_pool_matches_one_process():
    st = inputs.config_random(4, 3, 3, seed=91, eta_lo=-0.03, eta_hi=0.3, Lx=8.0, Ly=6.0, Lz=6.0)
    st2 = inputs.config_indentation(4, seed=92, step=3)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    R = fe.residual(disc, st, mat, d)
    K = fe.tangent(disc, st, mat, d)
    x = np.random.default_rng(5).standard_normal(st.U.shape)
    x[st.mask.astype(bool)] = 0.0
    full = (K @ x.reshape(-1)).reshape(x.shape) + R
    # nodes of the two lower element layers whose neighbours are all in layers 0..1
    m = st.mesh
    elems = [e for e in range(m.n_elems) if e // (m.nx * m.ny) < 2]
    nodes = [n for n in range(m.n_nodes) if n // ((m.nx + 1) * (m.ny + 1)) <= 1]
    with OraclePool(3) as pool:
        Rs = pool.residuals([st, st2])
        rows = pool.rows_Kx_plus_R(st, x, elems, nodes)
    np.testing.assert_allclose(Rs[0], R, rtol=0, atol=1e-12 * np.abs(R).max())
    R2 = fe.residual(fe.Discretisation(st2.mesh), st2, qp.material_from(st2.material, st2.tau))
    np.testing.assert_allclose(Rs[1], R2, rtol=0, atol=1e-12 * np.abs(R2).max())
    np.testing.assert_allclose(rows, full[:, nodes], rtol=0, atol=1e-11 * np.abs(full).max())
