"""Point-block Jacobi inverses (GPU tests): the smoother's stored inverse of
every node's 9x9 diagonal block of the finest-level tangent (Sec. 3.4,
point-block Jacobi with the nodal blocks inverted by Gauss-Jordan with
partial pivoting) against the inverse of the same block of the oracle's
assembled tangent, with Dirichlet rows and columns as identity; FP64 and
FP32 preconditioners, six and twelve variants."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _oracle_block_inverses(st, n_var):
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh, n_var=n_var)
    K = fe.tangent(disc, st, mat).tocsr()
    nn, nf = st.mesh.n_nodes, 3 + n_var
    out = np.empty((nn, nf, nf))
    for n in range(nn):
        idx = np.arange(nf) * nn + n
        out[n] = np.linalg.inv(K[idx][:, idx].toarray())
    return out


@pytest.mark.parametrize("n_var", [6, 12])
@pytest.mark.parametrize("prec, unit", [(abi.PFM_F64, 2.0 ** -53), (abi.PFM_F32, 2.0 ** -24)])
def test_block_inverses_match_oracle(binding, n_var, prec, unit):
    """Per block, the relative error of the inverse is bounded by a modest
    multiple of the unit roundoff of the preconditioner's precision times the
    block's condition number (entries rounded to that precision, summed over
    the element contributions, then Gauss-Jordan with partial pivoting)."""
    st = inputs.config_random(7, 5, 4, seed=131, eta_lo=-0.02, eta_hi=0.3 if n_var == 6 else 0.07, Lx=14.0,
                              Ly=10.0, Lz=8.0, n_var=n_var)
    inv_o = _oracle_block_inverses(st, n_var)
    kappa = np.linalg.cond(np.linalg.inv(inv_o))
    P = binding.problem_from_state(st)
    assert P.n_levels >= 2
    P.linearize(prec)
    inv_g = P.get_block_inverses(0, 0, st.mesh.n_nodes)
    err = np.abs(inv_g - inv_o).reshape(len(inv_o), -1).max(1) / np.abs(inv_o).reshape(len(inv_o), -1).max(1)
    bound = 200.0 * unit * kappa
    print(f"N = {n_var}, prec {prec}: worst error / bound {np.max(err / bound):.3f}, "
          f"kappa {kappa.min():.1f}..{kappa.max():.1f}")
    assert np.all(err <= bound), (err.max(), int(np.argmax(err / bound)))
    # a node range in the middle
    n0 = st.mesh.n_nodes // 3
    np.testing.assert_array_equal(P.get_block_inverses(0, n0, 5), inv_g[n0:n0 + 5])
    with pytest.raises(binding.PfmError):
        P.get_block_inverses(P.n_levels - 1, 0, 1)  # the coarsest level is solved directly
    P.close()
