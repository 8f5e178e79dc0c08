"""One V-cycle of the CUDA path (pfm_vcycle in FP64: Chebyshev point-block
Jacobi smoothing, restriction, prolongation, the dense coarse inverse, on
re-discretised levels) against the oracle's V-cycle (oracle/multigrid.py) on
the same state, right-hand side and smoother eigenvalue estimates (GPU
tests): nested two- and three-level hierarchies and non-nested ones (odd
grid dimensions: coarse states by Q1 interpolation, coarse Dirichlet DOFs by
the nearest fine node), with the penalty branch active. The smoother's lambda_max is an input of the method, read from the
library (pfm_get_level) and handed to the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp, transfer  # noqa: E402
from oracle import multigrid as mg  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


def _oracle_levels(st, n_levels, lams):
    mat = qp.material_from(st.material, st.tau)
    m = st.mesh
    dims = [(m.nx, m.ny, m.nz)]
    for _ in range(n_levels - 1):
        dims.append(tuple(-(-n // 2) for n in dims[-1]))
    levels, U, Un, mask = [], st.U, st.Un, st.mask
    for l, d in enumerate(dims):
        if l > 0:
            U = transfer.inject(dims[l - 1], d, U)
            Un = transfer.inject(dims[l - 1], d, Un)
            mask = mg.coarse_mask(dims[l - 1], d, mask)
        mesh = inputs.Mesh(d[0], d[1], d[2], m.Lx, m.Ly, m.Lz)
        s = inputs.State(mesh, U, Un, mask, st.tau, st.material)
        K = fe.tangent(fe.Discretisation(mesh), s, mat)
        L = dict(dims=d, K=K, mask=mask)
        if l < n_levels - 1:
            L["Dinv"] = mg.nodal_block_inverses(K, mesh.n_nodes, U.shape[0])
            L["lam"] = lams[l]
        levels.append(L)
    return levels


@pytest.mark.parametrize("dims, n_levels", [((6, 4, 4), 2), ((8, 4, 4), 3), ((9, 7, 6), 2), ((10, 6, 5), 3)])
def test_vcycle_matches_oracle(binding, dims, n_levels):
    nx, ny, nz = dims
    st = inputs.config_random(nx, ny, nz, seed=40 + nx, eta_lo=-0.02, eta_hi=0.3,
                              Lx=2.0 * nx, Ly=2.0 * ny, Lz=2.0 * nz)
    P = binding.problem_from_state(st, n_levels=n_levels)
    assert P.n_levels == n_levels
    P.linearize(abi.PFM_F64)
    lams = [P.get_level(l)[3] for l in range(n_levels - 1)]
    r = np.random.default_rng(nx).standard_normal(st.U.shape)
    r[st.mask.astype(bool)] = 0.0
    opts = abi.default_opts(abi.PFM_F64)
    z = P.vcycle(torch.from_numpy(r).cuda(), opts=opts).cpu().numpy()
    P.close()
    levels = _oracle_levels(st, n_levels, lams)
    zo = mg.vcycle(levels, r, opts.nu_pre, opts.nu_post, opts.nu_growth, opts.cheb_lo, opts.cheb_hi)
    rel = np.linalg.norm(z - zo) / np.linalg.norm(zo)
    print(f"{dims}, {n_levels} levels: ||z - z_oracle|| / ||z_oracle|| = {rel:.2e}")
    assert rel <= 1e-10
