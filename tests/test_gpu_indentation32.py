"""The 32^3 indentation configuration as written (GPU tests): 32^3 trilinear
hexahedra (323,433 DOFs), a spherical cap on the top face pressed in over 10
backward-Euler load steps (Sec. 5.1 load ramp; cap depth 0.02 L k / 10 at
step k), each step a full Newton solve (Sec. 3.4, Eq. linAlgEq) in plain
FP64: FGMRES(30) to 1e-8 with the FP64 4-level geometric multigrid, Newton
to ||R|| <= 1e-8 ||R_0||.

Parity per step (paths of a nonconvex problem may branch, so each step is
judged by its own equations): the oracle's residual of the GPU's end state,
against the oracle's residual of that step's initial iterate (the previous
state with the new cap values), evaluated on all host cores. The same ramp
solved with the mixed-precision preconditioner reaches the same states."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle_pool import OraclePool  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

N = 32
STEPS = 10


@pytest.fixture(scope="module")
def pool():
    # spawned workers hold no CUDA context; started before this module's first GPU call
    with OraclePool() as p:
        yield p


@pytest.fixture(scope="module")
def ramp64(pool):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding, driver
    st = inputs.config_indentation(N, seed=2, step=0, n_steps=STEPS)
    P = binding.problem_from_state(st)
    assert P.n_levels == 4
    opts = abi.default_opts(abi.PFM_F64, max_newton=12, newton_rtol=1e-8, restart=30, lin_rtol=1e-8,
                            max_lin_it=400)
    steps = []

    def keep(k, mask, values, Un, U, rep):
        steps.append(dict(k=k, mask=mask, values=values, Un=Un.cpu().numpy(), U=U.cpu().numpy(),
                          newton_its=rep.newton_its, lin_its=rep.lin_its_total, res0=rep.res0,
                          res=rep.res_final, status=rep.status))

    driver.load_ramp(P, st, upto=STEPS, n_steps=STEPS, opts=opts, on_step=keep)
    P.close()
    return st, steps


def test_every_step_converges_in_fp64(ramp64):
    st, steps = ramp64
    assert [s["k"] for s in steps] == list(range(1, STEPS + 1))
    for s in steps:
        assert s["status"] == 0 and 1 <= s["newton_its"] <= 12, s
        assert s["res"] <= 1e-8 * s["res0"], s
        # the prescribed cap values hold exactly
        D = s["mask"].astype(bool)
        assert np.array_equal(s["U"][D], s["values"][D])
    # the cap goes deeper every step
    assert steps[-1]["values"][2].min() == pytest.approx(-0.02 * st.mesh.Lz, rel=1e-12)


def test_oracle_residual_of_every_step(ramp64, pool):
    st, steps = ramp64
    starts, ends = [], []
    for s in steps:
        D = s["mask"].astype(bool)
        U0 = s["Un"].copy()
        U0[D] = s["values"][D]
        starts.append(inputs.State(st.mesh, U0, s["Un"], s["mask"], st.tau, st.material))
        ends.append(inputs.State(st.mesh, s["U"], s["Un"], s["mask"], st.tau, st.material))
    R = pool.residuals(starts + ends)
    ratios = []
    for k, s in enumerate(steps):
        r0 = np.linalg.norm(R[k])
        r1 = np.linalg.norm(R[STEPS + k])
        ratios.append(r1 / r0)
        # the GPU's own initial residual equals the oracle's
        assert abs(s["res0"] - r0) <= 1e-10 * r0
    print("oracle ||R(U_k)|| / ||R(U_k^0)|| per step:", " ".join(f"{x:.2e}" for x in ratios))
    assert max(ratios) <= 1e-8, ratios


def test_mixed_precision_ramp_tracks_fp64(ramp64):
    """The FP32-preconditioned solve of the same ramp (FP64 FGMRES and Newton)
    gives the same states: both meet the same tolerances, so their states
    agree to far below the size of one load increment."""
    from paper_2011_08802_gb300 import binding, driver
    st, steps = ramp64
    P = binding.problem_from_state(st)
    opts = abi.default_opts(abi.PFM_F32, max_newton=12, newton_rtol=1e-8, restart=30, lin_rtol=1e-8,
                            max_lin_it=400)
    out = []
    driver.load_ramp(P, st, upto=STEPS, n_steps=STEPS, opts=opts,
                     on_step=lambda k, m, v, Un, U, rep: out.append(U.cpu().numpy()))
    P.close()
    for s, U32 in zip(steps, out):
        inc = np.linalg.norm(s["U"] - s["Un"])
        assert np.linalg.norm(U32 - s["U"]) <= 1e-6 * inc
