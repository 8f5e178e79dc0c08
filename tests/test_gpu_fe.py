"""Parity of the CUDA element kernels with the CPU oracle (GPU tests):
Gauss-point physics, residual and energy, stored Hessians, tangent
application in FP64 and FP32, transpose application, Dirichlet rows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe, qp  # noqa: E402
from paper_2011_08802_gb300 import abi, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL64 = 1e-11   # FP64 kernels vs FP64 oracle (max-abs error / max-abs value)
RTOL32 = 2e-5    # FP32 tangent application vs FP64 oracle, per field


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08802_gb300 import binding as b
    return b


@pytest.fixture(scope="module")
def ragged(binding):
    """7x5x3 hexes (105 elements: 27 warps of 4, the last with one element),
    eta_hat in [-0.04, 0.32] so the penalty branch is active."""
    st = inputs.config_random(7, 5, 3, seed=31, eta_lo=-0.04, eta_hi=0.32, Lx=14.0, Ly=10.0, Lz=6.0)
    mat = qp.material_from(st.material, st.tau)
    disc = fe.Discretisation(st.mesh)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    K = fe.tangent(disc, st, mat, d)
    P = binding.problem_from_state(st)
    return dict(st=st, mat=mat, disc=disc, d=d, K=K, P=P)


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_qp_physics_matches_oracle(binding):
    rng = np.random.default_rng(40)
    st = inputs.config_random(2, 2, 2, seed=1)
    mat = qp.material_from(st.material, st.tau)
    B = 96
    F = np.eye(3) + 0.05 * rng.standard_normal((B, 3, 3))
    eh = rng.uniform(-0.05, 0.4, (B, 6))
    ehn = eh + 0.02 * rng.standard_normal((B, 6))
    for k in range(8):  # exactly and nearly degenerate C^e (F = F^t)
        e = np.zeros(6); e[k % 6] = 0.3 * (k + 1) / 8
        F[k] = np.einsum("i,ijk->jk", np.concatenate([[1 - e.sum()], e]), mat.U)
        eh[k] = e
        if k >= 4:
            F[k] = F[k] @ (np.eye(3) + 1e-7 * rng.standard_normal((3, 3)))
    F[8] = np.diag([1.02, 1.02, 0.97]); eh[8] = 0
    W = qp.local_energy(F, eh, ehn, mat, order=2)
    P = binding.problem_from_state(st)
    Wg, gg, Hg = P.qp_eval(torch.from_numpy(F.reshape(B, 9)).cuda(), torch.from_numpy(eh).cuda(),
                           torch.from_numpy(ehn).cuda())
    iu = np.triu_indices(15)
    assert _relerr(Wg.cpu().numpy(), W.v) < 1e-13
    assert _relerr(gg.cpu().numpy(), W.g) < 1e-13
    assert _relerr(Hg.cpu().numpy(), W.H[:, iu[0], iu[1]]) < 1e-12


def test_residual_and_energy(ragged):
    st, mat, disc, P = ragged["st"], ragged["mat"], ragged["disc"], ragged["P"]
    R, E = P.residual(energy=True)
    Ro = fe.residual(disc, st, mat, ragged["d"])
    assert _relerr(R.cpu().numpy(), Ro) < RTOL64
    assert abs(E - fe.energy(disc, st, mat)) < 1e-12 * abs(E)
    assert np.all(R.cpu().numpy()[st.mask.astype(bool)] == 0.0)


def test_stored_hessians(ragged):
    P = ragged["P"]
    P.linearize(abi.PFM_F32)
    Hg = P.get_hessians(0, P.n_elems)
    iu = np.triu_indices(15)
    Ho = ragged["d"]["H"][:, :, iu[0], iu[1]]
    assert _relerr(Hg, Ho) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobian_apply_fp64(ragged, seed):
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(seed).standard_normal(st.U.shape)
    y = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
    yo = (K @ v.reshape(-1)).reshape(v.shape)
    assert _relerr(y, yo) < RTOL64
    D = st.mask.astype(bool)
    assert np.all(y[D] == v[D])


def test_jacobian_apply_fp32(ragged):
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(5).standard_normal(st.U.shape).astype(np.float32)
    y = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
    yo = (K @ v.astype(np.float64).reshape(-1)).reshape(v.shape)
    for f in range(9):
        assert np.abs(y[f] - yo[f]).max() <= RTOL32 * np.abs(yo[f]).max(), f


def test_jacobian_apply_mixed_double_float(ragged):
    """FP32 input, FP64 output in double-float arithmetic: FP64-class accuracy."""
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(8).standard_normal(st.U.shape).astype(np.float32)
    y = P.jacobian_apply_mixed(torch.from_numpy(v).cuda()).cpu().numpy()
    yo = (K @ v.astype(np.float64).reshape(-1)).reshape(v.shape)
    assert _relerr(y, yo) < 1e-11


def test_jacobian_transpose(ragged):
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.linearize(abi.PFM_F64)
    rng = np.random.default_rng(6)
    v, w = rng.standard_normal(st.U.shape), rng.standard_normal(st.U.shape)
    vt, wt = torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda()
    Jtw = P.jacobian_transpose_apply(wt).cpu().numpy()
    assert _relerr(Jtw, (K.T @ w.reshape(-1)).reshape(w.shape)) < RTOL64
    Jv = P.jacobian_apply(vt).cpu().numpy()
    lhs, rhs = (w * Jv).sum(), (Jtw * v).sum()
    assert abs(lhs - rhs) <= 1e-11 * np.abs(w * Jv).sum()


def test_fp32_apply_needs_fp32_linearisation(ragged, binding):
    P = ragged["P"]
    P.linearize(abi.PFM_F64)
    v = torch.zeros(P.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(binding.PfmError):
        P.jacobian_apply(v)


def test_host_buffer_apply(ragged):
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(7).standard_normal(st.U.shape)
    y = P.jacobian_apply_host(v)
    assert _relerr(y, (K @ v.reshape(-1)).reshape(v.shape)) < RTOL64


def test_double_float_linearisation(ragged):
    """The FP64-class linearisation in double-float arithmetic: Hessians and
    the FP64 tangent application against the oracle, at the resolution of
    the double-float format (48 significant bits)."""
    P, K, st = ragged["P"], ragged["K"], ragged["st"]
    P.set_linearize_arithmetic(True)
    try:
        P.linearize(abi.PFM_F32)
        Hg = P.get_hessians(0, P.n_elems)
        iu = np.triu_indices(15)
        assert _relerr(Hg, ragged["d"]["H"][:, :, iu[0], iu[1]]) < 1e-12
        v = np.random.default_rng(12).standard_normal(st.U.shape)
        y = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
        assert _relerr(y, (K @ v.reshape(-1)).reshape(v.shape)) < 1e-11
    finally:
        P.set_linearize_arithmetic(False)


def test_autotune_cache_is_json(tmp_path):
    """The launch-shape autotuner keeps its choices in PFM_AUTOTUNE_FILE as a
    JSON array (checked in a fresh process, so that the tuning runs)."""
    import json
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.json"
    code = ("import sys; sys.path.insert(0, '.'); import torch; "
            "from paper_2011_08802_gb300 import abi, binding, inputs; "
            "st = inputs.config_random(12, 12, 12, seed=1); P = binding.problem_from_state(st); "
            "P.linearize(abi.PFM_F32); P.jacobian_apply(torch.zeros(P.shape, dtype=torch.float32, device='cuda')); "
            "torch.cuda.synchronize()")
    env = dict(os.environ, PFM_AUTOTUNE_FILE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=root, timeout=600)
    entries = json.loads(path.read_text())
    # a shape is the register-fed kernel (stages 0, 128 or 256 threads) or the
    # staged one (1-3 shared-memory stages per warp, 32-128 threads)
    def valid(e):
        if e["stages"] == 0:
            return e["threads"] in (128, 256)
        return e["stages"] in (1, 2, 3) and e["threads"] in (32, 64, 128)
    assert any(e["kernel"] == "k_japply" and e["precision"] == "f32" and valid(e)
               and e["ctas_per_sm"] >= 1 and e["ms_per_application"] > 0 for e in entries), entries
    assert all(valid(e) for e in entries), entries


@pytest.mark.parametrize("dims", [(16, 8, 12), (7, 5, 11)])
def test_host_buffer_pipeline_matches_device_apply(binding, dims):
    """The host-buffer entry point streams the input in and the result out in
    z-slabs while it computes; it gives the device entry point's product (a
    7x5 layer has 35 elements, so element blocks straddle the slab borders)."""
    nx, ny, nz = dims
    st = inputs.config_random(nx, ny, nz, seed=4, Lx=2.0 * nx, Ly=2.0 * ny, Lz=2.0 * nz)
    P = binding.problem_from_state(st)
    P.linearize(abi.PFM_F32)
    rng = np.random.default_rng(9)
    for dt, tol in ((np.float64, 1e-13), (np.float32, 3e-6)):
        v = rng.standard_normal(st.U.shape).astype(dt)
        y_dev = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy()
        y_host = P.jacobian_apply_host(torch.from_numpy(v).pin_memory())
        y_host = y_host.numpy() if hasattr(y_host, "numpy") else np.asarray(y_host)
        assert np.abs(y_host - y_dev).max() <= tol * np.abs(y_dev).max()
    P.close()
