"""Every launch shape of the tangent application, staged (k_japply_tma: bulk
copies of the Hessian store into shared memory) and register-fed, on ragged
grids (GPU tests). The shape of each size class is forced through the
autotuner's cache file (PFM_AUTOTUNE_FILE) in a fresh process, one grid per
size class, and the FP32-arithmetic application from the FP32 store and from
the binary16 copy is compared with the FP64 application of the same state
(k_japply<double>, checked against the oracle's assembled tangent by
test_gpu_fe.py): the FP32 store within FP32 rounding, the binary16 copy
within its 11-bit rounding."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (grid, forced shape (threads, resident CTAs per SM, stages; 0 stages = register-fed))
CASES = [
    ((7, 6, 5), (128, 2, 2)),     # 53 element blocks: size class 5
    ((9, 7, 5), (128, 1, 3)),     # 79: class 6
    ((11, 9, 7), (64, 3, 2)),     # 174: class 7
    ((13, 11, 9), (32, 7, 2)),    # 322: class 8
    ((17, 13, 11), (128, 4, 1)),  # 608: class 9
    ((21, 17, 13), (128, 4, 0)),  # 1161: class 10
    ((25, 21, 17), (128, 2, 1)),  # 2232: class 11
]

SCRIPT = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2011_08802_gb300 import abi, binding, inputs
store, cases = sys.argv[2], json.loads(sys.argv[3])
out = []
for (nx, ny, nz), _ in cases:
    st = inputs.config_random(nx, ny, nz, seed=nx + ny + nz, eta_lo=-0.03, eta_hi=0.3,
                              Lx=2.0 * nx, Ly=2.0 * ny, Lz=2.0 * nz)
    P = binding.problem_from_state(st)
    if store == "f16":
        P.set_preconditioner_store(True)
    P.linearize(abi.PFM_F32)
    v = np.random.default_rng(nx).standard_normal(st.U.shape).astype(np.float32)
    y64 = P.jacobian_apply(torch.from_numpy(v.astype(np.float64)).cuda()).cpu().numpy()
    y32 = P.jacobian_apply(torch.from_numpy(v).cuda()).cpu().numpy().astype(np.float64)
    err = [float(np.abs(y32[f] - y64[f]).max() / np.abs(y64[f]).max()) for f in range(y64.shape[0])]
    out.append({"grid": [nx, ny, nz], "err": err, "finite": bool(np.isfinite(y32).all())})
    P.close()
print(json.dumps(out))
'''


def _size_class(grid):
    b = (grid[0] * grid[1] * grid[2] + 3) // 4
    c = 0
    while b > 1:
        b >>= 1
        c += 1
    return c


@pytest.mark.parametrize("store, tol", [("f32", 2e-5), ("f16", 2e-3)])
def test_forced_launch_shapes(tmp_path, store, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path / "autotune.json"
    lines = []
    for grid, (threads, per_sm, stages) in CASES:
        lines.append('{"kernel": "k_japply", "precision": "%s", "size_class": %d, "threads": %d, '
                     '"ctas_per_sm": %d, "stages": %d, "ms_per_application": 0.0}'
                     % (store, _size_class(grid), threads, per_sm, stages))
    cache.write_text("[\n " + ",\n ".join(lines) + "\n]\n")
    env = dict(os.environ, PFM_AUTOTUNE_FILE=str(cache))
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, store, json.dumps(CASES)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for case in res:
        assert case["finite"], case
        assert max(case["err"]) < tol, case
    # the forced shapes were read: the cache written back after tuning the
    # coarse levels' size classes still holds them
    kept = cache.read_text()
    for grid, (threads, per_sm, stages) in CASES:
        assert ('"size_class": %d, "threads": %d, "ctas_per_sm": %d, "stages": %d'
                % (_size_class(grid), threads, per_sm, stages)) in kept
