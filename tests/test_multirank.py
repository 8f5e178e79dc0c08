"""Multi-process (world size 2) host logic on CPU with the gloo backend: the
bench's cross-rank reduction and the reference arm under torchrun (rank 0
prints one JSON line, the other rank exits 0 without work)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: step 100+10r ms, 4 applications of 2+r ms each on (1000+r) DOFs
    out = bench.reduce_over_ranks(100.0 + 10 * rank, 4 * (2.0 + rank), 4, 1000 + rank, dist, "cpu")
    q.put((rank, out))
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29611
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms_step, ms_apply, gdofs = res[0]
    assert res[1] == res[0]
    assert ms_step == 110.0 and ms_apply == 3.0
    # all DOF-applications over the slowest rank's application time
    assert abs(gdofs - (1000 * 4 + 1001 * 4) / (12.0 * 1e-3) / 1e9) < 1e-15


@pytest.mark.slow
def test_reference_arm_under_torchrun():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29612", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--edge", "16", "--sample", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["n_gpus"] == 2
