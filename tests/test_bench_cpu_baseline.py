"""The benchmark's CPU baseline legs (no GPU): the oracle's tangent
application timed on one core and on every host core at once (spawned
processes, a common window on the shared monotonic clock), and the
all-core leg failing fast, not hanging, when a worker cannot start."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_single_core_sample():
    value, desc, per = bench.oracle_jvp_sample(8, 3, 0.0, steps=3)
    assert value > 0.0 and per > 0.0
    assert "3^3-element block" in desc and "576 DOFs" in desc


def test_residual_sample():
    value, per = bench.oracle_residual_sample(8, 3, 0.1)
    assert value > 0.0 and per > 0.0


def test_all_cores_sample():
    value, desc, procs = bench.oracle_jvp_all_cores(8, 3, 1.0)
    assert procs == len(os.sched_getaffinity(0))
    assert value > 0.0
    assert f"by {procs} concurrent processes" in desc


def test_all_cores_fixed_steps():
    """The reference arm's form: W untimed and K timed applications per process."""
    value, desc, procs = bench.oracle_jvp_all_cores(8, 3, steps=4, warmup=1)
    assert value > 0.0
    assert f"{4 * procs} applications by {procs} concurrent processes" in desc


def test_workload_config_levels():
    from paper_2011_08802_gb300.binding import levels_to

    for n in (8, 9, 16, 24, 32, 100, 128):
        cfg = bench.workload_config(n, 1)
        assert f"{levels_to(n)}-level geometric MG" in cfg["workload"]
        assert f"{9 * (n + 1) ** 3} DOFs per GPU" in cfg["workload"]


def test_all_cores_fails_fast(monkeypatch):
    # the sample is built in the parent: a state the workers cannot use makes
    # every worker fail before the barrier, which they then break
    monkeypatch.setattr(bench, "oracle_sample_state", lambda n, e: (None, 1))
    t0 = time.monotonic()
    with pytest.raises(Exception):
        bench.oracle_jvp_all_cores(8, 3, 1.0)
    assert time.monotonic() - t0 < 60.0
