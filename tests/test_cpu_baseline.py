"""The timed CPU baseline of bench.py: the oracle in spawned single-thread processes (no GPU).

The pool is sized by cores and free memory, its workers start each round together, and a
worker that fails is reported at once rather than leaving the others waiting.
"""
import dataclasses
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_pool_size_is_bounded_by_cores_and_memory():
    assert bench.oracle_pool_size(16, 1e12) == 16                  # memory to spare
    assert bench.oracle_pool_size(16, 20e9, per_proc=3e9) == 3     # half of 20 GB holds 3
    assert bench.oracle_pool_size(16, 1e9) == 1                     # never fewer than one
    assert bench.oracle_pool_size(2, None) == 2
    assert bench.oracle_pool_size(64, None) == 4                    # memory unknown


def test_pool_rounds_time_every_worker():
    w = synth.get_workload("box64_n6l6")
    walls = bench.oracle_pool(w, 12, 2, reps=2)
    assert len(walls) == 2 and all(t > 0 for t in walls)


def test_failing_worker_is_reported():
    w = dataclasses.replace(synth.get_workload("box64_n6l6"), n_sparse=-1)   # no sparse set
    t0 = time.monotonic()
    with pytest.raises(RuntimeError, match="oracle worker"):
        bench.oracle_pool(w, 12, 2)
    assert time.monotonic() - t0 < 300
