"""The all-core oracle timing of the benchmark's CPU baseline (CPU): spawned
workers, one event each, barrier-synchronised clock, errors raised."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_parallel_oracle_times_every_worker():
    wall = bench._oracle_parallel_seconds([0, 1, 2], kind="tiny")
    assert 0.0 < wall < 60.0


def test_parallel_oracle_worker_error_raises():
    with pytest.raises(RuntimeError, match="oracle worker failed"):
        bench._oracle_parallel_seconds([0, 1], kind="no-such-event")
