"""The oracle still reproduces its stored snapshot on the tiny workload."""
import json
import os

from tests.golden.make_golden import snapshot

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_snapshot():
    with open(os.path.join(HERE, "golden", "tiny_oracle.json")) as f:
        gold = json.load(f)
    for s, want in gold["seeds"].items():
        got = snapshot(int(s))
        assert got["counts"] == want["counts"]
        assert got["tc"] == want["tc"]
