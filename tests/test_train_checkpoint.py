"""Checkpoint files of the network's training (CPU): every part of the state
round-trips, and the per-epoch shuffles do not depend on where a run starts."""
import numpy as np

from paper_2209_13711_gb300 import train as T


class FakeMlp:
    def __init__(self, st=None):
        self.st = st

    def state(self):
        return self.st

    def set_state(self, st):
        self.st = st


def test_checkpoint_round_trips_the_whole_state(tmp_path):
    rng = np.random.default_rng(0)
    st = dict(params=rng.normal(size=9409).astype(np.float32), m=rng.normal(size=9409).astype(np.float32),
              v=rng.random(9409).astype(np.float32), step=1234)
    path = str(tmp_path / "ck.npz")
    T.save_checkpoint(path, FakeMlp(st), 3, [0.5, 0.4, 0.3])
    got = FakeMlp()
    epoch, hist = T.load_checkpoint(path, got)
    assert epoch == 3 and hist == [0.5, 0.4, 0.3]
    assert got.st["step"] == 1234
    for k in ("params", "m", "v"):
        assert got.st[k].dtype == np.float32 and np.array_equal(got.st[k], st[k])


def test_epoch_shuffles_are_independent_of_the_start_epoch():
    a = [np.random.default_rng([5, ep]).permutation(100) for ep in range(3)]
    b = np.random.default_rng([5, 2]).permutation(100)
    assert np.array_equal(a[2], b) and not np.array_equal(a[1], a[2])
