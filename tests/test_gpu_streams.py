"""Contexts on separate CUDA streams (GPU): events run at once give the same
objects and TCs as each event run alone."""
import pytest
import torch

from synth import events as E
from tests.gpu_common import all_tuples, make_context

pytestmark = pytest.mark.gpu


def test_concurrent_contexts_match_alone(geom_full, maps_full):
    evs = [E.pileup_event(60, 70 + i, geom_full) for i in range(3)]
    ctxs = [make_context(geom_full, maps_full) for _ in evs]
    try:
        alone = []
        for c, ev in zip(ctxs, evs):
            c.run([ev])
            alone.append(all_tuples(c, 0))
        sts = [torch.cuda.Stream() for _ in evs]
        torch.cuda.synchronize()
        for _ in range(2):
            for c, ev, s in zip(ctxs, evs, sts):
                c.run([ev], stream=s.cuda_stream)
            torch.cuda.synchronize()
            for c, want in zip(ctxs, alone):
                assert all_tuples(c, 0) == want
    finally:
        for c in ctxs:
            c.close()
