"""Serving loop on the device: every request's results equal the event run alone (GPU)."""
import math

import numpy as np
import pytest

from synth import events as E
from tests.gpu_common import make_context

pytestmark = pytest.mark.gpu


def _tc_rows(tc):
    """TCs as a canonical sorted list of (type, seed, hits, pt, eta, phi0)."""
    rows = []
    for i in range(tc["n"]):
        h = tc["hits"][i]
        rows.append((int(tc["type"][i]), int(tc["seed"][i]), tuple(int(v) for v in h),
                     float(tc["pt"][i]), float(tc["eta"][i]), float(tc["phi0"][i])))
    return sorted(rows)


@pytest.fixture(scope="module")
def pool_events(geom_full):
    return [E.pileup_event(pu, 900 + i, geom_full) for i, pu in enumerate((150, 30, 60, 190, 5, 140))]


@pytest.fixture(scope="module")
def alone(geom_full, maps_full, pool_events):
    ctx = make_context(geom_full, maps_full, max_events=1)
    out = []
    for ev in pool_events:
        ctx.run([ev])
        out.append(_tc_rows(ctx.track_candidates(0)))
    ctx.close()
    return out


@pytest.mark.parametrize("rate", [math.inf, 1500.0])
def test_serving_mix_equals_alone(geom_full, maps_full, pool_events, alone, rate):
    from paper_2209_13711_gb300.serve import EventPool, make_requests, serve, summarize
    from synth.config import DEFAULT_CUTS
    pool = EventPool(pool_events)
    reqs = make_requests((pool.n_hits, pool.n_seeds), rate, 40, seed=7)
    out, sch = serve(geom_full.module_table(), maps_full, pool, reqs, cfg=DEFAULT_CUTS, max_slots=2, max_batch=4)
    s = summarize(out)
    assert s["served"] == 40 and s["rejected"] == 0
    if rate == math.inf:
        assert len(sch.slots) == 2 and max(b[1] for b in sch.batches) == 4
    for r in out:
        assert r.error is None
        assert _tc_rows(r.result) == alone[r.event], (r.rid, r.event, r.batch_size)
    for sl in sch.slots:
        sl.close()


def test_slot_reuse_and_budget(geom_full, maps_full, pool_events):
    """A budget below two slots' buffers keeps the loop on one slot; results still complete."""
    from paper_2209_13711_gb300.serve import DeviceSlot, EventPool, make_requests, serve, summarize
    from synth.config import DEFAULT_CUTS
    pool = EventPool(pool_events)
    first = DeviceSlot(geom_full.module_table(), maps_full, pool, cfg=DEFAULT_CUTS, max_events=2)
    reqs = make_requests((pool.n_hits, pool.n_seeds), math.inf, 10, seed=3)
    out, sch = serve(geom_full.module_table(), maps_full, pool, reqs, cfg=DEFAULT_CUTS,
                     budget_bytes=first.device_bytes + 1, max_slots=3, max_batch=2, slots=[first])
    assert len(sch.slots) == 1 and sch.slots[0] is first
    assert summarize(out)["served"] == 10
    assert all(r.batch_size <= 2 for r in out)
    first.close()


def _event_dict(ev, cuda=False):
    import torch
    d = dict(x=ev.x, y=ev.y, z=ev.z, module=ev.module, side=ev.side, seeds=np.ascontiguousarray(ev.seeds))
    d = {k: np.ascontiguousarray(v) for k, v in d.items()}
    if cuda:
        d = {k: torch.from_numpy(v).cuda() for k, v in d.items()}
    return d


def test_run_events_and_packed_readback(geom_full, maps_full, pool_events, alone):
    from paper_2209_13711_gb300.lst import tc_dict
    ctx = make_context(geom_full, maps_full, max_events=8)
    evs = [pool_events[i] for i in (1, 4, 2, 1)]
    idx = [1, 4, 2, 1]
    ctx.run(evs)
    off, rec = ctx.batch_track_candidates()
    assert len(off) == 5 and off[0] == 0 and off[-1] == len(rec)
    for j, e in enumerate(idx):
        assert _tc_rows(ctx.track_candidates(j)) == alone[e]
        assert _tc_rows(tc_dict(rec[off[j]:off[j + 1]])) == alone[e]
    for cuda in (False, True):
        ctx.run_events([_event_dict(ev, cuda) for ev in evs])
        off2, rec2 = ctx.batch_track_candidates()
        assert np.array_equal(off2, off)
        for j, e in enumerate(idx):
            assert _tc_rows(tc_dict(rec2[off2[j]:off2[j + 1]])) == alone[e]
    # a capacity below the total: the first records and a truncation warning
    from paper_2209_13711_gb300.lst import TC_DTYPE
    small = np.empty(10, TC_DTYPE)
    off3, rec3 = ctx.batch_track_candidates(out=small)
    assert len(rec3) == 10 and off3[-1] == off[-1]
    ctx.close()
