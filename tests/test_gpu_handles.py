"""Event handles of the C ABI (GPU): lst_run_event with host buffers read back by
handle, results kept across later runs, release and slot exhaustion."""
import ctypes as C

import numpy as np
import pytest

from synth import events as E
from synth.config import DEFAULT_CUTS
from tests.gpu_common import A_HALF, gpu_result, make_context, oracle_result
from tests.parity import compare

pytestmark = pytest.mark.gpu


def _tc_set(tc):
    return {(int(t), int(s), tuple(sorted(h[h >= 0].tolist()))) for t, s, h in zip(tc["type"], tc["seed"], tc["hits"])}


def _abi_run_event(ctx, ev):
    """lst_run_event on HOST buffers, then lst_get_track_candidates by the returned handle, all through ctypes."""
    from paper_2209_13711_gb300 import lst
    L = lst.library()
    cols = dict(x=np.ascontiguousarray(ev.x, np.float32), y=np.ascontiguousarray(ev.y, np.float32),
                z=np.ascontiguousarray(ev.z, np.float32), module=np.ascontiguousarray(ev.module, np.int32),
                side=np.ascontiguousarray(ev.side, np.uint8),
                seeds=np.ascontiguousarray(np.asarray(ev.seeds, np.float32).reshape(-1)))
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    hits = lst.LstHits(p(cols["x"]), p(cols["y"]), p(cols["z"]), p(cols["module"]), p(cols["side"]), len(ev.x))
    seeds = lst.LstSeeds(p(cols["seeds"]), len(cols["seeds"]) // 9)
    hid = C.c_int64(0)
    assert L.lst_run_event(ctx._h, C.byref(hits), C.byref(seeds), 0, None, C.byref(hid)) == 0
    assert (hid.value >> 32) != 0                      # a handle, never an event index
    n = C.c_int32(0)
    assert L.lst_get_track_candidates(ctx._h, hid.value, 0, C.byref(n), None, None, None, None) in (0, 1)
    k = n.value
    t, s = np.zeros(k, np.int32), np.zeros(k, np.int32)
    h, f = np.zeros((k, 10), np.int32), np.zeros((k, 3), np.float32)
    assert L.lst_get_track_candidates(ctx._h, hid.value, k, C.byref(n), p(t), p(s), p(h), p(f)) == 0
    return hid.value, dict(n=k, type=t, seed=s, hits=h, pt=f[:, 0], eta=f[:, 1], phi0=f[:, 2])


@pytest.mark.parametrize("kind,seed", [("tiny", 3), ("pu60", 4)])
def test_run_event_through_the_c_abi_matches_the_oracle(geom_barrel, maps_barrel, geom_full, maps_full, kind, seed):
    geom, maps = (geom_barrel, maps_barrel) if kind == "tiny" else (geom_full, maps_full)
    ev = E.tiny_event(seed, geom) if kind == "tiny" else E.pileup_event(60, seed, geom)
    ctx = make_context(geom, maps, max_events=1)
    hid, tc = _abi_run_event(ctx, ev)
    g = gpu_result(ctx, 0)
    assert _tc_set(tc) == _tc_set(g["tc"])           # the handle and the last-batch index name the same event
    g["tc"] = tc
    o = oracle_result(geom, maps, ev)
    s = compare(g, o, A_HALF, DEFAULT_CUTS)
    assert s["tc"][0] >= (8 if kind == "tiny" else 500)
    ctx.release([hid])
    ctx.close()


def test_handles_keep_results_across_later_runs(geom_full, maps_full):
    evs = [E.pileup_event(30, 40 + i, geom_full) for i in range(4)]
    alone = make_context(geom_full, maps_full, max_events=2)
    want = []
    for ev in evs:
        alone.run([ev])
        want.append((_tc_set(alone.track_candidates(0)), alone.stats(0)))
    alone.close()

    ctx = make_context(geom_full, maps_full, max_events=2)
    a = ctx.run(evs[:2], keep=True)
    b = ctx.run(evs[2:3], keep=True)
    ctx.run(evs[3:4])                                 # no handles: the last batch
    for hid, (tcs, st) in zip(a + b, want[:3]):
        assert _tc_set(ctx.track_candidates(hid)) == tcs
        assert ctx.stats(hid) == st
    assert _tc_set(ctx.track_candidates(0)) == want[3][0]
    from paper_2209_13711_gb300 import LstError
    with pytest.raises(LstError):
        ctx.objects("md", a[0])                       # intermediate objects belong to the last batch
    ctx.release(a[:1])
    with pytest.raises(LstError):
        ctx.track_candidates(a[0])                    # released
    with pytest.raises(LstError):
        ctx.release(a[:1])                            # released twice
    assert _tc_set(ctx.track_candidates(a[1])) == want[1][0]
    ctx.release(a[1:] + b)
    with pytest.raises(LstError):
        ctx.stats(b[0])
    ctx.close()


def test_result_slots_run_out_and_come_back(geom_full, maps_full):
    from paper_2209_13711_gb300 import LstError, lst
    ev = E.pileup_event(10, 50, geom_full)
    ctx = make_context(geom_full, maps_full, max_events=1)
    held = [ctx.run([ev], keep=True)[0] for _ in range(lst.LST_RESULT_SLOTS)]
    with pytest.raises(LstError, match="-6"):
        ctx.run([ev])                                 # every slot held: refused before anything is enqueued
    want = _tc_set(ctx.track_candidates(held[-1]))
    ctx.release(held[:1])
    ctx.run([ev])
    for hid in held[1:]:
        assert _tc_set(ctx.track_candidates(hid)) == want
    assert _tc_set(ctx.track_candidates(0)) == want
    ctx.release(held[1:])
    ctx.close()
