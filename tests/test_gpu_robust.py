"""Invariances and malformed input on the device (GPU): hit order, invalid and
NaN hits, malformed geometry."""
import numpy as np
import pytest

from paper_2209_13711_gb300 import LstError
from synth import events as E
from tests.gpu_common import gpu_result, make_context
from tests.parity import chain_tuples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_full(geom_full, maps_full):
    return make_context(geom_full, maps_full, max_events=2)


def _subset(ev, idx):
    return E.Event(x=ev.x[idx], y=ev.y[idx], z=ev.z[idx], module=ev.module[idx], side=ev.side[idx],
                   pid=ev.pid[idx], seeds=ev.seeds, seed_pid=ev.seed_pid, tracks=ev.tracks)


def _levels(ctx, mapping):
    """Object levels MD..pT3 as hit tuples in the original hit numbering."""
    g = gpu_result(ctx, 0)
    for k in ("lo", "up"):
        g["md"][k] = mapping[np.asarray(g["md"][k])]
    return {k: set(v) for k, v in chain_tuples(g).items()}, g


def _tc_set(g, mapping):
    tc = g["tc"]
    out = set()
    for t, s, h in zip(tc["type"], tc["seed"], tc["hits"]):
        out.add((int(t), int(s), tuple(sorted(int(mapping[x]) for x in h if x >= 0))))
    return out


def test_hit_order_does_not_change_the_objects(ctx_full, geom_full):
    ev = E.pileup_event(60, 2, geom_full)
    n = len(ev.x)
    ctx_full.run([ev])
    ref, _ = _levels(ctx_full, np.arange(n))
    perm = np.random.default_rng(5).permutation(n)      # new hit k is old hit perm[k]
    ctx_full.run([_subset(ev, perm)])
    got, _ = _levels(ctx_full, perm)
    assert got == ref


def test_hit_order_does_not_change_the_track_candidates(geom_barrel, maps_barrel):
    ctx = make_context(geom_barrel, maps_barrel, max_events=1)
    for seed in range(4):
        ev = E.tiny_event(seed, geom_barrel)
        n = len(ev.x)
        ctx.run([ev])
        ref = _tc_set(gpu_result(ctx, 0), np.arange(n))
        perm = np.random.default_rng(seed).permutation(n)
        ctx.run([_subset(ev, perm)])
        assert _tc_set(gpu_result(ctx, 0), perm) == ref
    ctx.close()


def test_invalid_hits_are_skipped_and_counted(ctx_full, geom_full):
    ev = E.pileup_event(20, 3, geom_full)
    n = len(ev.x)
    ctx_full.run([ev])
    ref, _ = _levels(ctx_full, np.arange(n))
    bad_mod = np.array([-1, geom_full.n_mod, 5, 7, 2**30], np.int32)
    bad_side = np.array([0, 1, 2, 255, 0], np.uint8)
    k = len(bad_mod)
    x = np.concatenate([ev.x, np.full(k, 30.0, np.float32)])
    y = np.concatenate([ev.y, np.full(k, 1.0, np.float32)])
    z = np.concatenate([ev.z, np.full(k, 2.0, np.float32)])
    order = np.random.default_rng(1).permutation(n + k)   # interleave the bad hits
    ev2 = E.Event(x=x[order], y=y[order], z=z[order],
                  module=np.concatenate([ev.module, bad_mod])[order],
                  side=np.concatenate([ev.side, bad_side])[order],
                  pid=np.concatenate([ev.pid, np.full(k, -1, np.int32)])[order],
                  seeds=ev.seeds, seed_pid=ev.seed_pid, tracks=ev.tracks)
    ctx_full.run([ev2])
    assert ctx_full.counters()[16] == k
    mapping = np.where(order < n, order, -1)
    got, g = _levels(ctx_full, mapping)
    assert got == ref
    assert not np.any(np.asarray(g["md"]["lo"]) < 0) and not np.any(np.asarray(g["md"]["up"]) < 0)


def test_nan_hits_build_no_objects(ctx_full, geom_full):
    ev = E.pileup_event(20, 4, geom_full)
    n = len(ev.x)
    bad = np.random.default_rng(2).choice(n, 50, replace=False)
    x = ev.x.copy()
    x[bad] = np.nan
    ev2 = E.Event(x=x, y=ev.y, z=ev.z, module=ev.module, side=ev.side, pid=ev.pid, seeds=ev.seeds,
                  seed_pid=ev.seed_pid, tracks=ev.tracks)
    ctx_full.run([ev2])
    g = gpu_result(ctx_full, 0)
    used = set(np.asarray(g["md"]["lo"]).tolist()) | set(np.asarray(g["md"]["up"]).tolist())
    assert not used & set(bad.tolist())
    assert g["tc"]["n"] > 0


def test_malformed_geometry_is_rejected(geom_full, maps_full):
    import paper_2209_13711_gb300 as P
    from synth.config import DEFAULT_CUTS
    co, ct, so, st = [np.array(a, np.int32) for a in maps_full]
    cases = []
    bad = ct.copy(); bad[3] = geom_full.n_mod                       # connection to a module that does not exist
    cases.append((co, bad, so, st))
    bad = st.copy(); bad[0] = -1                                    # superbin target out of range
    cases.append((co, ct, so, bad))
    i = int(np.flatnonzero(np.diff(so) > 0)[0])
    bad = so.copy(); bad[i + 1] = so[i] - 1                          # superbin offsets not monotone
    cases.append((co, ct, bad, st))
    cases.append((co, ct, so[:-2], st))                             # wrong number of superbins
    for maps in cases:
        with pytest.raises(LstError):
            P.Context(geom_full.module_table(), maps, cfg=DEFAULT_CUTS, capacity=P.default_capacity(1))
