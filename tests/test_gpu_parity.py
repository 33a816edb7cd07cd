"""Device chain vs FP64 oracle, element by element, through the C ABI (GPU)."""
import numpy as np
import pytest

from synth import events as E
from synth.config import DEFAULT_CUTS
from tests.gpu_common import A_HALF, all_tuples as _all_tuples, gpu_result, make_context, oracle_result
from tests.parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_barrel(geom_barrel, maps_barrel):
    return make_context(geom_barrel, maps_barrel, max_events=8)


@pytest.fixture(scope="module")
def ctx_full(geom_full, maps_full):
    return make_context(geom_full, maps_full, max_events=4)


def _no_drops(res):
    assert all(v == 0 for v in res["stats"]["dropped"].values()), res["stats"]


@pytest.mark.parametrize("seed", range(8))
def test_tiny_event_parity(ctx_barrel, geom_barrel, maps_barrel, seed):
    ev = E.tiny_event(seed, geom_barrel)
    ctx_barrel.run([ev])
    g = gpu_result(ctx_barrel)
    _no_drops(g)
    o = oracle_result(geom_barrel, maps_barrel, ev)
    s = compare(g, o, A_HALF, DEFAULT_CUTS)
    assert s["tc"][0] >= 8


@pytest.mark.parametrize("pu,seed", [(25, 1), (60, 2)])
def test_pileup_event_parity(ctx_full, geom_full, maps_full, pu, seed):
    ev = E.pileup_event(pu, seed, geom_full)
    ctx_full.run([ev])
    g = gpu_result(ctx_full)
    _no_drops(g)
    o = oracle_result(geom_full, maps_full, ev)
    compare(g, o, A_HALF, DEFAULT_CUTS)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pu200_event_parity(ctx_full, geom_full, maps_full, seed):
    """Full-size PU200 events (the benchmark's workload), every object level."""
    ev = E.pu200_event(seed, geom_full)
    ctx_full.run([ev])
    g = gpu_result(ctx_full)
    _no_drops(g)
    o = oracle_result(geom_full, maps_full, ev)
    s = compare(g, o, A_HALF, DEFAULT_CUTS)
    assert s["t5"][0] > 10000 and s["tc"][0] > 2000


def test_t5_stage_overflow_is_lossless(geom_full, maps_full):
    """A PU200 event searched with stages of 4 (T5) and 2 (pT) survivors per work
    item: many items take the second-enumeration path; every level still
    matches the oracle."""
    ctx = make_context(geom_full, maps_full, max_events=1)
    ctx.set_stage_limits(4, 2)
    ev = E.pu200_event(12, geom_full)
    ctx.run([ev])
    assert ctx.counters()[20] > 100 and ctx.counters()[28] > 100
    g = gpu_result(ctx)
    _no_drops(g)
    o = oracle_result(geom_full, maps_full, ev)
    compare(g, o, A_HALF, DEFAULT_CUTS)
    limited = _all_tuples(ctx, 0)
    ctx.set_stage_limits(0, 0)
    ctx.run([ev])
    assert ctx.counters()[20] == 0 and ctx.counters()[28] == 0
    assert _all_tuples(ctx, 0) == limited
    ctx.close()


def test_batch_equals_single_events(ctx_full, geom_full):
    evs = [E.pileup_event(pu, 40 + i, geom_full) for i, pu in enumerate((10, 50, 3, 80))]
    ctx_full.run(evs)
    batched = [_all_tuples(ctx_full, i) for i in range(len(evs))]
    for i, ev in enumerate(evs):
        ctx_full.run([ev])
        assert _all_tuples(ctx_full, 0) == batched[i]


def test_empty_and_seedless_events(ctx_barrel, geom_barrel, maps_barrel):
    empty = E.Event(x=np.zeros(0, np.float32), y=np.zeros(0, np.float32), z=np.zeros(0, np.float32),
                    module=np.zeros(0, np.int32), side=np.zeros(0, np.uint8), pid=np.zeros(0, np.int32),
                    seeds=np.zeros((0, 3, 3), np.float32), seed_pid=np.zeros(0, np.int32), tracks=None)
    ev = E.tiny_event(3, geom_barrel)
    seedless = E.Event(x=ev.x, y=ev.y, z=ev.z, module=ev.module, side=ev.side, pid=ev.pid,
                       seeds=np.zeros((0, 3, 3), np.float32), seed_pid=np.zeros(0, np.int32), tracks=ev.tracks)
    ctx_barrel.run([empty, seedless, empty])
    for i in (0, 2):
        g = gpu_result(ctx_barrel, i)
        assert g["tc"]["n"] == 0 and g["md"]["n"] == 0 and g["pls"]["n"] == 0
    g = gpu_result(ctx_barrel, 1)
    o = oracle_result(geom_barrel, maps_barrel, seedless)
    compare(g, o, A_HALF, DEFAULT_CUTS)
    assert set(g["tc"]["type"].tolist()) <= {2}


def test_device_resident_input(ctx_barrel, geom_barrel):
    torch = pytest.importorskip("torch")
    import paper_2209_13711_gb300 as P
    evs = [E.tiny_event(s, geom_barrel) for s in (5, 6)]
    b = P.pack_events(evs)
    ctx_barrel.run_packed(b)
    host = [_all_tuples(ctx_barrel, i) for i in range(2)]
    bd = {k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in b.items()}
    ctx_barrel.run_packed(bd, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert [_all_tuples(ctx_barrel, i) for i in range(2)] == host


@pytest.mark.parametrize("seed", range(4))
def test_noiseless_tracks_one_pt5_each(ctx_barrel, geom_barrel, seed):
    """Noiseless prompt tracks: one candidate per track, a pT5 for every fully contained one."""
    ev = E.tiny_event(seed, geom_barrel, smear=False)
    ctx_barrel.run([ev])
    tc = ctx_barrel.track_candidates(0)
    contained = {t for t in range(ev.tracks.n)
                 if len(ev.module[(ev.pid == t) & (ev.side == 0)]) == 6 and
                 sorted(ev.module[(ev.pid == t) & (ev.side == 0)]) == sorted(ev.module[(ev.pid == t) & (ev.side == 1)])}
    pids = []
    for i in range(tc["n"]):
        h = tc["hits"][i]
        p = set(ev.pid[h[h >= 0]].tolist())
        assert len(p) == 1
        pid = p.pop()
        if pid in contained:
            assert tc["type"][i] == 0
        pids.append(pid)
    assert len(pids) == len(set(pids)) and contained <= set(pids)


def test_capacity_errors(ctx_barrel, geom_barrel):
    import paper_2209_13711_gb300 as P
    evs = [E.tiny_event(0, geom_barrel)] * 9            # context holds 8 events
    with pytest.raises(P.LstError):
        ctx_barrel.run(evs)
    bad = E.tiny_event(1, geom_barrel)
    b = P.pack_events([bad])
    b["seed_off"] = np.array([0, -1], np.int32)          # negative seed count
    with pytest.raises(P.LstError):
        ctx_barrel.run_packed(b)


def test_truncation_is_counted(geom_full, maps_full):
    ctx = make_context(geom_full, maps_full, max_events=1, ls_per_event=2000)
    ev = E.pileup_event(40, 7, geom_full)
    ctx.run([ev])
    st = ctx.stats(0)
    assert st["dropped"]["ls"] > 0 and st["counts"]["ls"] <= 2000
    tc = ctx.track_candidates(0)
    assert tc["n"] >= 0
    ctx.close()


def test_grouped_and_per_thread_refine_agree(geom_full, maps_full):
    """Four PU200 events in one batch take the per-thread pT refine (more than
    16384 candidates); each event alone takes the grouped one. Same objects."""
    evs = [E.pu200_event(70 + i, geom_full) for i in range(4)]
    ctx = make_context(geom_full, maps_full, max_events=4)
    ctx.run(evs)
    assert ctx.counters()[4] > 16384 and ctx.counters()[5] > 16384
    batched = [_all_tuples(ctx, i) for i in range(4)]
    one = make_context(geom_full, maps_full, max_events=1)
    for i, ev in enumerate(evs):
        one.run([ev])
        assert one.counters()[4] <= 16384
        assert _all_tuples(one, 0) == batched[i]
    ctx.close()
    one.close()


def test_compact_storage_gives_the_same_objects(geom_full, maps_full):
    """16-bit copies for the searches' curvature prefilters and the cleaning's eta-phi lists: every object
    level and the track candidates equal those of the default storage, and the oracle's."""
    ev = E.pu200_event(7, geom_full)
    plain = make_context(geom_full, maps_full, max_events=1)
    plain.run([ev])
    want = _all_tuples(plain, 0)
    plain.close()
    ctx = make_context(geom_full, maps_full, max_events=1)
    ctx.set_compact_storage(True)
    ctx.run([ev])
    assert _all_tuples(ctx, 0) == want
    g = gpu_result(ctx)
    _no_drops(g)
    compare(g, oracle_result(geom_full, maps_full, ev), A_HALF, DEFAULT_CUTS)
    ctx.close()


def test_compact_storage_batch_equals_default(geom_full, maps_full):
    evs = [E.pileup_event(60 + 20 * i, 70 + i, geom_full) for i in range(6)]
    res = []
    for compact in (False, True):
        ctx = make_context(geom_full, maps_full, max_events=6)
        ctx.set_compact_storage(compact)
        ctx.run(evs)
        res.append([_all_tuples(ctx, e) for e in range(6)])
        ctx.close()
    assert res[0] == res[1]


@pytest.mark.parametrize("seed", [1, 2])
def test_displaced_muon_gun_parity(geom_full, seed):
    """Muons from vertices in a 5 cm cube, with the connection map that covers them: every object level and
    the track candidates against the oracle; T5s are built for muons with d0 above 1 cm."""
    import math
    from synth import maps as M
    maps = M.load_maps(geom_full, M.MapParams(d0_max=2.5 * math.sqrt(2.0)))
    ev = E.muon_gun_event(seed, geom_full, n=60)
    ctx = make_context(geom_full, maps, max_events=1)
    ctx.run([ev])
    g = gpu_result(ctx)
    _no_drops(g)
    s = compare(g, oracle_result(geom_full, maps, ev), A_HALF, DEFAULT_CUTS)
    assert s["t5"][0] > 0
    d0 = ev.tracks.d0
    t5_tc = [h[h >= 0] for t, h in zip(g["tc"]["type"], g["tc"]["hits"]) if t == 2]
    assert any(d0[np.bincount(ev.pid[h]).argmax()] > 1.0 for h in t5_tc if len(h))
    ctx.close()


def _fit_rows(ctx, event):
    """T5 / pT5 / pT3 fit outputs keyed by the object's hit tuple (object indices depend on the run)."""
    from tests.parity import chain_tuples
    g = gpu_result(ctx, event)
    T = chain_tuples(g)
    out = {}
    for kind, vals in (("t5", ("kappa", "chi2_rphi", "chi2_rz", "eta", "phi0", "pt")),
                       ("pt5", ("kappa", "chi2_rphi", "chi2_rz", "pt")), ("pt3", ("kappa", "chi2_rphi", "chi2_rz", "pt"))):
        v = np.stack([g[kind][c] for c in vals], 1).astype(np.float64)
        out[kind] = dict(zip(T[kind], v))
    return out


@pytest.mark.parametrize("n_ev", [1, 4])
def test_float_float_and_fp64_fits_agree(geom_full, maps_full, n_ev):
    """The refine fits in float-float (the default) and in FP64 give the same objects at every level, and fit
    outputs within 2e-6 relative (the FP32 storage of the outputs; the fits themselves agree to ~1e-10).
    One event takes the grouped pT refines, four events the per-thread ones."""
    evs = [E.pu200_event(90 + i, geom_full) for i in range(n_ev)]
    res = []
    for fp64 in (False, True):
        ctx = make_context(geom_full, maps_full, max_events=n_ev)
        ctx.set_fp64_fit(fp64)
        ctx.run(evs)
        res.append([(_all_tuples(ctx, i), _fit_rows(ctx, i)) for i in range(n_ev)])
        ctx.close()
    for (t_ff, f_ff), (t_64, f_64) in zip(*res):
        assert t_ff == t_64
        for kind in f_ff:
            assert f_ff[kind].keys() == f_64[kind].keys() and len(f_ff[kind]) > 100
            a = np.array([f_ff[kind][k] for k in f_64[kind]])
            b = np.array(list(f_64[kind].values()))
            d = np.abs(a - b)
            if kind == "t5":
                d[:, 4] = np.abs(np.angle(np.exp(1j * (a[:, 4] - b[:, 4]))))     # phi0 across the +-pi cut
            assert np.all(d <= 2e-6 * np.abs(b) + 1e-7), kind


def test_cleaning_cells_overflow_matches_the_oracle(geom_full, maps_full):
    """A cleaning distance of 0.3 makes the eta-phi cells 0.6 wide, so busy cells hold more entries than their
    8 slots and the lists' overflow path runs; the track candidates still match the oracle's."""
    import paper_2209_13711_gb300 as P
    from oracle import oracle as O
    cuts = dict(DEFAULT_CUTS, dr_clean=0.3)
    ev = E.pileup_event(60, 31, geom_full)
    ctx = P.Context(geom_full.module_table(), maps_full, cfg=cuts, capacity=P.default_capacity(1))
    ctx.run([ev])
    g = gpu_result(ctx)
    _no_drops(g)
    o = O.Setup(geom_full.module_table(), maps_full, cuts, ev).run()
    s = compare(g, o, A_HALF, cuts)
    assert s["tc"][0] >= 100
    ctx.close()
