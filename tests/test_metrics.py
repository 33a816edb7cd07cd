"""Efficiency / fake / duplicate rates on generator truth (CPU)."""
import numpy as np
import pytest

from paper_2209_13711_gb300.metrics import combine, match, rates


class _Tracks:
    def __init__(self, pt, eta):
        self.pt = np.asarray(pt, float)
        self.eta = np.asarray(eta, float)


def _tc(rows, seeds):
    hits = np.full((len(rows), 10), -1, np.int32)
    for i, r in enumerate(rows):
        hits[i, :len(r)] = r
    return dict(n=len(rows), hits=hits, seed=np.asarray(seeds, np.int32))


def test_match_majority_with_seed_hits():
    pid = np.array([0] * 10 + [1] * 10 + [-1] * 5)
    seed_pid = np.array([0, 1, -1])
    tc = _tc([list(range(10)),                       # 10/10 from particle 0
              list(range(6)) + list(range(10, 14)),  # 6/10: fake
              list(range(2, 10)) + [20, 21],         # 8/10 from 0 (noise hits count against)
              list(range(6)) + list(range(10, 14)),  # 6 + 3 seed hits of 0 = 9/13 = 0.69: fake
              list(range(10, 18)) + [3, 4],          # 8/10 from 1, seed of 1: 11/13
              []],                                   # pLS only: the seed's particle
             [-1, -1, -1, 0, 1, 1])
    assert list(match(tc, pid, seed_pid)) == [0, -1, 0, -1, 1, 1]
    assert match(tc, pid, seed_pid, frac=0.6)[1] == 0


def test_rates_count_efficiency_fakes_duplicates():
    pid = np.array([0] * 10 + [1] * 10 + [2] * 10)
    tr = _Tracks([2.0, 8.0, 0.5], [0.1, -1.0, 0.2])   # particle 2 below pT threshold
    tc = _tc([list(range(10)), list(range(10)), list(range(20, 30)), [0, 10, 20, 1, 11]], [-1, -1, -1, -1])
    r = rates(tc, pid, np.zeros(0, np.int32), tr, pt_min=1.0)
    assert r["findable"] == 2 and r["found"] == 1
    assert r["efficiency"] == pytest.approx(0.5)
    assert r["fake_rate"] == pytest.approx(0.25)       # the mixed TC
    assert r["duplicate_rate"] == pytest.approx(0.25)  # second TC of particle 0
    c = combine([r, r])
    assert c["efficiency"] == pytest.approx(0.5) and c["tcs"] == 8 and c["events"] == 2


def test_oracle_chain_physics_on_a_pileup_event(geom_full, maps_full):
    """The chain (oracle) finds most tracks above 2 GeV with few fakes and duplicates."""
    from oracle import oracle as O
    from synth import events as E
    from synth.config import DEFAULT_CUTS
    ev = E.pileup_event(10, 5, geom_full)
    o = O.Setup(geom_full.module_table(), maps_full, DEFAULT_CUTS, ev).run()["tc"]
    tc = dict(n=o["n"], hits=np.stack([o[f"h{i}"] for i in range(10)], 1), seed=o["seed"])
    r = rates(tc, ev.pid, ev.seed_pid, ev.tracks, pt_min=2.0, eta_max=2.4)
    assert r["findable"] > 20
    assert r["efficiency"] > 0.85
    assert r["fake_rate"] < 0.2 and r["duplicate_rate"] < 0.2


def test_curves_bin_counts_agree_with_rates():
    from paper_2209_13711_gb300.metrics import curves
    pid = np.array([0] * 10 + [1] * 10 + [2] * 10)
    tr = _Tracks([2.0, 8.0, 0.5], [0.1, -1.0, 0.2])
    tc = _tc([list(range(10)), list(range(10)), list(range(20, 30)), [0, 10, 20, 1, 11]], [-1, -1, -1, 5])
    tc.update(type=np.array([2, 2, 2, 1]), pt=np.array([2.1, 1.9, 0.6, 30.0]), eta=np.array([0.1, 0.1, 0.2, 2.0]))
    c = curves([(tc, pid, np.full(6, -1, np.int32), tr)])
    pe = c["pt_edges"]
    eff = np.array(c["efficiency_vs_pt"])
    # generated pT 2.0 -> bin [2, 3), 8.0 -> [5, 10), 0.5 -> [0.5, 0.8); particle 1 only in the mixed TC (a fake)
    assert eff[pe.index(2.0)].tolist() == [1, 1] and eff[pe.index(5.0)].tolist() == [0, 1]
    assert eff[pe.index(0.5)].tolist() == [1, 1] and eff[:, 1].sum() == 3
    # efficiency vs eta only for pT >= 1: two particles
    assert np.array(c["efficiency_vs_eta"])[:, 1].sum() == 2
    fake = np.array(c["fake_vs_pt"])
    assert fake[:, 1].sum() == 4 and fake[:, 0].sum() == 1 and fake[pe.index(20.0)].tolist() == [1, 1]
    dup = np.array(c["duplicate_vs_pt"])
    assert dup[:, 0].sum() == 1 and dup[pe.index(1.5)].tolist() == [1, 1]   # the second TC of particle 0
    assert c["by_type"]["T5"]["tcs"] == 3 and c["by_type"]["pT3"]["fake_rate"] == 1.0
    assert c["by_type"]["T5"]["duplicate_rate"] == pytest.approx(1 / 3)
    # pooled over bins the rates equal rates()
    r = rates(tc, pid, np.full(6, -1, np.int32), tr, pt_min=1.0)
    assert fake[:, 0].sum() / fake[:, 1].sum() == pytest.approx(r["fake_rate"])


def test_efficiency_without_bare_seeds():
    pid = np.array([0] * 10 + [1] * 10)
    tr = _Tracks([2.0, 3.0], [0.1, 0.2])
    tc = _tc([list(range(10)), []], [-1, 0])
    tc["type"] = np.array([2, 3])                       # a T5 of particle 0, a bare pLS of particle 1
    r = rates(tc, pid, np.array([1], np.int32), tr)
    assert r["efficiency"] == pytest.approx(1.0) and r["efficiency_ot"] == pytest.approx(0.5)
    assert combine([r, r])["efficiency_ot"] == pytest.approx(0.5)


def test_efficiency_vs_d0_by_type():
    from paper_2209_13711_gb300 import metrics as MT
    from synth.events import Tracks
    tr = Tracks(pt=np.full(4, 3.0), eta=np.zeros(4), phi0=np.zeros(4), q=np.ones(4), z0=np.zeros(4),
                x0=np.array([0.0, 0.0, 0.0, 0.0]), y0=np.array([0.1, 0.7, 1.7, 3.0]))
    # straight-line d0 = |y0| for phi0 = 0 up to the curvature; particle i owns hits 2i, 2i+1
    pid = np.repeat(np.arange(4), 10)
    hits = np.full((3, 10), -1)
    hits[0, :] = np.arange(0, 10)          # particle 0 by a pT5
    hits[1, :] = np.arange(20, 30)         # particle 2 by a T5
    hits[2, :] = np.arange(30, 40)         # particle 3 by a T5
    tc = dict(n=3, hits=hits, seed=np.array([-1, -1, -1]), type=np.array([0, 2, 2]))
    r = MT.efficiency_vs_d0([(tc, pid, np.zeros(0, np.int64), tr)], edges=(0.0, 0.5, 1.0, 2.0, 3.6))
    assert r["findable"] == [1, 1, 1, 1]
    assert r["efficiency"] == [1.0, 0.0, 1.0, 1.0]
    assert r["efficiency_by_type"]["T5"] == [0.0, 0.0, 1.0, 1.0]
    assert r["efficiency_by_type"]["pT5"] == [1.0, 0.0, 0.0, 0.0]
