"""Chain-level pins of the oracle: brute-force completeness and invariants."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from synth import events as E


def _setup(geom, maps, cuts, ev):
    return O.Setup(geom.module_table(), maps, cuts, ev)


def _sets(r):
    md = r["md"]
    md_t = [(int(a), int(b)) for a, b in zip(md["lo"], md["up"])]
    ls = r["ls"]
    ls_t = [(md_t[a], md_t[b]) for a, b in zip(ls["md_in"], ls["md_out"])]
    t3 = r["t3"]
    t3_t = [(ls_t[a][0], ls_t[a][1], ls_t[b][1]) for a, b in zip(t3["ls_in"], t3["ls_out"])]
    t5 = r["t5"]
    t5_t = [t3_t[a] + t3_t[b][1:] for a, b in zip(t5["t3_in"], t5["t3_out"])]
    return md_t, ls_t, t3_t, t5_t


@pytest.fixture(scope="module", params=[0, 1, 2, 3])
def tiny(request, geom_barrel, maps_barrel, cuts):
    ev = E.tiny_event(request.param, geom_barrel)
    S = _setup(geom_barrel, maps_barrel, cuts, ev)
    return ev, S, S.run()


def test_brute_force_md_ls(tiny, geom_barrel, maps_barrel):
    """All hit pairs / all MD pairs evaluated without the hierarchy equal the oracle's lists."""
    ev, S, r = tiny
    md_t, ls_t, _, _ = _sets(r)
    brute_md = set()
    for i, j in itertools.product(range(ev.n_hits), repeat=2):
        if ev.module[i] == ev.module[j] and ev.side[i] == 0 and ev.side[j] == 1:
            ok, _ = S.pred_md(i, j)
            if ok:
                brute_md.add((i, j))
    assert brute_md == set(md_t) and len(md_t) == len(set(md_t))
    co, ct = maps_barrel[0], maps_barrel[1]
    brute_ls = set()
    for A, B in itertools.product(sorted(brute_md), repeat=2):
        mA, mB = ev.module[A[0]], ev.module[B[0]]
        if mB not in ct[co[mA]:co[mA + 1]]:
            continue
        ok, _ = S.pred_chain(list(A) + list(B), 1)
        if ok:
            brute_ls.add((A, B))
    assert brute_ls == set(ls_t) and len(ls_t) == len(set(ls_t))


def test_brute_force_t3_t5(tiny):
    """All MD triples / 5-tuples linked by segments, evaluated directly, equal the oracle's T3 / T5."""
    ev, S, r = tiny
    md_t, ls_t, t3_t, t5_t = _sets(r)
    ls_set = set(ls_t)
    succ = {}
    for a, b in ls_set:
        succ.setdefault(a, []).append(b)
    brute_t3 = set()
    for a in succ:
        for b in succ[a]:
            for c in succ.get(b, []):
                ok, _ = S.pred_chain(list(a) + list(b) + list(c), 2)
                if ok:
                    brute_t3.add((a, b, c))
    assert brute_t3 == set(t3_t)
    brute_t5 = set()
    for t in brute_t3:
        for u in brute_t3:
            if u[0] == t[2]:
                tup = t + u[1:]
                ok, _ = S.pred_chain([h for md in tup for h in md], 3)
                if ok:
                    brute_t5.add(tup)
    assert brute_t5 == set(t5_t)


def test_brute_force_pixel_objects(tiny, geom_barrel, maps_barrel, cuts):
    """pT5 / pT3: every (passing pLS, T object whose inner module is in its superbin) pair evaluated directly."""
    ev, S, r = tiny
    md_t, ls_t, t3_t, t5_t = _sets(r)
    Pd = O.Predicates(S)
    so, st = maps_barrel[2], maps_barrel[3]
    mt = geom_barrel.module_table()

    def hit_row(h):
        m = ev.module[h]
        bar = mt["subdet"][m] == 0
        return [float(ev.x[h]), float(ev.y[h]), float(ev.z[h]), float(mt["sig_rphi"][m]),
                float(mt["sig_long"][m]) if bar else 0.0, 0.0 if bar else float(mt["sig_long"][m])]

    pls = r["pls"]
    for kind, objs, key in (("pt5", t5_t, "t5"), ("pt3", t3_t, "t3")):
        brute = set()
        for s in range(ev.n_seeds):
            if not pls["pass"][s] or pls["sb"][s] < 0:
                continue
            mods = set(st[so[pls["sb"][s]]:so[pls["sb"][s] + 1]].tolist())
            prow = [list(map(float, ev.seeds[s, j])) + [cuts["sig_pix"], cuts["sig_pix"], 0.0] for j in range(3)]
            for i, tup in enumerate(objs):
                if ev.module[tup[0][0]] not in mods:
                    continue
                rows = prow + [hit_row(md[0]) for md in tup]
                if key == "t5":
                    kt, sk = r["t5"]["kappa"][i], r["t5"]["sigk"][i]
                else:
                    kt, sk = r["t3"]["kappa"][i], r["t3"]["sigk"][i]
                ok, _ = Pd.pt(rows, pls["kappa"][s], pls["sigk"][s], kt, sk)
                if ok:
                    brute.add((s, tup))
        got = {(int(s), objs[o]) for s, o in zip(r[kind]["seed"], r[kind][key])}
        assert brute == got


def test_invariants(tiny, geom_barrel, maps_barrel):
    ev, S, r = tiny
    md = r["md"]
    # each MD: one lower and one upper hit of the same module
    assert np.all(ev.module[md["lo"]] == md["mod"]) and np.all(ev.module[md["up"]] == md["mod"])
    assert np.all(ev.side[md["lo"]] == 0) and np.all(ev.side[md["up"]] == 1)
    # each LS links map-connected modules
    co, ct = maps_barrel[0], maps_barrel[1]
    for a, b in zip(r["ls"]["md_in"], r["ls"]["md_out"]):
        m1, m2 = md["mod"][a], md["mod"][b]
        assert m2 in ct[co[m1]:co[m1 + 1]]
    # T3 segments share the middle MD, T5 triplets share an MD
    ls = r["ls"]
    assert np.all(ls["md_out"][r["t3"]["ls_in"]] == ls["md_in"][r["t3"]["ls_out"]])
    t3 = r["t3"]
    assert np.all(ls["md_out"][t3["ls_out"][r["t5"]["t3_in"]]] == ls["md_in"][t3["ls_in"][r["t5"]["t3_out"]]])
    # no two track candidates share a hit (OT hit or pixel seed)
    tc = r["tc"]
    seen = set()
    for i in range(tc["n"]):
        hs = [int(tc[f"h{j}"][i]) for j in range(10) if tc[f"h{j}"][i] >= 0]
        if tc["seed"][i] >= 0:
            hs.append(("seed", int(tc["seed"][i])))
        for h in hs:
            assert h not in seen
            seen.add(h)


def test_permutation_invariance(tiny, geom_barrel, maps_barrel, cuts):
    ev, S, r = tiny
    rng = np.random.default_rng(99)
    perm = rng.permutation(ev.n_hits)
    inv = np.argsort(perm)
    ev2 = E.Event(x=ev.x[perm], y=ev.y[perm], z=ev.z[perm], module=ev.module[perm], side=ev.side[perm],
                  pid=ev.pid[perm], seeds=ev.seeds, seed_pid=ev.seed_pid, tracks=ev.tracks)
    r2 = _setup(geom_barrel, maps_barrel, cuts, ev2).run()

    def tc_set(rr, mapping):
        out = set()
        tc = rr["tc"]
        for i in range(tc["n"]):
            hs = tuple(sorted(int(mapping[tc[f"h{j}"][i]]) for j in range(10) if tc[f"h{j}"][i] >= 0))
            out.add((int(tc["type"][i]), int(tc["seed"][i]), hs))
        return out

    assert tc_set(r, np.arange(ev.n_hits)) == tc_set(r2, perm)
    assert r["md"]["n"] == r2["md"]["n"] and r["t5"]["n"] == r2["t5"]["n"]


@pytest.mark.parametrize("seed", range(6))
def test_noiseless_one_candidate_per_track(seed, geom_barrel, maps_barrel, cuts):
    """Noiseless prompt tracks with a pixel seed and all six layers give exactly one pT5 each."""
    ev = E.tiny_event(seed, geom_barrel, smear=False)
    r = _setup(geom_barrel, maps_barrel, cuts, ev).run()
    # tracks whose two hits in every layer sit in one module
    good = []
    for t in range(ev.tracks.n):
        sel = ev.pid == t
        mods_lo = sorted(ev.module[sel & (ev.side == 0)])
        mods_up = sorted(ev.module[sel & (ev.side == 1)])
        if len(mods_lo) == 6 and mods_lo == mods_up:
            good.append(t)
    tc = r["tc"]
    pid_of_tc = []
    for i in range(tc["n"]):
        hs = [int(tc[f"h{j}"][i]) for j in range(10) if tc[f"h{j}"][i] >= 0]
        pids = set(ev.pid[hs].tolist())
        assert len(pids) == 1
        pid = pids.pop()
        if pid in good:
            assert tc["type"][i] == 0                  # pT5
        assert ev.seed_pid[tc["seed"][i]] == pid
        pid_of_tc.append(pid)
    assert sorted(pid_of_tc) == sorted(set(pid_of_tc))
    assert set(good) <= set(pid_of_tc)
    assert r["m_md"].shape[0] == 0 and r["m_t5"].shape[0] == 0


@pytest.mark.parametrize("pu,seed", [(10, 5), (25, 7)])
def test_cleaning_is_idempotent(pu, seed, geom_full, maps_full, cuts):
    """Re-running the cross-cleaning on its own output removes nothing: no kept
    pT3 is close to a kept pT5, no kept T5 to a kept pT5 or pT3, and no kept
    pLS to any kept pT5, pT3 or T5 (close: eta-phi distance below dr_clean, or
    a shared hit); no two kept objects share a hit or a seed."""
    ev = E.pileup_event(pu, seed, geom_full)
    tc = _setup(geom_full, maps_full, cuts, ev).run()["tc"]
    n = tc["n"]
    assert n > 20
    hits = [frozenset(int(tc[f"h{j}"][i]) for j in range(10) if tc[f"h{j}"][i] >= 0) for i in range(n)]
    kind = np.asarray(tc["type"])
    thr2 = cuts["dr_clean"] ** 2

    def close(i, j):
        dphi = (tc["phi0"][i] - tc["phi0"][j] + np.pi) % (2 * np.pi) - np.pi
        return bool(hits[i] & hits[j]) or (tc["eta"][i] - tc["eta"][j]) ** 2 + dphi ** 2 < thr2

    higher = {1: (0,), 2: (0, 1), 3: (0, 1, 2)}        # pT3 | T5 | pLS against the categories cleaned first
    by_kind = {k: np.flatnonzero(kind == k) for k in range(4)}
    assert all(len(by_kind[k]) for k in (0, 1, 3))
    for k, hs in higher.items():
        for i in by_kind[k]:
            for h in hs:
                for j in by_kind[h]:
                    assert not close(i, j), (k, i, h, j)
    seeds = [int(s) for s in tc["seed"] if s >= 0]
    assert len(seeds) == len(set(seeds))
    for i, j in itertools.combinations(range(n), 2):
        assert not (hits[i] & hits[j])


@pytest.mark.parametrize("pu,seed", [(10, 5), (25, 7)])
def test_cleaning_drops_only_with_cause(pu, seed, geom_full, maps_full, cuts):
    """Every candidate the cleaning drops has a reason in the output: a pT5 a
    hit-sharing pT5 with no larger score; a pT3 such a pT3 or closeness to a
    kept pT5; a T5 such a T5 or closeness to a kept pT5 or pT3; a passing pLS
    a kept pT5/pT3 built on it or closeness to any kept pT5, pT3 or T5."""
    ev = E.pileup_event(pu, seed, geom_full)
    r = _setup(geom_full, maps_full, cuts, ev).run()
    md, ls, t3, t5, pls, pt5, pt3, tc = (r[k] for k in ("md", "ls", "t3", "t5", "pls", "pt5", "pt3", "tc"))
    nh = len(ev.x)
    md_h = lambda m: {int(md["lo"][m]), int(md["up"][m])}
    t3_mds = lambda i: (ls["md_in"][t3["ls_in"][i]], ls["md_out"][t3["ls_in"][i]], ls["md_out"][t3["ls_out"][i]])
    t5_mds = lambda i: t3_mds(t5["t3_in"][i]) + t3_mds(t5["t3_out"][i])[1:]
    pix = lambda s: {nh + 3 * int(s) + j for j in range(3)}
    union = lambda ms: set().union(*(md_h(m) for m in ms))
    H = {0: [union(t5_mds(pt5["t5"][i])) | pix(pt5["seed"][i]) for i in range(pt5["n"])],
         1: [union(t3_mds(pt3["t3"][i])) | pix(pt3["seed"][i]) for i in range(pt3["n"])],
         2: [union(t5_mds(i)) for i in range(t5["n"])],
         3: [pix(pls["seed"][i]) for i in range(pls["n"])]}
    ang = {0: [(pls["eta"][s], pls["phi0"][s]) for s in pt5["seed"]],
           1: [(pls["eta"][s], pls["phi0"][s]) for s in pt3["seed"]],
           2: list(zip(t5["eta"], t5["phi0"])), 3: list(zip(pls["eta"], pls["phi0"]))}
    score = {0: pt5["score"], 1: pt3["score"], 2: t5["score"]}
    kept = {k: set(int(o) for t, o in zip(tc["type"], tc["obj"]) if t == k) for k in range(4)}
    thr2 = cuts["dr_clean"] ** 2

    def close(c1, i, c2, j):
        (e1, p1), (e2, p2) = ang[c1][i], ang[c2][j]
        dphi = (p1 - p2 + np.pi) % (2 * np.pi) - np.pi
        return bool(H[c1][i] & H[c2][j]) or (e1 - e2) ** 2 + dphi ** 2 < thr2

    def beaten(c, i):
        return any(j != i and H[c][i] & H[c][j] and score[c][j] <= score[c][i] for j in range(len(H[c])))

    dropped = {k: [i for i in range(len(H[k])) if i not in kept[k]] for k in range(3)}
    assert sum(len(v) for v in dropped.values()) > 0
    for i in dropped[0]:
        assert beaten(0, i), i
    for i in dropped[1]:
        assert beaten(1, i) or any(close(1, i, 0, j) for j in kept[0]), i
    for i in dropped[2]:
        assert beaten(2, i) or any(close(2, i, c, j) for c in (0, 1) for j in kept[c]), i
    linked = {int(pt5["seed"][j]) for j in kept[0]} | {int(pt3["seed"][j]) for j in kept[1]}
    for i in range(pls["n"]):
        if pls["pass"][i] and i not in kept[3]:
            assert int(pls["seed"][i]) in linked or any(close(3, i, c, j) for c in (0, 1, 2) for j in kept[c]), i
