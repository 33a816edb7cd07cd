"""Candidate-test counts of the benchmark (CPU): the vectorised counts of
metrics.candidate_tests equal a brute-force enumeration over the oracle's
objects of small events."""
import pytest

from oracle import oracle as O
from paper_2209_13711_gb300.metrics import candidate_tests
from synth import events as E
from synth.config import DEFAULT_CUTS


def brute_force(r, ev, maps, n_mod):
    conn_off, conn_tgt, sb_off, sb_tgt = maps
    conn = [set(conn_tgt[conn_off[m]:conn_off[m + 1]].tolist()) for m in range(n_mod)]
    md, ls, t3, t5, pls = r["md"], r["ls"], r["t3"], r["t5"], r["pls"]
    out = dict(md=0, ls=0, t3=0, t5=0, pt5=0, pt3=0)
    for a in range(ev.n_hits):
        for b in range(ev.n_hits):
            if ev.module[a] == ev.module[b] and ev.side[a] == 0 and ev.side[b] == 1:
                out["md"] += 1
    mod = md["mod"]
    for a in range(md["n"]):
        for b in range(md["n"]):
            out["ls"] += int(mod[b]) in conn[int(mod[a])]
    for a in range(ls["n"]):
        for b in range(ls["n"]):
            out["t3"] += ls["md_out"][a] == ls["md_in"][b]
    inner = [ls["md_in"][t3["ls_in"][i]] for i in range(t3["n"])]
    outer = [ls["md_out"][t3["ls_out"][i]] for i in range(t3["n"])]
    for a in range(t3["n"]):
        for b in range(t3["n"]):
            out["t5"] += outer[a] == inner[b]
    for p in range(pls["n"]):
        if not pls["pass"][p] or pls["sb"][p] < 0:
            continue
        s = int(pls["sb"][p])
        mods = set(sb_tgt[sb_off[s]:sb_off[s + 1]].tolist())
        out["pt3"] += sum(int(mod[inner[i]]) in mods for i in range(t3["n"]))
        out["pt5"] += sum(int(mod[inner[t5["t3_in"][i]]]) in mods for i in range(t5["n"]))
    return out


@pytest.mark.parametrize("which", ["tiny", "pu1"])
def test_candidate_tests_match_brute_force(which, geom_barrel, maps_barrel, geom_full, maps_full):
    if which == "tiny":
        geom, maps, ev = geom_barrel, maps_barrel, E.tiny_event(0, geom_barrel)
    else:
        geom, maps, ev = geom_full, maps_full, E.pileup_event(1, 3, geom_full)
    n_mod = len(maps[0]) - 1
    r = O.Setup(geom.module_table(), maps, DEFAULT_CUTS, ev).run()
    got = candidate_tests(r, ev.module, ev.side, *maps, n_mod)
    want = brute_force(r, ev, maps, n_mod)
    assert got == want
    assert min(got[k] for k in ("md", "ls", "t3")) > 0
