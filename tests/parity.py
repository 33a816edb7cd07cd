"""GPU-vs-oracle parity of the Segment Linking chain (test helper).

Objects are compared as sets of hit-index tuples. Candidates whose own cut
variable lies within 1e-5 relative of a threshold in the FP64 oracle (the
oracle's margin lists), and every object built on such a candidate, are
removed from both sides before the comparison. Track candidates are compared
after removing, in addition, every object whose cleaning decision could
depend on a removed object or on a near-threshold cleaning comparison (a
closure over hit sharing and eta-phi proximity, to the depth of the
cleaning's dependency chain). Derived FP32 quantities must satisfy
|x32 - x64| <= 1e-5 max(|x64|, scale), scale = the threshold the quantity is
cut against.
"""
import math

import numpy as np

REL = 1e-5


def _md_tuples(lo, up):
    return [(int(a), int(b)) for a, b in zip(lo, up)]


def chain_tuples(r):
    """Hit-index tuples of every level from a result dict (GPU or oracle layout)."""
    md_t = _md_tuples(r["md"]["lo"], r["md"]["up"])
    ls_t = [(md_t[a], md_t[b]) for a, b in zip(r["ls"]["md_in"], r["ls"]["md_out"])]
    t3_t = [(ls_t[a][0], ls_t[a][1], ls_t[b][1]) for a, b in zip(r["t3"]["ls_in"], r["t3"]["ls_out"])]
    t5_t = [t3_t[a] + t3_t[b][1:] for a, b in zip(r["t5"]["t3_in"], r["t5"]["t3_out"])]
    pt5_t = [(int(s), t5_t[o]) for s, o in zip(r["pt5"]["seed"], r["pt5"]["t5"])]
    pt3_t = [(int(s), t3_t[o]) for s, o in zip(r["pt3"]["seed"], r["pt3"]["t3"])]
    return dict(md=md_t, ls=ls_t, t3=t3_t, t5=t5_t, pt5=pt5_t, pt3=pt3_t)


class Margins:
    def __init__(self, orc):
        T = chain_tuples(orc)
        self.md = {(int(a), int(b)) for a, b in orc["m_md"]}
        self.ls = {(T["md"][a], T["md"][b]) for a, b in orc["m_ls"]}
        self.t3 = {(T["ls"][a][0], T["ls"][a][1], T["ls"][b][1]) for a, b in orc["m_t3"]}
        self.t5 = {T["t3"][a] + T["t3"][b][1:] for a, b in orc["m_t5"]}
        self.pls = {int(s) for s in orc["m_pls"].ravel()}
        self.pt5 = {(int(s), T["t5"][b]) for s, b in orc["m_pt5"]}
        self.pt3 = {(int(s), T["t3"][b]) for s, b in orc["m_pt3"]}

    def ex_md(self, t):
        return t in self.md

    def ex_ls(self, t):
        return t in self.ls or self.ex_md(t[0]) or self.ex_md(t[1])

    def ex_t3(self, t):
        return t in self.t3 or self.ex_ls((t[0], t[1])) or self.ex_ls((t[1], t[2]))

    def ex_t5(self, t):
        return t in self.t5 or self.ex_t3(t[:3]) or self.ex_t3(t[2:])

    def ex_pt5(self, t):
        return t in self.pt5 or t[0] in self.pls or self.ex_t5(t[1])

    def ex_pt3(self, t):
        return t in self.pt3 or t[0] in self.pls or self.ex_t3(t[1])

    def empty(self):
        return not (self.md or self.ls or self.t3 or self.t5 or self.pls or self.pt5 or self.pt3)


def close(x32, x64, scale):
    return abs(float(x32) - float(x64)) <= REL * max(abs(float(x64)), scale)


def compare(gpu, orc, a_half, cuts, check_tc=True):
    """Assert parity; returns a summary dict."""
    G = chain_tuples(gpu)
    O = chain_tuples(orc)
    M = Margins(orc)
    summary = {}
    for lvl in ("md", "ls", "t3", "t5", "pt5", "pt3"):
        ex = getattr(M, "ex_" + lvl)
        g = {t for t in G[lvl] if not ex(t)}
        o = {t for t in O[lvl] if not ex(t)}
        assert len(G[lvl]) == len(set(G[lvl])), f"{lvl}: duplicate GPU objects"
        only_g, only_o = g - o, o - g
        assert not only_g and not only_o, (f"{lvl}: {len(only_g)} GPU-only, {len(only_o)} oracle-only; "
                                           f"e.g. {sorted(only_g)[:2]} / {sorted(only_o)[:2]}")
        summary[lvl] = (len(g), len(G[lvl]) - len(g))
    # derived quantities of objects present on both sides
    def idx(lst):
        return {t: i for i, t in enumerate(lst)}
    two_a = 2 * a_half
    gi, oi = idx(G["md"]), idx(O["md"])
    for t, i in gi.items():
        j = oi.get(t)
        if j is None:
            continue
        assert close(gpu["md"]["dphi"][i], orc["md"]["dphi"][j], orc["md"]["thr_phi"][j]), ("md dphi", t)
        assert close(gpu["md"]["dlong"][i], orc["md"]["dlong"][j], orc["md"]["thr_long"][j]), ("md dlong", t)
    gi, oi = idx(G["ls"]), idx(O["ls"])
    for t, i in gi.items():
        j = oi.get(t)
        if j is not None:
            assert close(gpu["ls"]["dphi"][i], orc["ls"]["dphi"][j], orc["ls"]["thr_phi"][j]), ("ls dphi", t)
    gi, oi = idx(G["t3"]), idx(O["t3"])
    for t, i in gi.items():
        j = oi.get(t)
        if j is None:
            continue
        assert close(gpu["t3"]["beta"][i], orc["t3"]["beta"][j], orc["t3"]["thr_beta"][j]), ("t3 beta", t)
        assert close(gpu["t3"]["kappa"][i], orc["t3"]["kappa"][j], two_a), ("t3 kappa", t)
        assert close(gpu["t3"]["sigk"][i], orc["t3"]["sigk"][j], 0.0), ("t3 sigk", t)
    gi, oi = idx(G["t5"]), idx(O["t5"])
    for t, i in gi.items():
        j = oi.get(t)
        if j is None:
            continue
        g5, o5 = gpu["t5"], orc["t5"]
        assert close(g5["kappa"][i], o5["kappa"][j], two_a), ("t5 kappa", t)
        assert close(g5["chi2_rphi"][i], o5["chi2_rphi"][j], cuts["chi2_rphi_t5"]), ("t5 chi2", t)
        assert close(g5["chi2_rz"][i], o5["chi2_rz"][j], cuts["chi2_rz_t5"]), ("t5 chi2z", t)
        assert close(g5["eta"][i], o5["eta"][j], 1.0) and close(g5["phi0"][i], o5["phi0"][j], math.pi), ("t5 dir", t)
        assert close(g5["pt"][i], o5["pt"][j], 0.0), ("t5 pt", t)
    gp, op = gpu["pls"], orc["pls"]
    assert gp["n"] == op["n"]
    for s in range(op["n"]):
        if s in M.pls:
            continue
        assert gp["pass"][s] == op["pass"][s] and gp["sb"][s] == op["sb"][s], ("pls", s)
        assert close(gp["kappa"][s], op["kappa"][s], two_a), ("pls kappa", s)
        assert close(gp["eta"][s], op["eta"][s], 1.0) and close(gp["phi0"][s], op["phi0"][s], math.pi), ("pls dir", s)
        assert close(gp["z0"][s], op["z0"][s], cuts["z_lumi"]), ("pls z0", s)
    for lvl, cr, cz in (("pt5", "chi2_rphi_pt5", "chi2_rz_pt5"), ("pt3", "chi2_rphi_pt3", "chi2_rz_pt3")):
        gi, oi = idx(G[lvl]), idx(O[lvl])
        for t, i in gi.items():
            j = oi.get(t)
            if j is None:
                continue
            assert close(gpu[lvl]["kappa"][i], orc[lvl]["kappa"][j], two_a), (lvl, "kappa", t)
            assert close(gpu[lvl]["chi2_rphi"][i], orc[lvl]["chi2_rphi"][j], cuts[cr]), (lvl, "chi2", t)
            assert close(gpu[lvl]["chi2_rz"][i], orc[lvl]["chi2_rz"][j], cuts[cz]), (lvl, "chi2z", t)
    if check_tc:
        summary["tc"] = compare_tc(gpu, orc, G, O, M, cuts)
    return summary


def _obj_info(r, T, cat, i):
    """(hit set, eta, phi) of a cleaning candidate; cat 0 pT5, 1 pT3, 2 T5, 3 pLS."""
    pls = r["pls"]
    if cat == 3:
        s = i
        return {("p", s)}, float(pls["eta"][s]), float(pls["phi0"][s])
    if cat == 2:
        t = T["t5"][i]
        return {h for md in t for h in md}, float(r["t5"]["eta"][i]), float(r["t5"]["phi0"][i])
    key = "pt5" if cat == 0 else "pt3"
    s, t = T[key][i]
    return {("p", s)} | {h for md in t for h in md}, float(pls["eta"][s]), float(pls["phi0"][s])


def compare_tc(gpu, orc, G, O, M, cuts):
    def tc_set(tc):
        out = {}
        for i in range(tc["n"]):
            hs = tuple(sorted(int(h) for h in (tc["hits"][i] if "hits" in tc else
                                               [tc[f"h{j}"][i] for j in range(10)]) if h >= 0))
            out[(int(tc["type"][i]), int(tc["seed"][i]), hs)] = i
        return out

    g_tc, o_tc = tc_set(gpu["tc"]), tc_set(orc["tc"])
    # tainted seeds: margin objects on either side and near-threshold cleaning comparisons
    tainted = []
    for side, r, T in (("g", gpu, G), ("o", orc, O)):
        for i, t in enumerate(T["pt5"]):
            if M.ex_pt5(t):
                tainted.append(_obj_info(r, T, 0, i))
        for i, t in enumerate(T["pt3"]):
            if M.ex_pt3(t):
                tainted.append(_obj_info(r, T, 1, i))
        for i, t in enumerate(T["t5"]):
            if M.ex_t5(t):
                tainted.append(_obj_info(r, T, 2, i))
        for s in M.pls:
            tainted.append(_obj_info(r, T, 3, s))
    for c1, i1, c2, i2 in orc["m_clean"]:
        tainted.append(_obj_info(orc, O, int(c1), int(i1)))
        tainted.append(_obj_info(orc, O, int(c2), int(i2)))
    if tainted:
        # candidate universe: every cleaning candidate on both sides
        cands = []
        for r, T in ((gpu, G), (orc, O)):
            for cat, key in ((0, "pt5"), (1, "pt3"), (2, "t5")):
                for i in range(len(T[key])):
                    cands.append(_obj_info(r, T, cat, i))
            for s in range(r["pls"]["n"]):
                cands.append(_obj_info(r, T, 3, s))
        thr = cuts["dr_clean"] * (1 + 1e-4)
        taint_hits = set()
        taint_dirs = []
        for h, e, p in tainted:
            taint_hits |= h
            taint_dirs.append((e, p))
        for _ in range(5):                # depth of the cleaning's dependency chain
            new_hits, new_dirs = set(), []
            for h, e, p in cands:
                if h <= taint_hits:
                    continue
                near = bool(h & taint_hits) or any(
                    (e - e2) ** 2 + math.remainder(p - p2, 2 * math.pi) ** 2 < thr * thr for e2, p2 in taint_dirs)
                if near:
                    new_hits |= h
                    new_dirs.append((e, p))
            if not (new_hits - taint_hits):
                break
            taint_hits |= new_hits
            taint_dirs += new_dirs
    else:
        taint_hits = set()

    def ok(key):
        typ, seed, hs = key
        hits = set(hs) | ({("p", seed)} if seed >= 0 and typ != 2 else set())
        return not (hits & taint_hits)

    g = {k for k in g_tc if ok(k)}
    o = {k for k in o_tc if ok(k)}
    assert g == o, f"tc: {len(g - o)} GPU-only {sorted(g - o)[:2]}, {len(o - g)} oracle-only {sorted(o - g)[:2]}"
    # kinematics of matched candidates
    for k in g:
        i, j = g_tc[k], o_tc[k]
        assert close(gpu["tc"]["eta"][i], orc["tc"]["eta"][j], 1.0)
        assert close(gpu["tc"]["phi0"][i], orc["tc"]["phi0"][j], math.pi)
        assert close(gpu["tc"]["pt"][i], orc["tc"]["pt"][j], 0.0)
    return (len(g), len(g_tc) - len(g))
