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


# eta and phi0 are cut only in the cleaning, against the eta-phi distance 0.02: that is their scale
DIR_SCALE = 0.02


def close_angle(x32, x64):
    """Angles in (-pi, pi]: compared modulo 2 pi (a value within rounding of
    +-pi may be wrapped to the other end on one side), within REL of the
    value, at least of the cleaning's eta-phi scale."""
    d = (float(x32) - float(x64) + math.pi) % (2 * math.pi) - math.pi
    return abs(d) <= REL * max(abs(float(x64)), DIR_SCALE)


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
        assert close(g5["eta"][i], o5["eta"][j], DIR_SCALE) and close_angle(g5["phi0"][i], o5["phi0"][j]), ("t5 dir", t)
        assert close(g5["pt"][i], o5["pt"][j], 0.0), ("t5 pt", t)
    gp, op = gpu["pls"], orc["pls"]
    assert gp["n"] == op["n"]
    for s in range(op["n"]):
        if s in M.pls:
            continue
        assert gp["pass"][s] == op["pass"][s] and gp["sb"][s] == op["sb"][s], ("pls", s)
        assert close(gp["kappa"][s], op["kappa"][s], two_a), ("pls kappa", s)
        assert close(gp["eta"][s], op["eta"][s], DIR_SCALE) and close_angle(gp["phi0"][s], op["phi0"][s]), ("pls dir", s)
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
    """Track candidates, minus those whose cleaning decision may depend on arithmetic inside a margin.

    Cleaning order: duplicates inside a category (pT5, pT3, T5), then pT3 vs
    kept pT5, T5 vs kept pT5/pT3, unlinked pLS vs all kept. An object whose
    existence is uncertain (margin at object level, on either side) may change
    the dedup decision of same-category objects sharing a hit with it; an
    object whose keep decision is uncertain may change the decisions of
    later-category objects that share a hit, sit within dr_clean (1e-4
    widened) or use its seed.
    """
    thr2 = (cuts["dr_clean"] * (1 + 1e-4)) ** 2
    cats = ("pt5", "pt3", "t5", "pls")
    # universe: (cat, key) -> (hits, eta, phi, seed)
    U = {}
    for r, T in ((gpu, G), (orc, O)):
        for c, key in enumerate(cats):
            n = r["pls"]["n"] if key == "pls" else len(T[key])
            for i in range(n):
                h, e, p = _obj_info(r, T, c, i)
                k = i if key == "pls" else T[key][i]
                seed = i if key == "pls" else (T[key][i][0] if c < 2 else -1)
                U.setdefault((c, k), (h, e, p, seed))
    keys = list(U)
    kidx = {k: j for j, k in enumerate(keys)}
    cat = np.array([k[0] for k in keys])
    eta = np.array([U[k][1] for k in keys])
    phi = np.array([U[k][2] for k in keys])
    seed = np.array([U[k][3] for k in keys])
    hit_of = {}
    for j, k in enumerate(keys):
        for h in U[k][0]:
            hit_of.setdefault(h, []).append(j)
    exist_unc = set()
    for c, key in enumerate(cats[:3]):
        ex = getattr(M, "ex_" + key)
        for T in (G, O):
            for t in T[key]:
                if ex(t):
                    exist_unc.add(kidx[(c, t)])
    for s_ in M.pls:
        exist_unc.add(kidx[(3, s_)])
    dec = np.zeros(len(keys), bool)
    for j in exist_unc:
        dec[j] = True
        for h in U[keys[j]][0]:                       # same-category dedup partners
            for j2 in hit_of[h]:
                if cat[j2] == cat[j]:
                    dec[j2] = True
    for c1, i1, c2, i2 in orc["m_clean"]:
        k1 = (int(c1), int(i1) if c1 == 3 else O[cats[c1]][i1])
        dec[kidx[k1]] = True
        if c1 == c2:
            dec[kidx[(int(c2), O[cats[c2]][i2])]] = True
    # decisions flow downward in category order
    for c in (0, 1, 2):
        src = np.nonzero(dec & (cat == c))[0]
        if len(src) == 0:
            continue
        lower = cat > c
        for j in src:
            h, e, p, sd = U[keys[j]]
            for hh in h:
                for j2 in hit_of[hh]:
                    if cat[j2] > c:
                        dec[j2] = True
            de = eta - e
            dp = np.remainder(phi - p + np.pi, 2 * np.pi) - np.pi
            dec |= lower & ((de * de + dp * dp) < thr2)
            if sd >= 0:
                dec |= lower & (cat == 3) & (seed == sd)

    def tc_items(r):
        tc = r["tc"]
        out = {}
        for i in range(tc["n"]):
            hs = [int(h) for h in (tc["hits"][i] if "hits" in tc else [tc[f"h{j}"][i] for j in range(10)]) if h >= 0]
            out[(int(tc["type"][i]), int(tc["seed"][i]), tuple(sorted(hs)))] = i
        return out

    # map each candidate to its object through the hit set + seed
    by_sig = {}
    for j, k in enumerate(keys):
        h, e, p, sd = U[k]
        ot = tuple(sorted(x for x in h if not isinstance(x, tuple)))
        by_sig[(int(cat[j]), int(sd) if cat[j] != 2 else -1, ot)] = j
    g_tc, o_tc = tc_items(gpu), tc_items(orc)

    def ok(t):
        j = by_sig.get(t)
        return j is not None and not dec[j]

    g = {t for t in g_tc if ok(t)}
    o = {t for t in o_tc if ok(t)}
    assert g == o, f"tc: {len(g - o)} GPU-only {sorted(g - o)[:2]}, {len(o - g)} oracle-only {sorted(o - g)[:2]}"
    for t in g:
        i, j = g_tc[t], o_tc[t]
        assert close(gpu["tc"]["eta"][i], orc["tc"]["eta"][j], DIR_SCALE)
        assert close_angle(gpu["tc"]["phi0"][i], orc["tc"]["phi0"][j])
        assert close(gpu["tc"]["pt"][i], orc["tc"]["pt"][j], 0.0)
    return (len(g), len(g_tc) - len(g))
