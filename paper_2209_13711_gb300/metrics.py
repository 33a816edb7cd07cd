"""Track-candidate efficiency, fake rate and duplicate rate on generator truth.

These are the figures of merit of Section 2.2 of the paper (efficiency vs pT
and eta, fake and duplicate rates), computed here on the synthetic events'
truth instead of CMS simulation:

* a TC is matched to a generated particle when at least `frac` of its hits
  (outer-tracker hits, plus the three pixel hits of its seed, if any) come
  from that particle; otherwise it is a fake;
* efficiency: the fraction of findable particles (pT and |eta| in range) that
  at least one TC is matched to;
* duplicate rate: the fraction of TCs matched to a particle that an earlier
  TC is already matched to.

`candidate_tests` counts the combinatorics of one event: how many candidates
each stage's kernel puts to its predicates (Section 2.1: every hit pair of a
module, every MD pair of connected modules, every pair of objects sharing an
MD, every passing pLS against the objects of its superbin's modules).
"""
from __future__ import annotations

import numpy as np


def match(tc, pid, seed_pid, frac=0.75):
    """Particle matched to each TC (-1: fake). tc: dict with hits [n, 10]
    (event-local hit indices, -1 padded) and seed [n] (-1: none)."""
    n = int(tc["n"])
    out = np.full(n, -1, np.int64)
    for i in range(n):
        h = tc["hits"][i]
        p = list(pid[h[h >= 0]])
        s = int(tc["seed"][i])
        if s >= 0:
            p += [int(seed_pid[s])] * 3
        if not p:
            continue
        vals, cnt = np.unique(np.asarray(p), return_counts=True)
        k = int(np.argmax(np.where(vals >= 0, cnt, -1)))
        if vals[k] >= 0 and cnt[k] >= frac * len(p):
            out[i] = vals[k]
    return out


def rates(tc, pid, seed_pid, tracks, pt_min=1.0, eta_max=2.4, frac=0.75):
    """Efficiency, fake and duplicate rates of one event's TCs.

    tracks: the generated particles (pt, eta arrays indexed by particle id).
    When tc has a "type" column, efficiency_ot also counts the particles
    found by TCs with outer-tracker objects only (pT5, pT3, T5: not a bare
    pLS, which matches its seed's particle by construction).
    """
    m = match(tc, pid, seed_pid, frac)
    n_tc = len(m)
    findable = np.flatnonzero((tracks.pt >= pt_min) & (np.abs(tracks.eta) <= eta_max))
    matched = set(int(p) for p in m if p >= 0)
    found = sum(1 for p in findable if int(p) in matched)
    found_ot = found
    if "type" in tc:
        ot = np.asarray(tc["type"]) != 3
        matched_ot = set(int(p) for p in m[ot] if p >= 0)
        found_ot = sum(1 for p in findable if int(p) in matched_ot)
    seen, dup = set(), 0
    for p in m:
        if p < 0:
            continue
        if p in seen:
            dup += 1
        seen.add(p)
    return dict(efficiency=found / max(1, len(findable)), fake_rate=float(np.sum(m < 0)) / max(1, n_tc),
                duplicate_rate=dup / max(1, n_tc), tcs=n_tc, findable=int(len(findable)), found=int(found),
                efficiency_ot=found_ot / max(1, len(findable)), found_ot=int(found_ot))


PT_EDGES = (0.5, 0.8, 1.0, 1.5, 2.0, 3.0, 5.0, 10.0, 20.0, 50.0, 100.0)
ETA_EDGES = tuple(round(-2.4 + 0.4 * i, 1) for i in range(13))
TC_TYPES = ("pT5", "pT3", "T5", "pLS")


def curves(per_event, pt_min=1.0, eta_max=2.4, frac=0.75, pt_edges=PT_EDGES, eta_edges=ETA_EDGES):
    """Binned figures of merit over several events (Section 2.2's plots).

    per_event: (tc, pid, seed_pid, tracks) per event; tc as in rates(), plus
    its "type" (0 pT5, 1 pT3, 2 T5, 3 pLS), "pt" and "eta".
      efficiency vs generated pT (|eta| <= eta_max) and vs generated eta
        (pT >= pt_min): found / findable per bin;
      fake and duplicate rates vs the TC's own pT and eta: per bin of TCs;
      by TC type: TC count, fake and duplicate rates.
    Each bin holds [numerator, denominator]; bins are [lo, hi)."""
    pe, ee = np.asarray(pt_edges, float), np.asarray(eta_edges, float)
    z = lambda e: np.zeros((len(e) - 1, 2), np.int64)
    eff_pt, eff_eta, fake_pt, fake_eta, dup_pt, dup_eta = z(pe), z(ee), z(pe), z(ee), z(pe), z(ee)
    by_type = {t: [0, 0, 0] for t in TC_TYPES}        # TCs, fakes, duplicates

    def add(h, edges, x, num):
        b = np.searchsorted(edges, x, side="right") - 1
        ok = (b >= 0) & (b < len(edges) - 1)
        np.add.at(h[:, 1], b[ok], 1)
        np.add.at(h[:, 0], b[ok], np.asarray(num, np.int64)[ok])

    for tc, pid, seed_pid, tracks in per_event:
        m = match(tc, pid, seed_pid, frac)
        found = np.zeros(len(tracks.pt), bool)
        found[m[m >= 0]] = True
        gpt, geta = np.asarray(tracks.pt, float), np.asarray(tracks.eta, float)
        sel = np.abs(geta) <= eta_max
        add(eff_pt, pe, gpt[sel], found[sel])
        sel = gpt >= pt_min
        add(eff_eta, ee, geta[sel], found[sel])
        seen, dup = set(), np.zeros(len(m), bool)
        for i, p in enumerate(m):
            if p >= 0:
                dup[i] = p in seen
                seen.add(int(p))
        fake = m < 0
        tpt, teta = np.asarray(tc["pt"], float), np.asarray(tc["eta"], float)
        add(fake_pt, pe, tpt, fake)
        add(fake_eta, ee, teta, fake)
        add(dup_pt, pe, tpt, dup)
        add(dup_eta, ee, teta, dup)
        for t, name in enumerate(TC_TYPES):
            k = np.asarray(tc["type"]) == t
            by_type[name][0] += int(k.sum())
            by_type[name][1] += int((k & fake).sum())
            by_type[name][2] += int((k & dup).sum())
    L = lambda h: h.tolist()
    return dict(pt_edges=list(pe), eta_edges=list(ee), efficiency_vs_pt=L(eff_pt), efficiency_vs_eta=L(eff_eta),
                fake_vs_pt=L(fake_pt), fake_vs_eta=L(fake_eta), duplicate_vs_pt=L(dup_pt),
                duplicate_vs_eta=L(dup_eta),
                by_type={t: dict(tcs=v[0], fake_rate=v[1] / max(1, v[0]), duplicate_rate=v[2] / max(1, v[0]))
                         for t, v in by_type.items()})


D0_EDGES = (0.0, 0.25, 0.5, 1.0, 1.5, 2.0, 2.5, 3.6)


def efficiency_vs_d0(per_event, edges=D0_EDGES, pt_min=1.0, eta_max=2.4, frac=0.75):
    """Efficiency against the generated transverse impact parameter d0 (cm), overall and by the type of the
    TC that finds the particle (the displaced-track study of Section 2.2: the T5 has no d0 cut).

    per_event: (tc, pid, seed_pid, tracks) per event, tracks with a d0 property. Per d0 bin: findable
    particles (pT >= pt_min, |eta| <= eta_max), found by any TC, and found by a TC of each type (a particle
    found by TCs of several types counts for each)."""
    e = np.asarray(edges, float)
    nb = len(e) - 1
    findable = np.zeros(nb, np.int64)
    found = np.zeros(nb, np.int64)
    by_type = {t: np.zeros(nb, np.int64) for t in TC_TYPES}
    for tc, pid, seed_pid, tracks in per_event:
        m = match(tc, pid, seed_pid, frac)
        d0 = np.asarray(tracks.d0, float)
        ok = (np.asarray(tracks.pt) >= pt_min) & (np.abs(np.asarray(tracks.eta)) <= eta_max)
        b = np.searchsorted(e, d0, side="right") - 1
        ok &= (b >= 0) & (b < nb)
        any_found = np.zeros(len(d0), bool)
        any_found[m[m >= 0]] = True
        np.add.at(findable, b[ok], 1)
        np.add.at(found, b[ok], any_found[ok].astype(np.int64))
        types = np.asarray(tc["type"])
        for t, name in enumerate(TC_TYPES):
            f = np.zeros(len(d0), bool)
            sel = (types == t) & (m >= 0)
            f[m[sel]] = True
            np.add.at(by_type[name], b[ok], f[ok].astype(np.int64))
    eff = lambda num: [round(float(a) / max(1, int(d)), 4) for a, d in zip(num, findable)]
    return dict(d0_edges=list(e), findable=findable.tolist(), efficiency=eff(found),
                efficiency_by_type={t: eff(v) for t, v in by_type.items()})


def combine(per_event):
    """Pool the counts of several events' rates() results."""
    tcs = sum(r["tcs"] for r in per_event)
    fnd = sum(r["findable"] for r in per_event)
    return dict(efficiency=sum(r["found"] for r in per_event) / max(1, fnd),
                efficiency_ot=sum(r.get("found_ot", r["found"]) for r in per_event) / max(1, fnd),
                fake_rate=sum(r["fake_rate"] * r["tcs"] for r in per_event) / max(1, tcs),
                duplicate_rate=sum(r["duplicate_rate"] * r["tcs"] for r in per_event) / max(1, tcs),
                tcs=tcs, findable=fnd, events=len(per_event))


def _csr_sums(off, tgt, w):
    """Per row r of a CSR map: sum of w[t] over its targets t."""
    cs = np.concatenate([[0], np.cumsum(w[np.asarray(tgt, np.int64)], dtype=np.int64)])
    off = np.asarray(off, np.int64)
    return cs[off[1:]] - cs[off[:-1]]


def candidate_tests(obj, hit_module, hit_side, conn_off, conn_tgt, sb_off, sb_tgt, n_mod):
    """Candidates put to each stage's predicates in one event.

    obj: the event's objects by kind ("md", "ls", "t3", "t5", "pls"), with the
    columns of lst_get_objects; hit_module / hit_side: the event's hits;
    conn_*: module connectivity CSR; sb_*: superbin -> modules CSR.
      md:  lower x upper hits of each module;
      ls:  each MD x the MDs of the modules its module connects to;
      t3:  each LS x the LS whose inner MD is its outer MD;
      t5:  each T3 x the T3 whose inner MD is its outer MD;
      pt5 / pt3: each passing pLS x the T5 / T3 whose inner MD lies in a module
           of the pLS's superbin.
    """
    hit_module = np.asarray(hit_module, np.int64)
    side = np.asarray(hit_side)
    lo = np.bincount(hit_module[side == 0], minlength=n_mod).astype(np.int64)
    up = np.bincount(hit_module[side == 1], minlength=n_mod).astype(np.int64)
    md, ls, t3, t5, pls = obj["md"], obj["ls"], obj["t3"], obj["t5"], obj["pls"]
    n_md = int(md["n"])
    md_mod = np.asarray(md["mod"], np.int64) % n_mod
    md_per_mod = np.bincount(md_mod, minlength=n_mod).astype(np.int64)
    ls_in, ls_out = np.asarray(ls["md_in"], np.int64), np.asarray(ls["md_out"], np.int64)
    ls_from = np.bincount(ls_in, minlength=n_md).astype(np.int64)
    t3_inner = ls_in[np.asarray(t3["ls_in"], np.int64)]
    t3_outer = ls_out[np.asarray(t3["ls_out"], np.int64)]
    t3_from = np.bincount(t3_inner, minlength=n_md).astype(np.int64)
    t5_inner = t3_inner[np.asarray(t5["t3_in"], np.int64)]
    t5_from = np.bincount(t5_inner, minlength=n_md).astype(np.int64)
    sb = np.asarray(pls["sb"], np.int64)[(np.asarray(pls["pass"]) != 0) & (np.asarray(pls["sb"]) >= 0)]

    def per_sb(from_md):
        per_mod = np.bincount(md_mod, weights=from_md, minlength=n_mod).astype(np.int64)
        return _csr_sums(sb_off, sb_tgt, per_mod)

    return {
        "md": int((lo * up).sum()),
        "ls": int((md_per_mod * _csr_sums(conn_off, conn_tgt, md_per_mod)).sum()),
        "t3": int(ls_from[ls_out].sum()),
        "t5": int(t3_from[t3_outer].sum()),
        "pt5": int(per_sb(t5_from)[sb].sum()),
        "pt3": int(per_sb(t3_from)[sb].sum()),
    }
