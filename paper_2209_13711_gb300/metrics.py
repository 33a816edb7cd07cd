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
    """
    m = match(tc, pid, seed_pid, frac)
    n_tc = len(m)
    findable = np.flatnonzero((tracks.pt >= pt_min) & (np.abs(tracks.eta) <= eta_max))
    matched = set(int(p) for p in m if p >= 0)
    found = sum(1 for p in findable if int(p) in matched)
    seen, dup = set(), 0
    for p in m:
        if p < 0:
            continue
        if p in seen:
            dup += 1
        seen.add(p)
    return dict(efficiency=found / max(1, len(findable)), fake_rate=float(np.sum(m < 0)) / max(1, n_tc),
                duplicate_rate=dup / max(1, n_tc), tcs=n_tc, findable=int(len(findable)), found=int(found))


def combine(per_event):
    """Pool the counts of several events' rates() results."""
    tcs = sum(r["tcs"] for r in per_event)
    fnd = sum(r["findable"] for r in per_event)
    return dict(efficiency=sum(r["found"] for r in per_event) / max(1, fnd),
                fake_rate=sum(r["fake_rate"] * r["tcs"] for r in per_event) / max(1, tcs),
                duplicate_rate=sum(r["duplicate_rate"] * r["tcs"] for r in per_event) / max(1, tcs),
                tcs=tcs, findable=fnd, events=len(per_event))
