"""Occupancy study: object counts per module and per event, the memory they
imply, and what truncating at smaller capacities costs in efficiency.

Section 3 of the paper sizes its object buffers per module and caps each
module's count at the 99.9 % or 99.99 % quantile of the occupancy seen in
simulation, which shrinks the memory about 5x for a 1-2 % efficiency loss.
This library allocates flat per-event arenas instead (objects of all modules
packed one after another, per-unit offsets and counts beside them), so its
memory follows the event's total count, not the sum of per-module maxima.
The study measures both on generated PU200 events:

* per-module occupancy of MD, LS, T3 and T5 (an LS, T3 or T5 is counted in the
  module of its innermost MD), its quantiles over (event, module) pairs, and
  the memory a per-module slot layout sized at those quantiles would take;
* per-event totals and their quantiles, and the memory of this library's
  layout at those capacities (measured with lst_device_bytes);
* the chain run with one kind's per-event capacity scaled below its largest
  observed total: counted drops, efficiency (also without bare-pLS TCs, which
  match their seed's particle whatever the outer tracker found), fake and
  duplicate rates, and the memory saved.

    python -m paper_2209_13711_gb300.occupancy --events 64 --batch 16
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

KINDS = ("md", "ls", "t3", "t5")
CAP_FIELD = {"md": "md_per_event", "ls": "ls_per_event", "t3": "t3_per_event", "t5": "t5_per_event"}


def module_occupancy(obj, n_mod):
    """Objects per module (module of the innermost MD) for one event's objects."""
    mod = np.asarray(obj["md"]["mod"], np.int64) % n_mod
    ls_mod = mod[np.asarray(obj["ls"]["md_in"], np.int64)]
    t3_mod = ls_mod[np.asarray(obj["t3"]["ls_in"], np.int64)]
    t5_mod = t3_mod[np.asarray(obj["t5"]["t3_in"], np.int64)]
    return {k: np.bincount(m, minlength=n_mod) for k, m in zip(KINDS, (mod, ls_mod, t3_mod, t5_mod))}


def slot_bytes(occ, bytes_per, quantiles):
    """Memory per event of per-module slots: every module gets the same cap per
    kind, the given quantile of the (event, module) occupancy."""
    out = {}
    for q in quantiles:
        caps = {k: int(np.ceil(np.percentile(occ[k], q))) for k in KINDS}
        n_mod = occ["md"].shape[1]
        out[f"q{q:g}"] = {"caps_per_module": caps,
                          "bytes_per_event": int(sum(n_mod * caps[k] * bytes_per[k] for k in KINDS)),
                          "modules_over_cap_frac": {k: float((occ[k] > caps[k]).mean()) for k in KINDS}}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=64)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--scales", type=float, nargs="+", default=[0.9, 0.75, 0.5])
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from synth import events as E, geometry as G, maps as M
    from synth.config import DEFAULT_CUTS

    from . import lst as L
    from . import metrics as MT
    geom = G.make_geometry(barrel_only=False)
    maps = M.load_maps(geom)
    n_mod = geom.n_mod
    evs = [E.pu200_event(50000 + i, geom) for i in range(args.events)]
    batches = [evs[i:i + args.batch] for i in range(0, len(evs), args.batch)]

    # ---- occupancy at the default capacities (no drops) -------------------
    ctx = L.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=L.default_capacity(args.batch))
    occ = {k: [] for k in KINDS}
    totals = {k: [] for k in KINDS}
    base_rates = []
    for b in batches:
        ctx.run(b)
        for j, ev in enumerate(b):
            obj = {k: ctx.objects(k, j) for k in KINDS}
            st = ctx.stats(j)
            assert all(v == 0 for v in st["dropped"].values()), st
            for k, v in module_occupancy(obj, n_mod).items():
                occ[k].append(v)
                totals[k].append(int(obj[k]["n"]))
            base_rates.append(MT.rates(ctx.track_candidates(j), ev.pid, ev.seed_pid, ev.tracks))
    ctx.close()
    occ = {k: np.stack(v) for k, v in occ.items()}
    totals = {k: np.asarray(v) for k, v in totals.items()}

    # ---- bytes per object of this library's layout (slope of device bytes) -
    def dev_bytes(**cap):
        c = L.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=L.default_capacity(1, **cap))
        try:
            return c.device_bytes
        finally:
            c.close()
    base = dev_bytes()
    dflt = L.default_capacity(1)
    bytes_per = {}
    for k in KINDS:
        d = 65536
        bytes_per[k] = (dev_bytes(**{CAP_FIELD[k]: getattr(dflt, CAP_FIELD[k]) + d}) - base) / d

    out = {"events": args.events, "n_mod": n_mod, "bytes_per_object": {k: round(v, 2) for k, v in bytes_per.items()},
           "per_event_total": {k: {"mean": float(v.mean()), "max": int(v.max()),
                                   "q99.9": float(np.percentile(v, 99.9))} for k, v in totals.items()},
           "per_module": {k: {"mean": float(v.mean()), "q99.9": float(np.percentile(v, 99.9)),
                              "q99.99": float(np.percentile(v, 99.99)), "max": int(v.max())}
                          for k, v in occ.items()},
           "slot_layout": slot_bytes(occ, bytes_per, (100, 99.99, 99.9)),
           "flat_layout_bytes_per_event_at_max_totals": int(sum(totals[k].max() * bytes_per[k] for k in KINDS)),
           "baseline": MT.combine(base_rates)}

    # ---- truncation: one kind's per-event capacity scaled below its largest
    # total at a time (the others at their defaults) --------------------------
    def run_with(caps):
        ctx = L.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=L.default_capacity(args.batch, **caps))
        dropped = {k: 0 for k in KINDS}
        rates = []
        try:
            for b in batches:
                ctx.run(b)
                for j, ev in enumerate(b):
                    st = ctx.stats(j)
                    for k in KINDS:
                        dropped[k] += st["dropped"][k]
                    rates.append(MT.rates(ctx.track_candidates(j), ev.pid, ev.seed_pid, ev.tracks))
        finally:
            ctx.close()
        c = MT.combine(rates)
        return {"dropped_per_event": {k: v / args.events for k, v in dropped.items()},
                "efficiency": round(c["efficiency"], 4), "efficiency_ot": round(c["efficiency_ot"], 4),
                "fake_rate": round(c["fake_rate"], 4), "duplicate_rate": round(c["duplicate_rate"], 4)}

    trunc = []
    for k in KINDS:
        for s in args.scales:
            cap = max(1, int(s * totals[k].max()))
            r = run_with({CAP_FIELD[k]: cap})
            r.update(kind=k, scale_of_max_total=s, cap_per_event=cap,
                     arena_bytes_saved_per_event=int((totals[k].max() - cap) * bytes_per[k]))
            trunc.append(r)
    out["truncation"] = trunc
    print(json.dumps(out))


if __name__ == "__main__":
    main()
