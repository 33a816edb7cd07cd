"""Run the chain on synthetic events and print what it built.

    python -m paper_2209_13711_gb300.run --events 8 --pileup 200 --repeat 2
    python -m paper_2209_13711_gb300.run --events 64 --pileup-range 50 200 --autotune --profile

Events come from the seeded generator (`synth.events`, full barrel+endcap
geometry): --pileup 200 gives the PU200 event (8000 tracks + 12 jet-like
tracks); other values give 40 tracks per pileup unit. The batch runs --repeat
times through one context (the first run captures the graph); the output is
one JSON line with per-event object counts, the device time of the last run
and, with --profile, the per-stage device times of one more run.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=1)
    ap.add_argument("--pileup", type=float, default=200.0)
    ap.add_argument("--pileup-range", type=float, nargs=2, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--profile", action="store_true")
    ap.add_argument("--t3-net", default=None, help="learned triplet selection saved by train --kind t3")
    ap.add_argument("--t5-net", default=None, help="network-scored T5 selection saved by train --kind t5")
    ap.add_argument("--fp64-fit", action="store_true", help="refine fits in FP64 instead of float-float")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    from synth import events as E, geometry as G, maps as M
    from synth.config import DEFAULT_CUTS

    from . import lst as L
    geom = G.make_geometry(barrel_only=False)
    maps = M.load_maps(geom)
    rng = np.random.default_rng(args.seed)
    evs = []
    for i in range(args.events):
        if args.pileup_range:
            evs.append(E.pileup_event(float(rng.uniform(*args.pileup_range)), args.seed * 1000 + i, geom))
        elif args.pileup == 200.0:
            evs.append(E.pu200_event(args.seed * 1000 + i, geom))
        else:
            evs.append(E.pileup_event(args.pileup, args.seed * 1000 + i, geom))
    ctx = L.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=L.default_capacity(args.events))
    if args.fp64_fit:
        ctx.set_fp64_fit(True)
    nets = []
    if args.t3_net:
        z = np.load(args.t3_net)
        nets.append(L.Mlp(params=z["params"]))
        ctx.set_t3_selection(nets[-1], threshold=float(z["threshold"]))
    if args.t5_net:
        z = np.load(args.t5_net)
        nets.append(L.Mlp(params=z["params"]))
        ctx.set_t5_selection(nets[-1], threshold=float(z["threshold"]),
                             prefilter_scale=float(z["prefilter_scale"]) if "prefilter_scale" in z.files else 1.0)
    b = L.pack_events(evs)
    bd = {k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in b.items()}
    st = torch.cuda.current_stream()
    out = {"events": args.events, "hits": int(b["hit_off"][-1]), "seeds": int(b["seed_off"][-1])}
    if args.autotune:
        before, after = ctx.autotune(bd, reps=2, stream=st.cuda_stream)
        out["autotune_stage_ms"] = [round(before, 4), round(after, 4)]
    ms = 0.0
    for _ in range(max(1, args.repeat)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_packed(bd, stream=st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    out["last_run_ms"] = round(ms, 4)
    out["events_per_s"] = round(args.events / (ms / 1e3), 2)
    counts = [ctx.stats(e) for e in range(args.events)]
    out["objects"] = {k: int(sum(c["counts"][k] for c in counts)) for k in counts[0]["counts"]}
    out["dropped"] = {k: int(sum(c["dropped"][k] for c in counts)) for k in counts[0]["dropped"]}
    if args.profile:
        ctx.set_profiling(True)
        ctx.run_packed(bd, stream=st.cuda_stream)
        out["stage_ms"] = {n: round(t, 4) for n, t in ctx.kernel_times()}
        ctx.set_profiling(False)
    ctx.close()
    for m in nets:
        m.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
