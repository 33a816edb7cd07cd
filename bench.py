#!/usr/bin/env python
"""Benchmark: PU200 events/s of the Segment Linking chain on GB300.

A step is one pass of the whole chain (binning, MD, LS, T3, T5, pLS, pT5,
pT3, cross-cleaning, track candidates) over one synthetic PU200 event
(8000 tracks + 12 jet-like tracks, 13260-module geometry). The device-timed
`value` has the event's hits already in HBM; `e2e` goes through the C ABI
from pinned host buffers and includes the host-to-device copy of the hits
and seeds and the device-to-host read of the track candidates. The L2 cache
is flushed (a 256 MiB write) between timed steps, outside the timed spans.

Multi-GPU: events are independent, so N ranks run N replicas on their own
events (weak scaling, no collective on the data path); the time is the max
over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PU200 events/sec"
UNIT = "events/s"
WORKLOAD = ("PU200 ttbar-like single event: 8000 prompt tracks (beamspot sigma_z 5 cm, dN/dpT ~ pT^-3 above "
            "0.5 GeV, |eta| < 2.4) + 12 jet-like tracks, 2% noise hits, one 3-hit pixel seed per track; "
            "13260-module barrel+endcap geometry")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


EVENT_POOL = 32


def event_seeds(rank, n):
    """Generator seeds of rank `rank`'s n events (disjoint across ranks)."""
    return [rank * 100000 + i for i in range(n)]


def max_over_ranks(values, ws):
    """Element-wise maximum of per-rank timings (identity on one rank). Uses the
    default process group: NCCL with CUDA tensors, gloo with CPU tensors."""
    import torch
    if ws <= 1:
        return [float(v) for v in values]
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(ws, steps, seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return ws * steps / seconds


def measured_counters(kernel, workload="pu200"):
    """Per-launch ncu counters of `kernel` from the committed profile
    summaries (their machine-readable blocks), merged; a block whose kernel
    sources changed since its capture is skipped."""
    import glob
    import hashlib
    out = {}
    for fn in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        kv = {}
        with open(fn) as f:
            for line in f:
                if ":" in line and not line.startswith(("|", "#", "`", " ", "*")):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel") != kernel or "sources_sha256" not in kv or kv.get("workload", "pu200") != workload:
            continue
        h = hashlib.sha256()
        try:
            for src in kv.get("sources", "").split():
                with open(os.path.join(ROOT, src), "rb") as f:
                    h.update(f.read())
        except OSError:
            continue
        if h.hexdigest() != kv["sources_sha256"]:
            continue
        for k, v in kv.items():
            if k.endswith("_per_launch"):
                out[k] = float(v)
    return out


def measured_traffic(kernel, workload="pu200"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of the
    workload (pu200: one PU200 event; pu200xN: N of them in one batch), or None
    when there is none or the kernel's sources changed since it was taken."""
    v = measured_counters(kernel, workload).get("dram_bytes_per_launch")
    return None if v is None else int(v)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def algorithmic_bytes(kernel, st, n_hits, n_seeds, n_mod):
    """Compulsory bytes of one launch: its inputs read once and outputs written once (from object counts;
    for a batch, st holds the counts summed over its events and n_mod the modules times the events)."""
    c = st["counts"]
    md, ls, t3, t5, pls, p5, p3 = (c[k] for k in ("md", "ls", "t3", "t5", "pls", "pt5", "pt3"))
    table = {
        "md": n_hits * 16 + n_mod * 2 * 4 + md * 44 + n_mod * 8,          # sorted hits in, MDs out
        "ls": md * 24 + n_mod * 8 + ls * 12 + md * 8,                     # MD anchors+stubs in, LS out
        "t3": ls * 8 + md * 24 + t3 * 20 + md * 8,                        # LS + MDs in, T3 out
        "t5": t3 * 16 + ls * 4 + md * 16 + t5 * 56 + md * 8,              # T3 + MDs in, T5 out
        "pt5": n_seeds * 48 + md * 16 + t5 * 16 + p5 * 28,
        "pt3": n_seeds * 48 + md * 16 + t3 * 8 + p3 * 28,
    }
    return table.get(kernel)


def run_ours(args):
    import numpy as np
    import torch

    import paper_2209_13711_gb300 as P
    from paper_2209_13711_gb300.metrics import candidate_tests
    from synth import events as E, geometry as G, maps as M
    from synth.config import DEFAULT_CUTS

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    geom = G.make_geometry(barrel_only=False)
    maps = M.load_maps(geom)
    ctx = P.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=P.default_capacity(1), device=local)
    n_ev = args.steps + args.warmup
    pool = min(n_ev, EVENT_POOL)
    # rank r processes its own events (disjoint seeds); steps cycle over a pool of distinct events
    events = [E.pu200_event(s, geom) for s in event_seeds(rank, pool)]
    packed = [P.pack_events([e]) for e in events]
    pick = lambda i: i % pool
    dev = [{k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in b.items()}
           for b in packed]
    pinned = [{k: (torch.from_numpy(v).pin_memory() if k not in ("hit_off", "seed_off") else v)
               for k, v in b.items()} for b in packed]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- the device's FP32 / FP64 / atomic rates (calibration, untimed) --
    peaks = P.measure_peaks(local)
    # ---- launch shapes tuned on a warm-up event (setup, untimed) ---------
    tune = autotune(ctx, dev[0], st)
    # ---- device-timed: inputs resident in HBM ---------------------------
    for i in range(args.warmup):
        ctx.run_packed(dev[pick(i)], stream=st.cuda_stream)
    barrier()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    with ClockSampler(local) as clk:
        barrier()
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev0[i].record(st)
            ctx.run_packed(dev[pick(args.warmup + i)], stream=st.cuda_stream)
            ev1[i].record(st)
            launches += ctx.launch_count
        barrier()
    dev_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    stats0 = ctx.stats(0)
    # ---- end to end through the C ABI from pinned host memory -----------
    e2e_s = 0.0
    h2d = d2h = 0
    # the result lands in pinned host memory too (a direct copy, not one staged through a driver buffer)
    rec_buf = torch.empty(ctx.capacity.tc_per_event * P.lst.TC_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    records = rec_buf.numpy().view(P.lst.TC_DTYPE)
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        b = pinned[pick(args.warmup + i)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.run_packed(b, stream=st.cuda_stream)
        off, rec = ctx.batch_track_candidates(out=records)
        t1 = time.perf_counter()
        e2e_s += t1 - t0
        h2d += sum(int(v.numel() * v.element_size()) for k, v in b.items() if k not in ("hit_off", "seed_off"))
        h2d += 8 * len(b["hit_off"])
        d2h += off.nbytes + rec.nbytes
    # ---- per-kernel device times (profiling pass, same workload) --------
    ctx.set_profiling(True)
    per_kernel, tests = {}, []
    n_prof = min(args.steps, 5)
    for i in range(n_prof):
        flush.fill_(i & 0xff)
        ctx.run_packed(dev[pick(args.warmup + i)], stream=st.cuda_stream)
        for name, ms in ctx.kernel_times():
            per_kernel.setdefault(name, []).append(ms)
        e = events[pick(args.warmup + i)]
        objs = {k: ctx.objects(k, 0) for k in ("md", "ls", "t3", "t5", "pls")}
        tests.append(candidate_tests(objs, e.module, e.side, *maps, geom.n_mod))
    ctx.set_profiling(False)
    kavg = {k: sum(v) / len(v) for k, v in per_kernel.items()}
    tests_ev = {k: sum(t[k] for t in tests) / n_prof for k in tests[0]}
    top = max(kavg, key=kavg.get)
    # timing across ranks
    dev_ms, e2e_s = max_over_ranks([dev_ms, e2e_s], ws)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    value = whole_job_rate(ws, args.steps, dev_ms / 1e3)
    hbm_peak, peak_kind = _peaks()
    last = events[pick(args.warmup + args.steps - 1)]
    b_alg = algorithmic_bytes(top, stats0, len(last.x), len(last.seeds), geom.n_mod)
    roof = None
    if b_alg is not None:
        achieved = b_alg / (kavg[top] / 1e3) / 1e9
        roof = {"kernel": top, "bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 5), "traffic": measured_traffic(top), "peak_source": peak_kind,
                "algorithmic_bytes": int(b_alg), "kernel_ms": round(kavg[top], 4)}
    cnt = measured_counters(top)
    alu = atomics = None
    if "fp32_flop_per_launch" in cnt:
        a = cnt["fp32_flop_per_launch"] / (kavg[top] / 1e3) / 1e12
        alu = {"kernel": top, "bound": "alu", "achieved": round(a, 3), "peak": round(peaks["fp32_tflops"], 2),
               "unit": "TFLOP/s", "frac": round(a / peaks["fp32_tflops"], 4),
               "peak_source": "measured (lst_measure_peaks FFMA probe)",
               "fp32_flop_per_launch": int(cnt["fp32_flop_per_launch"]),
               "fp64_flop_per_launch": int(cnt.get("fp64_flop_per_launch", 0))}
    if "atom_inst_per_launch" in cnt:
        n_at = cnt["atom_inst_per_launch"] + cnt.get("red_inst_per_launch", 0.0)
        a = n_at / (kavg[top] / 1e3) / 1e9
        atomics = {"kernel": top, "achieved": round(a, 4), "peak": round(peaks["atom_warp_gops"], 3),
                   "unit": "G atomic instructions/s", "frac": round(a / peaks["atom_warp_gops"], 5),
                   "peak_source": "measured (lst_measure_peaks, single-lane atomics on distinct lines)",
                   "atomic_inst_per_launch": int(n_at)}
    stage_of = {"md": "md", "ls": "ls", "t3": "t3", "t5": "t5", "pt5": "pt5", "pt3": "pt3"}
    cand = {"per_event": {k: int(v) for k, v in tests_ev.items()},
            "per_s": {k: round(v / (kavg[stage_of[k]] / 1e3), 1) for k, v in tests_ev.items()
                      if kavg.get(stage_of[k])},
            "chain_per_s": round(sum(tests_ev.values()) / (dev_ms / args.steps / 1e3), 1),
            "definition": "candidates put to each stage's predicates (metrics.candidate_tests), mean over "
                          f"the {n_prof} profiled events; per_s divides by the stage's search-kernel time"}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_step": 1, "path": "plain, one event per launch sequence",
                   "events": f"{pool} distinct PU200 events per rank, cycled over the {args.steps} steps",
                   "l2": "flushed between steps (256 MiB write, outside the timed spans)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "e2e": {"value": round(whole_job_rate(ws, args.steps, e2e_s), 2), "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": launches,
        "autotune": tune,
        "clocks": clk.summary(),
        "roofline": roof,
        "alu_roofline": alu,
        "atomics": atomics,
        "candidate_tests": cand,
        "peaks_probe": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in peaks.items() if k != "ms"},
        "kernel_ms": {k: round(v, 4) for k, v in sorted(kavg.items(), key=lambda kv: -kv[1])},
        "objects_per_event": stats0["counts"],
        "dropped_per_event": stats0["dropped"],
    }
    out["physics"] = measure_physics(P, ctx, dev, events, st)
    out["physics"]["d0_scan"] = measure_d0_scan(P, E, geom, maps, DEFAULT_CUTS, st)
    out["streams"] = measure_streams(P, geom, maps, DEFAULT_CUTS, dev, st)
    out["batched"] = measure_batched(P, E, geom, maps, DEFAULT_CUTS, flush, st, steps=max(2, min(args.steps, 5)))
    out["batched_pu200"] = measure_batched_pu200(P, E, geom, maps, DEFAULT_CUTS, flush, st,
                                                 steps=max(2, min(args.steps, 5)), events=events)
    out["compact_storage"] = measure_compact(P, geom, maps, DEFAULT_CUTS, flush, st, events)
    out["fit_precision"] = measure_fit_precision(P, geom, maps, DEFAULT_CUTS, flush, st, events)
    out["mlp"] = measure_mlp(P, E, geom, maps, DEFAULT_CUTS, flush, st, dev)
    out["mlp_t3"] = measure_mlp_t3(P, E, geom, maps, DEFAULT_CUTS, flush, st, dev, events)
    out["serving"] = measure_serving(E, geom, maps, DEFAULT_CUTS)
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


def autotune(ctx, batch, st, reps=3):
    """Tune every stage's launch shape on the batch; report what changed."""
    default = {c["name"]: (c["blocks_per_sm"], c["block"]) for c in ctx.launch_config()}
    before, after = ctx.autotune(batch, reps=reps, stream=st.cuda_stream)
    now = {c["name"]: (c["blocks_per_sm"], c["block"]) for c in ctx.launch_config()}
    changed = {k: {"blocks_per_sm": v[0], "block": v[1]} for k, v in now.items() if v != default[k]}
    return {"stage_sum_ms_default": round(before, 4), "stage_sum_ms_tuned": round(after, 4), "changed": changed}


def measure_physics(P, ctx, dev, events, st, n=16):
    """Efficiency, fake and duplicate rates of the device TCs on generator truth
    (Section 2.2's figures of merit), pooled over the first n pool events, and
    the same binned in pT and eta and split by TC type."""
    from paper_2209_13711_gb300 import metrics as MT
    out = {}
    res = {1.0: [], 5.0: []}
    per_event = []
    for i in range(min(n, len(events))):
        ctx.run_packed(dev[i], stream=st.cuda_stream)
        off, rec = ctx.batch_track_candidates()
        tc = P.lst.tc_dict(rec[off[0]:off[1]])
        ev = events[i]
        for ptm in res:
            res[ptm].append(MT.rates(tc, ev.pid, ev.seed_pid, ev.tracks, pt_min=ptm, eta_max=2.4))
        per_event.append((tc, ev.pid, ev.seed_pid, ev.tracks))
    for ptm, r in res.items():
        c = MT.combine(r)
        out[f"pt_ge_{ptm:g}GeV"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in c.items()}
    cv = MT.curves(per_event)
    for t in cv["by_type"].values():
        t["fake_rate"], t["duplicate_rate"] = round(t["fake_rate"], 4), round(t["duplicate_rate"], 4)
    out["curves"] = cv
    out["definition"] = ("TC matched when >= 75% of its hits (seed pixel hits included) come from one particle; "
                         "findable: generated pT above the bin edge and |eta| <= 2.4")
    return out


def measure_streams(P, geom, maps, cuts, dev, st, n_events=96, streams=(1, 2, 4, 8)):
    """The paper's multi-stream comparison (Section 2.2: 1 vs 8 CUDA streams):
    one PU200 event per launch sequence, with n contexts each on its own
    stream running different events at once, L2 not flushed (the streams
    overlap). events/s = events / wall time on the device."""
    import torch
    out = {}
    ctxs = [P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(1)) for _ in range(max(streams))]
    sts = [torch.cuda.Stream() for _ in ctxs]
    for c, s in zip(ctxs, sts):                      # capture every context's graph
        c.run_packed(dev[0], stream=s.cuda_stream)
    torch.cuda.synchronize()
    for n in streams:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for s in sts[:n]:
            s.wait_event(e0)
        for i in range(n_events):
            ctxs[i % n].run_packed(dev[i % len(dev)], stream=sts[i % n].cuda_stream)
        for s in sts[:n]:
            st.wait_stream(s)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"{n}_streams"] = round(n_events / (ms / 1e3), 1)
    for c in ctxs:
        c.close()
    out["unit"] = "events/s"
    out["events"] = n_events
    return out


def measure_batched(P, E, geom, maps, cuts, flush, st, steps, n_batch=64):
    """64 events of uneven pileup (uniform in 50-200, 40 tracks per unit) in one
    graph launch, against the same events one per launch."""
    import numpy as np
    import torch
    rng = np.random.default_rng(777)
    pus = rng.uniform(50.0, 200.0, n_batch)
    events = [E.pileup_event(float(pu), 5000 + i, geom) for i, pu in enumerate(pus)]
    ctx = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(n_batch))
    b = P.pack_events(events)
    bd = {k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in b.items()}
    tune = autotune(ctx, bd, st, reps=2)
    for _ in range(2):
        ctx.run_packed(bd, stream=st.cuda_stream)
    torch.cuda.synchronize()
    ms = 0.0
    for i in range(steps):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_packed(bd, stream=st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    dropped = sum(sum(ctx.stats(e)["dropped"].values()) for e in range(n_batch))
    ctx.close()
    # the same events, one per launch sequence
    ctx1 = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(1))
    singles = [P.pack_events([ev]) for ev in events]
    singles = [{k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in x.items()}
               for x in singles]
    ctx1.run_packed(singles[0], stream=st.cuda_stream)
    torch.cuda.synchronize()
    ms1 = 0.0
    for x in singles:
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx1.run_packed(x, stream=st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms1 += e0.elapsed_time(e1)
    ctx1.close()
    return {"value": round(n_batch * steps / (ms / 1e3), 2), "unit": "events/s", "events_per_batch": n_batch,
            "ms_per_batch": round(ms / steps, 3), "pileup": "uniform 50-200, 40 tracks per pileup unit",
            "launch": "one CUDA graph per batch", "dropped_objects": int(dropped), "autotune": tune,
            "plain_same_events": {"value": round(n_batch / (ms1 / 1e3), 2), "unit": "events/s",
                                  "launch": "one graph per event"}}


def measure_batched_pu200(P, E, geom, maps, cuts, flush, st, steps, events, sizes=(16, 64)):
    """PU200 events batched into one graph launch (16 and 64 per batch): events/s, and the batch's dominant
    kernel against the HBM roofline (algorithmic bytes of the whole batch over its live time, ncu traffic of
    the same launch from the committed summary when its sources are unchanged)."""
    import torch
    evs = list(events) + [E.pu200_event(s, geom) for s in range(len(events), max(sizes))]
    hbm_peak, peak_kind = _peaks()
    out = {}
    for n in sizes:
        ctx = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(n))
        b = P.pack_events(evs[:n])
        bd = {k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in b.items()}
        tune = autotune(ctx, bd, st, reps=2)
        for _ in range(2):
            ctx.run_packed(bd, stream=st.cuda_stream)
        torch.cuda.synchronize()
        ms = 0.0
        for i in range(steps):
            flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.run_packed(bd, stream=st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        tot = {"counts": {}, "dropped": 0}
        for e in range(n):
            s_ = ctx.stats(e)
            for k, v in s_["counts"].items():
                tot["counts"][k] = tot["counts"].get(k, 0) + v
            tot["dropped"] += sum(s_["dropped"].values())
        ctx.set_profiling(True)
        per = {}
        for i in range(2):
            flush.fill_(i & 0xff)
            ctx.run_packed(bd, stream=st.cuda_stream)
            for name, kms in ctx.kernel_times():
                per.setdefault(name, []).append(kms)
        ctx.set_profiling(False)
        ctx.close()
        kavg = {k: sum(v) / len(v) for k, v in per.items()}
        top = max(kavg, key=kavg.get)
        wl = f"pu200x{n}"
        rec = {"value": round(n * steps / (ms / 1e3), 2), "unit": "events/s", "ms_per_batch": round(ms / steps, 3),
               "launch": "one CUDA graph per batch", "dropped_objects": int(tot["dropped"]),
               "stage_sum_ms": round(sum(kavg.values()), 4),
               "kernel_ms": {k: round(v, 4) for k, v in sorted(kavg.items(), key=lambda kv: -kv[1])[:8]},
               "autotune_stage_sum_ms": [tune.get("stage_sum_ms_default"), tune.get("stage_sum_ms_tuned")]}
        b_alg = algorithmic_bytes(top, tot, int(b["hit_off"][-1]), int(b["seed_off"][-1]), geom.n_mod * n)
        if b_alg is not None:
            achieved = b_alg / (kavg[top] / 1e3) / 1e9
            traffic = measured_traffic(top, wl)
            rec["roofline"] = {"kernel": top, "bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak,
                               "unit": "GB/s", "frac": round(achieved / hbm_peak, 5), "traffic": traffic,
                               "traffic_over_algorithmic": None if traffic is None else round(traffic / b_alg, 3),
                               "peak_source": peak_kind, "algorithmic_bytes": int(b_alg),
                               "kernel_ms": round(kavg[top], 4)}
        out[f"{n}_events"] = rec
    out["workload"] = "PU200 events (the headline event recipe, seeds 0..63), one batch per launch sequence"
    out["l2"] = "flushed between batches (256 MiB write, outside the timed spans)"
    return out


def measure_d0_scan(P, E, geom, maps, cuts, st, n_events=32, n_muons=40):
    """Efficiency against the transverse impact parameter for displaced muons (vertices uniform in a 5 cm
    cube, zero pileup; the study of Section 2.2), by the type of the TC that finds each muon: with the
    connection map that covers vertices up to the cube's corner (2.5 sqrt(2) cm), and with the prompt maps."""
    import math
    from paper_2209_13711_gb300.metrics import efficiency_vs_d0
    from synth import maps as M
    evs = [E.muon_gun_event(9000 + i, geom, n=n_muons) for i in range(n_events)]
    out = {"events": n_events, "muons_per_event": n_muons, "muon_pt": "uniform 2-10 GeV", "eta": "|eta| < 2.4",
           "vertex": "uniform in a 5 cm cube"}
    for name, mp in (("displaced_map", M.load_maps(geom, M.MapParams(d0_max=2.5 * math.sqrt(2.0)))),
                     ("prompt_map", maps)):
        ctx = P.Context(geom.module_table(), mp, cfg=cuts, capacity=P.default_capacity(n_events))
        ctx.run(evs, stream=st.cuda_stream)
        per_event = [(ctx.track_candidates(e), ev.pid, ev.seed_pid, ev.tracks) for e, ev in enumerate(evs)]
        ctx.close()
        out[name] = efficiency_vs_d0(per_event)
    out["connections"] = {"displaced_map": int(len(M.load_maps(geom, M.MapParams(d0_max=2.5 * math.sqrt(2.0)))[1])),
                          "prompt_map": int(len(maps[1]))}
    return out


def _time_modes(P, geom, maps, cuts, flush, st, evs, modes, touched, reps=3):
    """Device time per batch of `evs` and the stage times of `touched` for each context set-up in `modes`
    (name -> function of the context), default launch shapes, L2 flushed before every run."""
    import torch
    b = P.pack_events(evs)
    bd = {k: (torch.from_numpy(v).cuda() if k not in ("hit_off", "seed_off") else v) for k, v in b.items()}
    rec = {}
    for mode, setup in modes.items():
        ctx = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(len(evs)))
        setup(ctx)
        for _ in range(2):
            ctx.run_packed(bd, stream=st.cuda_stream)
        torch.cuda.synchronize()
        ms = 0.0
        for i in range(reps):
            flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.run_packed(bd, stream=st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        counts = [ctx.stats(e)["counts"] for e in range(len(evs))]
        ctx.set_profiling(True)
        per = {}
        for i in range(reps):
            flush.fill_(i & 0xff)
            ctx.run_packed(bd, stream=st.cuda_stream)
            for name, kms in ctx.kernel_times():
                per.setdefault(name, []).append(kms)
        ctx.set_profiling(False)
        ctx.close()
        rec[mode] = {"ms_per_batch": round(ms / reps, 4), "events_per_s": round(1e3 * len(evs) * reps / ms, 2),
                     "stage_ms": {k: round(sum(per[k]) / len(per[k]), 4) for k in touched if k in per},
                     "counts": counts}
    return rec


def measure_compact(P, geom, maps, cuts, flush, st, events, sizes=(1, 64), reps=3):
    """Compact (16-bit) storage against the default, at 1 and 64 PU200 events per batch: device time per
    batch and the stage times of the kernels that read the 16-bit copies (default launch shapes for both, so
    that only the storage differs). Objects are identical by construction (tested on the GPU)."""
    from synth import events as E
    evs = list(events) + [E.pu200_event(s, geom) for s in range(len(events), max(sizes))]
    touched = ("t5", "pt3", "clean_pt3_cross", "clean_t5", "clean_pls")
    out = {}
    for n in sizes:
        rec = _time_modes(P, geom, maps, cuts, flush, st, evs[:n],
                          {"default": lambda c: None, "compact": lambda c: c.set_compact_storage(True)}, touched, reps)
        for mode in ("default", "compact"):
            counts = rec[mode].pop("counts")
            t3 = sum(c["t3"] for c in counts)
            rec[mode].pop("events_per_s")
            rec[mode]["triplet_curvature_bytes"] = int(t3 * (8 if mode == "default" else 12))
        rec["speedup"] = round(rec["default"]["ms_per_batch"] / rec["compact"]["ms_per_batch"], 3)
        out[f"{n}_events"] = rec
    out["note"] = ("compact keeps the FP32 (kappa, sigma) for the exact decisions and adds a 4-byte FP16 copy per "
                   "triplet that the searches read instead of the 8-byte pair; the eta-phi list entries shrink "
                   "from 8 to 4 bytes")
    return out


def measure_fit_precision(P, geom, maps, cuts, flush, st, events, sizes=(1, 64), reps=3):
    """The refine fits in float-float on the FP32 pipe (the default) against FP64, at 1 and 64 PU200 events per
    batch: device time per batch and the refine stage times (default launch shapes for both). The objects
    agree (tested on the GPU); the counts are reported as a check."""
    from synth import events as E
    evs = list(events) + [E.pu200_event(s, geom) for s in range(len(events), max(sizes))]
    touched = ("t5_refine", "pt5_refine", "pt3_refine")
    out = {}
    for n in sizes:
        rec = _time_modes(P, geom, maps, cuts, flush, st, evs[:n],
                          {"float_float": lambda c: None, "fp64": lambda c: c.set_fp64_fit(True)}, touched, reps)
        same = rec["float_float"].pop("counts") == rec["fp64"].pop("counts")
        rec["speedup"] = round(rec["fp64"]["ms_per_batch"] / rec["float_float"]["ms_per_batch"], 3)
        rec["same_object_counts"] = same
        out[f"{n}_events"] = rec
    return out


def measure_mlp(P, E, geom, maps, cuts, flush, st, dev_events):
    """Network-scored T5 selection: trained here (128 PU200 events, the training
    set held in device memory, the library's own kernels), compared with the
    hand-set cuts on 8 other events at matched efficiency, then timed on the
    benchmark's PU200 events."""
    import torch
    from paper_2209_13711_gb300 import train as T
    from synth.mlp_init import init_params
    t0 = time.perf_counter()
    ctx = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(16))
    ctx.set_t5_selection(None, prefilter_scale=3.0, capture_features=True)
    tr = T.collect(ctx, (E.pu200_event(40000 + i, geom) for i in range(128)), batch=16, device=True)
    va = T.collect(ctx, [E.pu200_event(41000 + i, geom) for i in range(8)], batch=16)
    ctx.close()
    mlp = P.Mlp(max_batch=4096, params=init_params(0))
    T.train(mlp, tr["X"], tr["y"], epochs=3)
    quality = T.evaluate(mlp, va)
    train_s = time.perf_counter() - t0
    ctx1 = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(1))
    ctx1.set_t5_selection(mlp, threshold=quality["threshold"], prefilter_scale=3.0)
    ctx1.run_packed(dev_events[0], stream=st.cuda_stream)
    torch.cuda.synchronize()
    ms = 0.0
    for i, b in enumerate(dev_events):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx1.run_packed(b, stream=st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    st0 = ctx1.stats(0)
    ctx1.set_profiling(True)
    ctx1.run_packed(dev_events[0], stream=st.cuda_stream)
    stage = {n: round(t, 4) for n, t in ctx1.kernel_times() if n.startswith("t5")}
    ctx1.set_profiling(False)
    ctx1.close()
    mlp.close()
    return {"value": round(len(dev_events) / (ms / 1e3), 2), "unit": "events/s",
            "selection": "T5 validity from the BF16 network (prefilter widened x3)",
            "t5_per_event": st0["counts"]["t5"], "tc_per_event": st0["counts"]["tc"], "t5_stage_ms": stage,
            "quality_at_matched_efficiency": {"cut": quality["cut"], "network": quality["network"],
                                              "threshold": round(quality["threshold"], 4),
                                              "samples_train": int(len(tr["y"])), "samples_eval": int(len(va["y"])),
                                              "train_events": 128, "eval_events": 8},
            "train_and_eval_s": round(train_s, 1)}


def measure_mlp_t3(P, E, geom, maps, cuts, flush, st, dev_events, events, n_train=16, n_eval=4, n_phys=16):
    """Learned triplet selection: a network trained here (T3s of 16 PU200 events, 2e5 per event, the library's
    own kernels) prunes triplets before the T5 and pT3 searches, at the threshold that keeps 99 % of true T3s on
    4 other events. Timed on the benchmark's PU200 events against the plain path's value, with the T3 fake
    fraction and the track-candidate figures of merit of 16 events with and without it."""
    import numpy as np
    import torch
    from paper_2209_13711_gb300 import metrics as MT
    from paper_2209_13711_gb300 import train as T
    from synth.mlp_init import init_params
    t0 = time.perf_counter()
    ctx = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(4))
    ctx.set_t3_selection(None, capture_features=True)
    tr = T.collect_t3(ctx, (E.pu200_event(43000 + i, geom) for i in range(n_train)), batch=4, max_per_event=200000)
    va = T.collect_t3(ctx, [E.pu200_event(44000 + i, geom) for i in range(n_eval)], batch=4, device=False)
    ctx.close()
    mlp = P.Mlp(max_batch=4096, params=init_params(3))
    T.train(mlp, tr["X"], tr["y"], epochs=3)
    s = T.scores_of(mlp, va["X"])
    thr = T.threshold_keeping(s, va["y"], 0.99)
    fake = va["y"] < 0.5
    train_s = time.perf_counter() - t0
    ctx1 = P.Context(geom.module_table(), maps, cfg=cuts, capacity=P.default_capacity(1))
    ctx1.set_t3_selection(mlp, threshold=thr)
    tune = autotune(ctx1, dev_events[0], st)
    ctx1.run_packed(dev_events[0], stream=st.cuda_stream)
    torch.cuda.synchronize()
    ms = 0.0
    for i, b in enumerate(dev_events):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx1.run_packed(b, stream=st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    ctx1.set_profiling(True)
    ctx1.run_packed(dev_events[0], stream=st.cuda_stream)
    stage = {n: round(t, 4) for n, t in ctx1.kernel_times() if n.startswith(("t3", "t5", "pt3"))}
    ctx1.set_profiling(False)
    phys = {}
    for mode in ("cuts", "network"):
        ctx1.set_t3_selection(mlp if mode == "network" else None, threshold=thr)
        rates, t5c = [], 0
        for i in range(min(n_phys, len(dev_events))):
            ctx1.run_packed(dev_events[i], stream=st.cuda_stream)
            ev = events[i]
            rates.append(MT.rates(ctx1.track_candidates(0), ev.pid, ev.seed_pid, ev.tracks))
            t5c += int(ctx1.counters()[21])
        c = MT.combine(rates)
        phys[mode] = {k: round(c[k], 4) for k in ("efficiency", "efficiency_ot", "fake_rate", "duplicate_rate")}
        phys[mode]["t5_search_survivors_per_event"] = t5c // n_phys
    ctx1.close()
    mlp.close()
    return {"value": round(len(dev_events) / (ms / 1e3), 2), "unit": "events/s",
            "selection": "T3s pruned by the BF16 network before the T5 and pT3 searches; hand-set cuts elsewhere",
            "threshold": round(thr, 4),
            "t3_selection_on_eval_events": {"true_kept": round(float(np.mean(s[~fake] >= thr)), 4),
                                            "fake_pruned": round(float(np.mean(s[fake] < thr)), 4),
                                            "fake_fraction_before": round(float(fake.mean()), 4),
                                            "fake_fraction_after": round(float(np.sum(fake & (s >= thr)) /
                                                                               max(1, np.sum(s >= thr))), 4)},
            "stage_ms": stage, "track_candidates": phys,
            "autotune_stage_sum_ms": [tune["stage_sum_ms_default"], tune["stage_sum_ms_tuned"]],
            "samples_train": int(len(tr["y"])), "train_events": n_train, "eval_events": n_eval,
            "train_and_eval_s": round(train_s, 1)}


def measure_serving(E, geom, maps, cuts, pool_size=32):
    """Poisson request streams (pileup uniform in 140-200) served by continuous
    batching on three resident contexts of 16 events each, against the plain
    path (one context, one event per launch). Latency: arrival to track
    candidates on the host."""
    import math
    import numpy as np
    from paper_2209_13711_gb300 import serve as S
    rng = np.random.default_rng(4242)
    pus = rng.uniform(140.0, 200.0, pool_size)
    pool = S.EventPool([E.pileup_event(float(pu), 8000 + i, geom) for i, pu in enumerate(pus)])
    sizes = (pool.n_hits, pool.n_seeds)
    table = geom.module_table()

    def run(slots, max_slots, max_batch, rate, n, seed):
        reqs = S.make_requests(sizes, rate, n, seed=seed)
        out, sch = S.serve(table, maps, pool, reqs, cfg=cuts, max_slots=max_slots, max_batch=max_batch, slots=slots)
        return S.summarize(out), sch

    def fmt(s):
        return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in s.items()}

    res = {"pool": f"{pool_size} events, pileup uniform 140-200 (40 tracks per unit), inputs in pinned host memory",
           "budget_gb": 60, "slots": 3, "events_per_slot": 16, "latency": "arrival to track candidates on the host"}
    _, sch = run(None, 3, 16, math.inf, 96, 1)                # opens and captures every slot
    slots = sch.slots
    res["slot_device_gb"] = round(slots[0].device_bytes / 1e9, 3)
    s, _ = run(slots, 3, 16, math.inf, 480, 2)
    res["saturated"] = fmt(s)
    res["poisson"] = {}
    for rate in (200.0, 500.0, 1000.0):
        s, _ = run(slots, 3, 16, rate, int(2.0 * rate), 3)
        res["poisson"][f"{int(rate)}Hz"] = fmt(s)
    for sl in slots:
        sl.close()
    _, sch1 = run(None, 1, 1, math.inf, 8, 4)
    plain = {}
    s, _ = run(sch1.slots, 1, 1, math.inf, 160, 5)
    plain["saturated"] = fmt(s)
    for rate in (200.0, 1000.0):
        s, _ = run(sch1.slots, 1, 1, rate, int(1.0 * rate), 6)
        plain[f"{int(rate)}Hz"] = fmt(s)
    sch1.slots[0].close()
    res["plain_one_event_per_launch"] = plain
    return res


def _oracle_event_seconds(seed):
    from oracle import oracle as O
    from synth import events as E, geometry as G, maps as M
    from synth.config import DEFAULT_CUTS
    geom = G.make_geometry(barrel_only=False)
    maps = M.load_maps(geom)
    ev = E.pu200_event(seed, geom)
    S = O.Setup(geom.module_table(), maps, DEFAULT_CUTS, ev)
    t0 = time.perf_counter()
    S.run()
    return time.perf_counter() - t0


def _oracle_worker(seed, kind, barrier, q):
    """One oracle event in its own process: build the inputs, wait for the other
    workers, then time the chain on the shared monotonic clock."""
    try:
        from oracle import oracle as O
        from synth import events as E, geometry as G, maps as M
        from synth.config import DEFAULT_CUTS
        make = {"pu200": E.pu200_event, "tiny": E.tiny_event}[kind]
        geom = G.make_geometry(barrel_only=kind == "tiny")
        maps = M.load_maps(geom)
        ev = make(seed, geom)
        S = O.Setup(geom.module_table(), maps, DEFAULT_CUTS, ev)
        barrier.wait(timeout=600)
        t0 = time.monotonic()
        S.run()
        q.put((t0, time.monotonic(), None))
    except Exception as e:  # reported to the parent, which raises
        barrier.abort()
        q.put((0.0, 0.0, repr(e)))


def _oracle_parallel_seconds(seeds, kind="pu200"):
    """Wall time of len(seeds) oracle events run at once, one process each
    (spawned, so no process inherits a CUDA context). The clock runs from the
    first start to the last finish, after all inputs are built."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(len(seeds)), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(s, kind, barrier, q)) for s in seeds]
    for p in procs:
        p.start()
    try:
        res = [q.get(timeout=1200) for _ in procs]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    errs = [e for _, _, e in res if e]
    if errs:
        raise RuntimeError("oracle worker failed: " + errs[0])
    return max(t1 for _, t1, _ in res) - min(t0 for t0, _, _ in res)


def cpu_baseline(args, budget_s=30.0):
    """The FP64 oracle, as it stands, on this host's cores: one PU200 event per
    core at once (the headline), and one thread alone."""
    t, n = 0.0, 0
    while n == 0 or (t < budget_s / 2 and n < 3):
        t += _oracle_event_seconds(n)
        n += 1
    cores = os.cpu_count() or 1
    wall = _oracle_parallel_seconds(list(range(100, 100 + cores)))
    return {"value": round(cores / wall, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} PU200 events (seeds 100..{99 + cores}), one per core in spawned processes, full "
                      f"chain, FP64; timed from the first start to the last finish",
            "single_thread": {"value": round(n / t, 4), "unit": UNIT, "cores": 1,
                              "sample": f"{n} PU200 event(s), seeds 0..{n - 1}, one after another"},
            "host_cpus": os.cpu_count()}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    import platform
    budget = 150.0
    cores = os.cpu_count() or 1
    # warm-up: args.warmup oracle events, run side by side like a timed step (page cache, library load)
    if args.warmup > 0:
        _oracle_parallel_seconds(list(range(1000, 1000 + args.warmup)))
    times, seed = [], 0
    t_start = time.perf_counter()
    for i in range(args.steps):
        times.append(_oracle_parallel_seconds(list(range(seed, seed + cores))))
        seed += cores
        if time.perf_counter() - t_start > budget:
            break
    k = len(times)
    value = k * cores / sum(times)
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": k,
        "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / k, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_step": cores,
                   "path": f"FP64 CPU oracle, {cores} PU200 events per step, one per host core"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{k * cores} PU200 events in {k} step(s) of {cores} concurrent processes "
                                   f"(timed steps capped at {budget:.0f} s)",
                         "host": platform.machine()},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
