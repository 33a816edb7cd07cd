"""Shared set-up of the GPU tests: contexts, oracle runs, result dicts."""
from oracle import oracle as O
from synth.config import DEFAULT_CUTS

A_HALF = DEFAULT_CUTS["k_field"] * DEFAULT_CUTS["b_field"] / (200.0 * DEFAULT_CUTS["pt_min"])


def make_context(geom, maps, max_events=1, **cap):
    import paper_2209_13711_gb300 as P
    cap_ = P.default_capacity(max_events, **cap)
    return P.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=cap_)


def gpu_result(ctx, event=0):
    out = {k: ctx.objects(k, event) for k in ("md", "ls", "t3", "t5", "pls", "pt5", "pt3")}
    out["tc"] = ctx.track_candidates(event)
    out["stats"] = ctx.stats(event)
    return out


def oracle_result(geom, maps, ev):
    return O.Setup(geom.module_table(), maps, DEFAULT_CUTS, ev).run()


def all_tuples(ctx, event):
    """Every object level of an event as sets of hit tuples, and the TC set."""
    from tests.parity import chain_tuples
    g = gpu_result(ctx, event)
    T = chain_tuples(g)
    tc = {(int(t), int(s), tuple(sorted(h[h >= 0].tolist())))
          for t, s, h in zip(g["tc"]["type"], g["tc"]["seed"], g["tc"]["hits"])}
    return {k: set(v) for k, v in T.items()}, tc
