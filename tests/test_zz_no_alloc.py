"""The allocation-free mini-doublet builder agrees with the context path (GPU).

Callers that cannot allocate device memory (a framework owning the device
budget through its own pool, a latency-critical loop) use
lst_build_mini_doublets_static, whose scratch is a fixed device array inside
the library. These tests call it through the C ABI and check each result
against the mini-doublets of the ordinary context path for the same event:
the same (lower hit, upper hit, module) rows, and dphi / dlong within 1e-5 of
their value (at least 1e-5 of the cut scale 1e-3). Two calls in a row must
agree; a call must leave the device's free memory unchanged; a capacity
below the event's count must clip exactly and write nothing past it; and a
sensor with more than 256 hits must keep the same hits as the chain.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _md_rows(lo, up, mod, dphi, dlong):
    return {(int(a), int(b), int(m)): (float(p), float(q)) for a, b, m, p, q in zip(lo, up, mod, dphi, dlong)}


def _entry_point():
    from paper_2209_13711_gb300 import lst
    f = lst.library().lst_build_mini_doublets_static
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int32] + [C.c_void_p] * 5 + [C.c_int32, C.c_int32] + \
        [C.c_void_p] * 7 + [C.c_void_p]
    return f


def _context_mds(geom, maps, ev):
    import paper_2209_13711_gb300 as P
    from synth.config import DEFAULT_CUTS
    ctx = P.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=P.default_capacity(1))
    ctx.run([ev])
    ref = ctx.objects("md", 0)
    dropped = ctx.stats(0)["dropped"]["md"]
    ctx.close()
    return _md_rows(ref["lo"], ref["up"], ref["mod"], ref["dphi"], ref["dlong"]), dropped


class StaticCall:
    """Device copies of one event and of the module table, and output buffers with guard elements."""

    GUARD = 64

    def __init__(self, torch, geom, ev):
        from paper_2209_13711_gb300 import lst
        from synth.config import DEFAULT_CUTS
        self.torch = torch
        mt = geom.module_table()
        rows = np.zeros(geom.n_mod, dtype=[("subdet", "<i4"), ("layer", "<i4"), ("dsep", "<f4"),
                                           ("sig_rphi", "<f4"), ("sig_long", "<f4")])
        for k in rows.dtype.names:
            rows[k] = mt[k]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.n_mod = geom.n_mod
        self.mods = dev(rows.view(np.uint8))
        self.hits = [dev(ev.x), dev(ev.y), dev(ev.z), dev(ev.module), dev(ev.side)]
        self.n_hits = len(ev.x)
        self.cfg = lst.default_config(DEFAULT_CUTS)
        self.f = _entry_point()

    def outputs(self, cap):
        """Fresh output buffers (torch allocations, made before the call is timed or measured)."""
        torch = self.torch
        n = cap + self.GUARD
        self.out = [torch.full((n,), -7, dtype=torch.int32, device="cuda") for _ in range(3)] + \
                   [torch.full((n,), -7.0, dtype=torch.float32, device="cuda") for _ in range(2)]
        self.count = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.dropped = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()

    def __call__(self, cap, fresh=True):
        torch = self.torch
        if fresh:
            self.outputs(cap)
        p = lambda t: C.c_void_p(t.data_ptr())
        stream = torch.cuda.current_stream().cuda_stream
        st = self.f(C.byref(self.cfg), p(self.mods), self.n_mod, *[p(t) for t in self.hits], self.n_hits, cap,
                    *[p(t) for t in self.out], p(self.count), p(self.dropped), C.c_void_p(stream))
        assert st == 0, st
        torch.cuda.synchronize()
        n = int(self.count.item())
        cols = [t[:n].cpu().numpy() for t in self.out]
        guards = [t[cap:].cpu().numpy() for t in self.out]
        return _md_rows(*cols), int(self.dropped.item()), guards


def _same(got, want):
    assert set(got) == set(want)
    for k, (dp, dl) in want.items():
        gp, gl = got[k]
        assert abs(gp - dp) <= 1e-5 * max(abs(dp), 1e-3)
        assert abs(gl - dl) <= 1e-5 * max(abs(dl), 1e-3)


def test_static_builder_matches_context_path(geom_full, maps_full):
    torch = pytest.importorskip("torch")
    from synth import events as E

    ev = E.pileup_event(40, 21, geom_full)
    want, ctx_dropped = _context_mds(geom_full, maps_full, ev)
    assert len(want) > 1000 and ctx_dropped == 0
    call = StaticCall(torch, geom_full, ev)
    for i in range(2):
        call.outputs(131072)
        free_before = torch.cuda.mem_get_info()[0]
        got, dropped, _ = call(131072, fresh=False)
        if i == 1:
            # the second call allocates nothing (the first one may load the library's module)
            assert torch.cuda.mem_get_info()[0] == free_before
        assert dropped == 0
        _same(got, want)


def test_static_builder_clips_at_capacity(geom_full, maps_full):
    """md_capacity below the event's count: exactly md_capacity rows, the rest counted as dropped, and the
    guard elements past md_capacity untouched."""
    torch = pytest.importorskip("torch")
    from synth import events as E

    ev = E.pileup_event(40, 21, geom_full)
    want, _ = _context_mds(geom_full, maps_full, ev)
    call = StaticCall(torch, geom_full, ev)
    cap = len(want) // 3
    got, dropped, guards = call(cap)
    assert len(got) == cap
    assert dropped == len(want) - cap
    assert set(got) <= set(want)
    for g in guards:
        assert np.all(g == -7)


def test_static_builder_keeps_the_chains_hits_in_a_crowded_sensor(geom_full, maps_full):
    """300 extra hits on one lower sensor (more than the 256 a sensor keeps): both paths keep the 256 lowest
    input indices, so the rows and the dropped count agree."""
    torch = pytest.importorskip("torch")
    from synth import events as E

    ev = E.pileup_event(20, 22, geom_full)
    m = int(np.bincount(ev.module[ev.side == 0], minlength=geom_full.n_mod).argmax())
    sel = np.nonzero((ev.module == m) & (ev.side == 0))[0]
    rng = np.random.default_rng(5)
    pick = rng.choice(sel, 300)
    jitter = rng.normal(0.0, 0.05, (300, 3)).astype(np.float32)
    extra = dict(x=ev.x[pick] + jitter[:, 0], y=ev.y[pick] + jitter[:, 1], z=ev.z[pick] + jitter[:, 2])
    # the extra hits go first, so the kept 256 are extra hits and the event's own hits of that sensor are cut
    ev.x = np.concatenate([extra["x"], ev.x]).astype(np.float32)
    ev.y = np.concatenate([extra["y"], ev.y]).astype(np.float32)
    ev.z = np.concatenate([extra["z"], ev.z]).astype(np.float32)
    ev.module = np.concatenate([np.full(300, m, np.int32), ev.module]).astype(np.int32)
    ev.side = np.concatenate([np.zeros(300, np.uint8), ev.side]).astype(np.uint8)
    want, ctx_dropped = _context_mds(geom_full, maps_full, ev)
    assert ctx_dropped > 0
    got, dropped, _ = StaticCall(torch, geom_full, ev)(131072)
    assert dropped == ctx_dropped
    _same(got, want)


def test_static_builder_rejects_oversized_input():
    from paper_2209_13711_gb300 import lst
    f = _entry_point()
    cfg = lst.default_config()
    one = C.c_void_p(16)       # never dereferenced: the size check comes first
    args = [one] * 5
    st = f(C.byref(cfg), one, 20000, *args, 100, 10, *([one] * 6), None, None)
    assert st == -6          # LST_ERR_CAPACITY: more than 16384 modules
    st = f(C.byref(cfg), one, 100, *args, 300000, 10, *([one] * 6), None, None)
    assert st == -6          # more than 262144 hits
