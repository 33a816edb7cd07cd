"""The allocation-free mini-doublet builder agrees with the context path (GPU).

Callers that cannot allocate device memory (a framework owning the device
budget through its own pool, a latency-critical loop) use
lst_build_mini_doublets_static, whose scratch is a fixed device array inside
the library. This test calls it through the C ABI twice in a row and checks
each result against the mini-doublets of the ordinary context path for the
same event: the same (lower hit, upper hit, module) rows, and dphi / dlong
within 1e-5 of their value (at least 1e-5 of the cut scale 1e-3).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _md_rows(lo, up, mod, dphi, dlong):
    return {(int(a), int(b), int(m)): (float(p), float(q)) for a, b, m, p, q in zip(lo, up, mod, dphi, dlong)}


def test_static_builder_matches_context_path(geom_full, maps_full):
    torch = pytest.importorskip("torch")
    import paper_2209_13711_gb300 as P
    from paper_2209_13711_gb300 import lst
    from synth import events as E
    from synth.config import DEFAULT_CUTS

    ev = E.pileup_event(40, 21, geom_full)
    ctx = P.Context(geom_full.module_table(), maps_full, cfg=DEFAULT_CUTS, capacity=P.default_capacity(1))
    ctx.run([ev])
    ref = ctx.objects("md", 0)
    want = _md_rows(ref["lo"], ref["up"], ref["mod"], ref["dphi"], ref["dlong"])
    assert len(want) > 1000
    ctx.close()

    L = lst.library()
    f = L.lst_build_mini_doublets_static
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int32] + [C.c_void_p] * 5 + [C.c_int32, C.c_int32] + \
        [C.c_void_p] * 7 + [C.c_void_p]
    mt = geom_full.module_table()
    rows = np.zeros(geom_full.n_mod, dtype=[("subdet", "<i4"), ("layer", "<i4"), ("dsep", "<f4"),
                                            ("sig_rphi", "<f4"), ("sig_long", "<f4")])
    for k in rows.dtype.names:
        rows[k] = mt[k]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mods = dev(rows.view(np.uint8))
    hx, hy, hz, hm, hs = dev(ev.x), dev(ev.y), dev(ev.z), dev(ev.module), dev(ev.side)
    cap = 131072
    cfg = lst.default_config(DEFAULT_CUTS)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out_lo = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
        out_up = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
        out_mod = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
        out_dphi = torch.zeros(cap, dtype=torch.float32, device="cuda")
        out_dlong = torch.zeros(cap, dtype=torch.float32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        dropped = torch.zeros(1, dtype=torch.int32, device="cuda")
        p = lambda t: C.c_void_p(t.data_ptr())
        st = f(C.byref(cfg), p(mods), geom_full.n_mod, p(hx), p(hy), p(hz), p(hm), p(hs), len(ev.x), cap,
               p(out_lo), p(out_up), p(out_mod), p(out_dphi), p(out_dlong), p(count), p(dropped), C.c_void_p(stream))
        assert st == 0, st
        torch.cuda.synchronize()
        n = int(count.item())
        assert int(dropped.item()) == 0
        got = _md_rows(out_lo[:n].cpu().numpy(), out_up[:n].cpu().numpy(), out_mod[:n].cpu().numpy(),
                       out_dphi[:n].cpu().numpy(), out_dlong[:n].cpu().numpy())
        assert n == len(want) and set(got) == set(want), call
        for k, (dp, dl) in want.items():
            gp, gl = got[k]
            assert abs(gp - dp) <= 1e-5 * max(abs(dp), 1e-3)
            assert abs(gl - dl) <= 1e-5 * max(abs(dl), 1e-3)


def test_static_builder_rejects_oversized_input():
    from paper_2209_13711_gb300 import lst
    L = lst.library()
    f = L.lst_build_mini_doublets_static
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int32] + [C.c_void_p] * 5 + [C.c_int32, C.c_int32] + \
        [C.c_void_p] * 7 + [C.c_void_p]
    cfg = lst.default_config()
    one = C.c_void_p(16)       # never dereferenced: the size check comes first
    args = [one] * 5
    st = f(C.byref(cfg), one, 20000, *args, 100, 10, *([one] * 6), None, None)
    assert st == -6          # LST_ERR_CAPACITY: more than 16384 modules
    st = f(C.byref(cfg), one, 100, *args, 300000, 10, *([one] * 6), None, None)
    assert st == -6          # more than 262144 hits
