"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the benchmark's CPU-baseline leg use
this module. It never imports the device package.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

KINDS = dict(md=0, ls=1, t3=2, t4=None, t5=3, pls=4, pt3=5, pt5=6, tc=7,
             m_md=10, m_ls=11, m_t3=12, m_t5=13, m_pls=14, m_pt3=15, m_pt5=16, m_clean=17)
COLUMNS = {
    "md": (["lo", "up", "mod", "margin"], ["dphi", "dlong", "thr_phi", "thr_long"]),
    "ls": (["md_in", "md_out", "margin"], ["dphi", "thr_phi"]),
    "t3": (["ls_in", "ls_out", "margin"], ["beta", "thr_beta", "kappa", "sigk", "rz", "thr_rz"]),
    "t5": (["t3_in", "t3_out", "margin"], ["kappa", "chi2_rphi", "chi2_rz", "eta", "phi0", "pt", "score", "sigk"]),
    "pls": (["seed", "pass", "sb", "margin"], ["kappa", "sigk", "eta", "phi0", "z0", "pt"]),
    "pt3": (["seed", "t3", "margin"], ["kappa", "chi2_rphi", "chi2_rz", "score", "pt"]),
    "pt5": (["seed", "t5", "margin"], ["kappa", "chi2_rphi", "chi2_rz", "score", "pt"]),
    "tc": (["type", "seed", "obj"] + [f"h{i}" for i in range(10)], ["pt", "eta", "phi0"]),
}
STAGES = ("md", "ls", "t3", "t5", "pls", "pt5", "pt3", "tc")   # run(upto=i) stops after STAGES[i]


class OGeom(C.Structure):
    _fields_ = [("n_mod", C.c_int32), ("subdet", C.c_void_p), ("layer", C.c_void_p), ("surf", C.c_void_p),
                ("dsep", C.c_void_p), ("sig_rphi", C.c_void_p), ("sig_long", C.c_void_p),
                ("conn_off", C.c_void_p), ("conn_tgt", C.c_void_p), ("sb_off", C.c_void_p),
                ("sb_tgt", C.c_void_p), ("n_sb", C.c_int32)]


class OCfg(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("pt_min", "k_field", "b_field", "z_lumi", "n_md", "n_ls", "n_t3", "n_t5",
                                          "n_pt", "tol_r", "chi2_rphi_t5", "chi2_rz_t5", "chi2_rphi_pt3",
                                          "chi2_rz_pt3", "chi2_rphi_pt5", "chi2_rz_pt5", "pls_pt_tol", "sig_pix",
                                          "sb_eta_max")] + \
        [("sb_n_eta", C.c_int32), ("sb_n_phi", C.c_int32), ("dr_clean", C.c_double), ("margin_rel", C.c_double)]


class OEvent(C.Structure):
    _fields_ = [("n_hits", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("module", C.c_void_p), ("side", C.c_void_p), ("n_seeds", C.c_int32), ("seeds", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_run.restype = C.c_void_p
        L.oracle_run.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.oracle_free.argtypes = [C.c_void_p]
        L.oracle_count.argtypes = [C.c_void_p, C.c_int]
        L.oracle_ncols.argtypes = [C.c_int, C.c_int]
        L.oracle_fetch.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.oracle_pred_md.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.oracle_pred_chain.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.oracle_pls.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_fit.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.oracle_tri.argtypes = [C.c_void_p, C.c_void_p]
        L.oracle_t5_features.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_t3_features.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_md_d.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_ls_d.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
        L.oracle_t3_d.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_t5_d.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_pls_d.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_pt_d.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Setup:
    """Geometry, maps, config and event marshalled once for the C oracle."""

    def __init__(self, module_table, maps, cfg, event=None):
        self._keep = []
        mt = {k: np.ascontiguousarray(v) for k, v in module_table.items()}
        co, ct, so, st = [np.ascontiguousarray(a, dtype=np.int32) for a in maps]
        self._keep += list(mt.values()) + [co, ct, so, st]
        self.geom = OGeom(n_mod=len(mt["subdet"]), subdet=_ptr(mt["subdet"]), layer=_ptr(mt["layer"]),
                          surf=_ptr(mt["surf"]), dsep=_ptr(mt["dsep"]), sig_rphi=_ptr(mt["sig_rphi"]),
                          sig_long=_ptr(mt["sig_long"]), conn_off=_ptr(co), conn_tgt=_ptr(ct), sb_off=_ptr(so),
                          sb_tgt=_ptr(st), n_sb=len(so) - 1)
        self.cfg = OCfg(**{k: cfg[k] for k, _ in OCfg._fields_})
        self.n_sb = len(so) - 1
        if event is not None:
            self.set_event(event)

    def set_event(self, ev):
        cols = dict(x=np.ascontiguousarray(ev.x, np.float32), y=np.ascontiguousarray(ev.y, np.float32),
                    z=np.ascontiguousarray(ev.z, np.float32), module=np.ascontiguousarray(ev.module, np.int32),
                    side=np.ascontiguousarray(ev.side, np.uint8),
                    seeds=np.ascontiguousarray(np.asarray(ev.seeds, np.float32).reshape(-1, 9)))
        self._ev = cols
        self.event = OEvent(n_hits=len(cols["x"]), x=_ptr(cols["x"]), y=_ptr(cols["y"]), z=_ptr(cols["z"]),
                            module=_ptr(cols["module"]), side=_ptr(cols["side"]), n_seeds=len(cols["seeds"]),
                            seeds=_ptr(cols["seeds"]))

    # -- full chain -------------------------------------------------------
    def run(self, upto="tc"):
        L = lib()
        h = L.oracle_run(C.byref(self.geom), C.byref(self.cfg), C.byref(self.event), STAGES.index(upto))
        try:
            out = {}
            for name, code in KINDS.items():
                if code is None:
                    continue
                n = L.oracle_count(h, code)
                ni, nd = L.oracle_ncols(code, 0), L.oracle_ncols(code, 1)
                I = np.zeros((n, ni), np.int32)
                D = np.zeros((n, max(nd, 1)), np.float64)
                if n:
                    L.oracle_fetch(h, code, _ptr(I), _ptr(D) if nd else None)
                if name in COLUMNS:
                    icol, dcol = COLUMNS[name]
                    rec = {c: I[:, j] for j, c in enumerate(icol)}
                    rec.update({c: D[:, j] for j, c in enumerate(dcol)})
                    rec["n"] = n
                    out[name] = rec
                else:
                    out[name] = I
            return out
        finally:
            L.oracle_free(h)

    # -- single predicates (brute-force tests) ------------------------------
    def pred_md(self, hl, hu):
        nr = C.c_int(0)
        ok = lib().oracle_pred_md(C.byref(self.geom), C.byref(self.cfg), C.byref(self.event), int(hl), int(hu),
                                  C.byref(nr))
        return bool(ok), bool(nr.value)

    def t5_features(self, md_hits):
        """Scoring features (48) of the T5 formed by five (lower, upper) hit pairs."""
        h = np.ascontiguousarray(np.asarray(md_hits, np.int32).ravel())
        out = np.zeros(48)
        lib().oracle_t5_features(C.byref(self.geom), C.byref(self.cfg), C.byref(self.event), _ptr(h), _ptr(out))
        return out

    def t3_features(self, md_hits):
        """Scoring features (48) of the T3 formed by three (lower, upper) hit pairs."""
        h = np.ascontiguousarray(np.asarray(md_hits, np.int32).ravel())
        out = np.zeros(48)
        lib().oracle_t3_features(C.byref(self.geom), C.byref(self.cfg), C.byref(self.event), _ptr(h), _ptr(out))
        return out

    def pred_chain(self, md_hits, kind):
        h = np.ascontiguousarray(np.asarray(md_hits, np.int32).ravel())
        nr = C.c_int(0)
        ok = lib().oracle_pred_chain(C.byref(self.geom), C.byref(self.cfg), C.byref(self.event), _ptr(h), int(kind),
                                     C.byref(nr))
        return bool(ok), bool(nr.value)


def pls_fields(cfg, seed9):
    s = np.ascontiguousarray(np.asarray(seed9, np.float32).ravel())
    o = np.zeros(3, np.int32)
    d = np.zeros(6)
    c = OCfg(**{k: cfg[k] for k, _ in OCfg._fields_})
    lib().oracle_pls(C.byref(c), _ptr(s), _ptr(o), _ptr(d))
    return dict(pass_=int(o[0]), sb=int(o[1]), near=int(o[2]), kappa=d[0], sigk=d[1], eta=d[2], phi0=d[3], z0=d[4],
                pt=d[5])


def fit(rows):
    """rows: [n, 6] = (x, y, z, sig_rphi, sig_z, sig_r) -> (kappa, chi2_rphi, chi2_rz, tanl)."""
    r = np.ascontiguousarray(np.asarray(rows, np.float64))
    out = np.zeros(4)
    lib().oracle_fit(_ptr(r), len(r), _ptr(out))
    return out


def tri(rows):
    """rows: [3, 6] -> (beta, sig_beta, kappa, sigk)."""
    r = np.ascontiguousarray(np.asarray(rows, np.float64))
    out = np.zeros(4)
    lib().oracle_tri(_ptr(r), _ptr(out))
    return out


def _d(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, np.float64).ravel())
    return a


class Predicates:
    """FP64-input single-candidate evaluations (closed-form pins)."""

    def __init__(self, setup: Setup):
        self.s = setup

    def md(self, m, L, U):
        out = np.zeros(5)
        L_, U_ = _d(L), _d(U)
        ok = lib().oracle_md_d(C.byref(self.s.geom), C.byref(self.s.cfg), int(m), _ptr(L_), _ptr(U_), _ptr(out))
        return bool(ok), dict(dphi=out[0], dlong=out[1], thr_phi=out[2], thr_long=out[3], near=bool(out[4]))

    def ls(self, mA, LA, UA, mB, LB, UB):
        out = np.zeros(9)
        a = [_d(v) for v in (LA, UA, LB, UB)]
        ok = lib().oracle_ls_d(C.byref(self.s.geom), C.byref(self.s.cfg), int(mA), _ptr(a[0]), _ptr(a[1]), int(mB),
                               _ptr(a[2]), _ptr(a[3]), _ptr(out))
        return bool(ok), dict(num=out[0], thr_p=out[1], dphi=out[2], thr_phi=out[3], alpha_in=out[4],
                              thr_in=out[5], alpha_out=out[6], thr_out=out[7], near=bool(out[8]))

    def t3(self, rows):
        out = np.zeros(7)
        r = _d(rows)
        ok = lib().oracle_t3_d(C.byref(self.s.cfg), _ptr(r), _ptr(out))
        return bool(ok), dict(beta=out[0], thr_beta=out[1], kappa=out[2], sigk=out[3], rz=out[4], thr_rz=out[5],
                              near=bool(out[6]))

    def t5(self, rows):
        out = np.zeros(11)
        r = _d(rows)
        ok = lib().oracle_t5_d(C.byref(self.s.cfg), _ptr(r), _ptr(out))
        return bool(ok), dict(dkappa=out[0], thr_dkappa=out[1], kappa=out[2], chi2_rphi=out[3], chi2_rz=out[4],
                              eta=out[5], phi0=out[6], pt=out[7], score=out[8], near=bool(out[9]), sigk=out[10])

    def pls(self, q):
        io = np.zeros(3, np.int32)
        do = np.zeros(6)
        qq = _d(q)
        lib().oracle_pls_d(C.byref(self.s.cfg), _ptr(qq), _ptr(io), _ptr(do))
        return dict(pass_=bool(io[0]), sb=int(io[1]), near=bool(io[2]), kappa=do[0], sigk=do[1], eta=do[2],
                    phi0=do[3], z0=do[4], pt=do[5])

    def pt(self, rows, kappa_pls, sigk_pls, kappa_t, sigk_t):
        r = _d(rows)
        n = len(r) // 6
        out = np.zeros(7)
        ok = lib().oracle_pt_d(C.byref(self.s.cfg), _ptr(r), n, kappa_pls, sigk_pls, kappa_t, sigk_t, _ptr(out))
        return bool(ok), dict(kappa=out[0], chi2_rphi=out[1], chi2_rz=out[2], score=out[3], near=bool(out[4]),
                              dkappa=out[5], thr_dkappa=out[6])
