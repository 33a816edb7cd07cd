"""Python binding of the C ABI in include/lst.h (argument marshalling only).

Every step of the chain runs in the CUDA kernels of liblst.so; this module
packs arrays, passes pointers and unpacks results. Inputs are numpy arrays
or pinned CPU tensors (host memory: the library copies them) or CUDA torch
tensors (device memory: read in place). Calling into it without a built
library raises LstError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblst.so")

KIND_NAMES = ("md", "ls", "t3", "t5", "pls", "pt5", "pt3")
COLUMNS = {
    "md": (["lo", "up", "mod"], ["dphi", "dlong"]),
    "ls": (["md_in", "md_out"], ["dphi"]),
    "t3": (["ls_in", "ls_out"], ["beta", "kappa", "sigk"]),
    "t5": (["t3_in", "t3_out"], ["kappa", "chi2_rphi", "chi2_rz", "eta", "phi0", "pt", "score"]),
    "pls": (["seed", "pass", "sb"], ["kappa", "sigk", "eta", "phi0", "z0", "pt"]),
    "pt5": (["seed", "t5"], ["kappa", "chi2_rphi", "chi2_rz", "score", "pt"]),
    "pt3": (["seed", "t3"], ["kappa", "chi2_rphi", "chi2_rz", "score", "pt"]),
}
STAT_NAMES = ("md", "ls", "t3", "t5", "pls", "pt5", "pt3", "tc")


class LstConfig(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "pt_min", "k_field", "b_field", "z_lumi", "n_md", "n_ls", "n_t3", "n_t5", "n_pt", "tol_r",
        "chi2_rphi_t5", "chi2_rz_t5", "chi2_rphi_pt3", "chi2_rz_pt3", "chi2_rphi_pt5", "chi2_rz_pt5",
        "pls_pt_tol", "sig_pix", "sb_eta_max")] + \
        [("sb_n_eta", C.c_int32), ("sb_n_phi", C.c_int32), ("dr_clean", C.c_double)]


class LstCapacity(C.Structure):
    _fields_ = [(n, C.c_int32) for n in (
        "max_events", "max_hits", "max_seeds", "md_per_event", "ls_per_event", "t3_per_event", "t5_per_event",
        "pt3_per_event", "pt5_per_event", "tc_per_event")]


LST_RESULT_SLOTS = 4          # result slots of a context (include/lst.h)


class LstModule(C.Structure):
    _fields_ = [("subdet", C.c_int32), ("layer", C.c_int32), ("dsep", C.c_float), ("sig_rphi", C.c_float),
                ("sig_long", C.c_float)]


class LstHits(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("module", C.c_void_p),
                ("side", C.c_void_p), ("n", C.c_int32)]


class LstSeeds(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("n", C.c_int32)]


class LstStats(C.Structure):
    _fields_ = [("counts", C.c_int32 * 8), ("dropped", C.c_int32 * 8)]


class LstPeaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("fp64_tflops", C.c_double), ("atom_warp_gops", C.c_double),
                ("atom_same_gops", C.c_double), ("red_lane_gops", C.c_double), ("ms", C.c_float * 5),
                ("sm_count", C.c_int32), ("clock_khz", C.c_int32)]


class LstError(RuntimeError):
    pass


_lib = None


def library():
    """Load liblst.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LstError(f"liblst.so is not built ({LIB_PATH}); run paper_2209_13711_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, p = C.c_void_p, C.c_int32, C.c_int64, C.POINTER
        L.lst_status_str.restype = C.c_char_p
        L.lst_status_str.argtypes = [i32]
        L.lst_config_default.argtypes = [vp]
        L.lst_capacity_default.argtypes = [vp, i32]
        L.lst_create.argtypes = [p(vp), vp, vp, i32]
        L.lst_destroy.argtypes = [vp]
        L.lst_destroy.restype = None
        L.lst_load_geometry.argtypes = [vp, vp, i32, vp, vp, vp, vp, i32]
        L.lst_run_batch.argtypes = [vp, vp, vp, vp, vp, i32, i32, vp, vp]
        L.lst_run_event.argtypes = [vp, vp, vp, i32, vp, vp]
        L.lst_release_event.argtypes = [vp, i64]
        L.lst_get_track_candidates.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp]
        L.lst_object_columns.argtypes = [i32, vp, vp]
        L.lst_get_objects.argtypes = [vp, i64, i32, i32, vp, vp, vp]
        L.lst_get_stats.argtypes = [vp, i64, vp]
        L.lst_last_launch_count.argtypes = [vp]
        L.lst_set_profiling.argtypes = [vp, i32]
        L.lst_get_counters.argtypes = [vp, vp, i32]
        L.lst_set_stage_limits.argtypes = [vp, i32, i32]
        L.lst_set_compact_storage.argtypes = [vp, i32]
        L.lst_set_fp64_fit.argtypes = [vp, i32]
        L.lst_launch_stage_count.argtypes = []
        L.lst_launch_stage_count.restype = i32
        L.lst_get_launch_config.argtypes = [vp, i32, C.POINTER(C.c_char_p), vp, vp, vp]
        L.lst_set_launch_config.argtypes = [vp, i32, i32, i32]
        L.lst_autotune.argtypes = [vp, vp, vp, vp, vp, i32, i32, vp, i32, vp, vp]
        L.lst_run_events.argtypes = [vp, vp, vp, i32, i32, vp, vp]
        L.lst_get_batch_track_candidates.argtypes = [vp, i32, vp, vp]
        L.lst_query.argtypes = [vp]
        L.lst_query.restype = i32
        L.lst_device_bytes.argtypes = [vp]
        L.lst_device_bytes.restype = C.c_int64
        L.lst_mlp_create.argtypes = [p(vp), i32, i32]
        L.lst_mlp_destroy.argtypes = [vp]
        L.lst_mlp_destroy.restype = None
        L.lst_mlp_set_params.argtypes = [vp, vp]
        L.lst_mlp_get_params.argtypes = [vp, vp]
        L.lst_mlp_get_state.argtypes = [vp, vp, vp, vp, vp]
        L.lst_mlp_set_state.argtypes = [vp, vp, vp, vp, i64]
        L.lst_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
        L.lst_mlp_gradient.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.lst_mlp_train_step.argtypes = [vp, vp, vp, i32, C.c_float, vp, vp]
        L.lst_set_t5_selection.argtypes = [vp, vp, C.c_float, C.c_float, i32]
        L.lst_get_t5_candidates.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp]
        L.lst_set_t3_selection.argtypes = [vp, vp, C.c_float, i32]
        L.lst_get_t3_candidates.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp]
        L.lst_get_kernel_times.argtypes = [vp, i32, vp, vp, vp]
        L.lst_measure_peaks.argtypes = [i32, vp]
        L.lst_build_mini_doublets_static.argtypes = [vp, vp, i32] + [vp] * 5 + [i32, i32] + [vp] * 7 + [vp]
        for f in ("lst_config_default", "lst_capacity_default", "lst_create", "lst_load_geometry", "lst_run_batch",
                  "lst_run_event", "lst_get_track_candidates", "lst_object_columns", "lst_get_objects",
                  "lst_get_stats", "lst_last_launch_count", "lst_set_profiling", "lst_get_kernel_times",
                  "lst_get_counters", "lst_mlp_create", "lst_mlp_set_params", "lst_mlp_get_params",
                  "lst_mlp_forward", "lst_mlp_gradient", "lst_mlp_train_step", "lst_set_t5_selection",
                  "lst_get_t5_candidates", "lst_measure_peaks", "lst_build_mini_doublets_static",
                  "lst_release_event", "lst_run_events", "lst_get_batch_track_candidates", "lst_mlp_get_state",
                  "lst_mlp_set_state", "lst_set_compact_storage", "lst_set_t3_selection", "lst_set_fp64_fit",
                  "lst_get_t3_candidates"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def _check(status):
    if status < 0:
        raise LstError(f"lst error {status}: {library().lst_status_str(status).decode()}")
    return status


TC_DTYPE = np.dtype([("type", "<i4"), ("seed", "<i4"), ("hits", "<i4", (10,)), ("pt", "<f4"), ("eta", "<f4"),
                     ("phi0", "<f4"), ("reserved", "<i4")])


def tc_dict(rec):
    """Packed records of one event as the dict track_candidates returns."""
    return dict(n=len(rec), type=rec["type"].copy(), seed=rec["seed"].copy(), hits=rec["hits"].copy(),
                pt=rec["pt"].copy(), eta=rec["eta"].copy(), phi0=rec["phi0"].copy())


def _numel(a):
    return a.numel() if hasattr(a, "numel") else np.asarray(a).size


_INPUT_DTYPES = (("x", "float32"), ("y", "float32"), ("z", "float32"), ("module", "int32"), ("side", "uint8"),
                 ("seeds", "float32"))


def _on_device(a):
    return bool(getattr(a, "is_cuda", False))


def _contiguous(a):
    return a.is_contiguous() if hasattr(a, "is_contiguous") else bool(np.asarray(a).flags["C_CONTIGUOUS"])


def _input_kind(d, n_hits, n_seeds):
    """True when every input array of d (x, y, z, module, side, seeds) is a
    CUDA tensor, False when none is (numpy arrays or CPU tensors). Raises
    LstError, before anything is enqueued, for a mix of the two, a dtype other
    than the one the library reads, a non-contiguous array, or an array
    shorter than the n_hits hits (9 n_seeds floats for seeds) it must hold:
    the library reads these pointers without knowing their sizes."""
    kinds = set()
    for k, dt in _INPUT_DTYPES:
        a = d[k]
        kinds.add(_on_device(a))
        got = str(a.dtype).replace("torch.", "")
        if got != dt:
            raise LstError(f"{k}: dtype {got}, the library reads {dt}")
        if not _contiguous(a):
            raise LstError(f"{k}: not contiguous")
        need = 9 * int(n_seeds) if k == "seeds" else int(n_hits)
        if _numel(a) < need:
            raise LstError(f"{k}: {_numel(a)} elements, {need} needed")
    if len(kinds) > 1:
        raise LstError("the inputs mix host arrays and CUDA tensors")
    return kinds.pop()


def _device_array(t, name, dtype, shape):
    """Pointer of a contiguous CUDA tensor of the given dtype and shape;
    LstError otherwise (the library would read it on the device)."""
    if not _on_device(t):
        raise LstError(f"{name}: a CUDA tensor is required")
    got = str(t.dtype).replace("torch.", "")
    if got != dtype:
        raise LstError(f"{name}: dtype {got}, expected {dtype}")
    if not _contiguous(t):
        raise LstError(f"{name}: not contiguous")
    if tuple(t.shape) != tuple(shape):
        raise LstError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    return _ptr(t)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def default_config(overrides=None):
    c = LstConfig()
    _check(library().lst_config_default(C.byref(c)))
    for k, v in (overrides or {}).items():
        if any(k == f for f, _ in LstConfig._fields_):
            setattr(c, k, v)
    return c


def default_capacity(max_events=1, **overrides):
    k = LstCapacity()
    _check(library().lst_capacity_default(C.byref(k), int(max_events)))
    for n, v in overrides.items():
        setattr(k, n, int(v))
    return k


def measure_peaks(device=0):
    """The device's FP32/FP64 FMA and global atomic rates, measured by the
    library's calibration kernels (lst_measure_peaks), as a dict."""
    p = LstPeaks()
    _check(library().lst_measure_peaks(device, C.byref(p)))
    return {"fp32_tflops": p.fp32_tflops, "fp64_tflops": p.fp64_tflops, "atom_warp_gops": p.atom_warp_gops,
            "atom_same_gops": p.atom_same_gops, "red_lane_gops": p.red_lane_gops, "ms": list(p.ms),
            "sm_count": p.sm_count, "clock_mhz": p.clock_khz / 1000.0}


LST_MODULE_BYTES = C.sizeof(LstModule)


def _device_min(t, name, dtype, n):
    """Pointer of a contiguous CUDA tensor of the given dtype with at least n
    elements; LstError otherwise (the library reads or writes n elements of
    it on the device without knowing its size)."""
    if not _on_device(t):
        raise LstError(f"{name}: a CUDA tensor is required")
    got = str(t.dtype).replace("torch.", "")
    if got != dtype:
        raise LstError(f"{name}: dtype {got}, expected {dtype}")
    if not _contiguous(t):
        raise LstError(f"{name}: not contiguous")
    if _numel(t) < n:
        raise LstError(f"{name}: {_numel(t)} elements, {n} needed")
    return _ptr(t)


def build_mini_doublets_static(cfg, modules, n_mod, x, y, z, module, side, n_hits, md_capacity, md_lower,
                               md_upper, md_module, md_dphi, md_dlong, md_count, md_dropped=None, stream=None):
    """lst_build_mini_doublets_static: the allocation-free MD builder of one
    event. cfg is an LstConfig; every array is a contiguous CUDA tensor:
    modules holds the lst_module rows as bytes (uint8, n_mod rows); x, y, z
    float32, module int32 and side uint8 with n_hits elements; md_lower,
    md_upper, md_module int32 and md_dphi, md_dlong float32 with md_capacity
    elements; md_count and md_dropped (optional) one int32 each. Every array
    is checked before the call (LstError): the library reads and writes them
    by pointer. Asynchronous on `stream` (a cudaStream_t handle; None: the
    legacy default stream)."""
    n_mod, n_hits, md_capacity = int(n_mod), int(n_hits), int(md_capacity)
    if n_mod <= 0 or n_hits < 0 or md_capacity < 0:
        raise LstError("build_mini_doublets_static: n_mod > 0, n_hits >= 0 and md_capacity >= 0 are required")
    ptrs = [_device_min(modules, "modules", "uint8", n_mod * LST_MODULE_BYTES)]
    ptrs += [_device_min(a, k, dt, n_hits) for a, k, dt in ((x, "x", "float32"), (y, "y", "float32"),
                                                               (z, "z", "float32"), (module, "module", "int32"),
                                                               (side, "side", "uint8"))]
    ptrs += [_device_min(a, k, dt, md_capacity) for a, k, dt in ((md_lower, "md_lower", "int32"),
                                                                    (md_upper, "md_upper", "int32"),
                                                                    (md_module, "md_module", "int32"),
                                                                    (md_dphi, "md_dphi", "float32"),
                                                                    (md_dlong, "md_dlong", "float32"))]
    ptrs.append(_device_min(md_count, "md_count", "int32", 1))
    ptrs.append(_device_min(md_dropped, "md_dropped", "int32", 1) if md_dropped is not None else None)
    s = C.c_void_p(stream) if stream is not None else None
    _check(library().lst_build_mini_doublets_static(C.byref(cfg), ptrs[0], n_mod, *ptrs[1:6], n_hits, md_capacity,
                                                    *ptrs[6:], s))


def pack_events(events):
    """Concatenate per-event arrays (numpy) into one batch."""
    hit_off = np.zeros(len(events) + 1, np.int32)
    seed_off = np.zeros(len(events) + 1, np.int32)
    for i, ev in enumerate(events):
        hit_off[i + 1] = hit_off[i] + len(ev.x)
        seed_off[i + 1] = seed_off[i] + len(ev.seeds)
    cat = lambda name, dt: np.ascontiguousarray(np.concatenate([np.asarray(getattr(e, name), dt).ravel()
                                                                 for e in events]) if events else np.zeros(0, dt))
    return dict(x=cat("x", np.float32), y=cat("y", np.float32), z=cat("z", np.float32),
                module=cat("module", np.int32), side=cat("side", np.uint8), seeds=cat("seeds", np.float32),
                hit_off=hit_off, seed_off=seed_off)


class Context:
    """One library context: geometry resident on the device, one batch at a time."""

    def __init__(self, module_table, maps, cfg=None, capacity=None, device=0):
        L = library()
        self._cfg = cfg if isinstance(cfg, LstConfig) else default_config(cfg)
        self._cap = capacity if capacity is not None else default_capacity(1)
        h = C.c_void_p()
        _check(L.lst_create(C.byref(h), C.byref(self._cfg), C.byref(self._cap), int(device)))
        self._h = h
        n_mod = len(module_table["subdet"])
        mods = (LstModule * n_mod)()
        for i in range(n_mod):
            mods[i] = LstModule(int(module_table["subdet"][i]), int(module_table["layer"][i]),
                                float(module_table["dsep"][i]), float(module_table["sig_rphi"][i]),
                                float(module_table["sig_long"][i]))
        co, ct, so, st = [np.ascontiguousarray(a, np.int32) for a in maps]
        _check(L.lst_load_geometry(self._h, mods, n_mod, _ptr(co), _ptr(ct), _ptr(so), _ptr(st), len(so) - 1))
        self.n_events = 0
        self.event_ids = None
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            library().lst_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def capacity(self):
        return self._cap

    # -- running ----------------------------------------------------------
    def run_packed(self, b, stream=None, keep=False):
        """b: dict from pack_events (numpy) or the same keys as CUDA torch tensors
        (hit_off / seed_off stay numpy: they are host arrays). keep=True asks
        for event handles: the batch's track candidates and statistics stay
        readable through them across later runs until release(); the handles
        are returned (and kept in self.event_ids)."""
        dev = _input_kind(b, int(b["hit_off"][-1]), int(b["seed_off"][-1]))
        hits = LstHits(_ptr(b["x"]), _ptr(b["y"]), _ptr(b["z"]), _ptr(b["module"]), _ptr(b["side"]),
                       int(b["hit_off"][-1]))
        seeds = LstSeeds(_ptr(b["seeds"]), int(b["seed_off"][-1]))
        ho = np.ascontiguousarray(b["hit_off"], np.int32)
        so = np.ascontiguousarray(b["seed_off"], np.int32)
        self._keep = (b, ho, so)          # the library may read host inputs until the call returns
        s = C.c_void_p(stream) if stream is not None else None
        ids = (C.c_int64 * (len(ho) - 1))() if keep else None
        _check(library().lst_run_batch(self._h, C.byref(hits), _ptr(ho), C.byref(seeds), _ptr(so), len(ho) - 1,
                                       1 if dev else 0, s, ids))
        self.n_events = len(ho) - 1
        self.event_ids = list(ids) if keep else None
        return self.event_ids

    def run(self, events, stream=None, keep=False):
        return self.run_packed(pack_events(list(events)), stream, keep)

    def release(self, ids):
        """Release event handles (lst_release_event)."""
        for i in ids:
            _check(library().lst_release_event(self._h, int(i)))

    def run_events(self, events, stream=None, keep=False):
        """events: per-event dicts with x, y, z, module, side, seeds (numpy,
        pinned CPU tensors, or CUDA tensors; one kind for the whole batch).
        The library gathers them into its input staging (lst_run_events)."""
        n = len(events)
        hits = (LstHits * n)()
        seeds = (LstSeeds * n)()
        kinds = {_input_kind(e, _numel(e["x"]), _numel(e["seeds"]) // 9) for e in events}
        if len(kinds) > 1:
            raise LstError("the events mix host arrays and CUDA tensors")
        dev = kinds.pop() if kinds else False
        for i, e in enumerate(events):
            hits[i] = LstHits(_ptr(e["x"]), _ptr(e["y"]), _ptr(e["z"]), _ptr(e["module"]), _ptr(e["side"]),
                              int(len(e["x"])))
            seeds[i] = LstSeeds(_ptr(e["seeds"]), int(_numel(e["seeds"]) // 9))
        self._keep = (events, hits, seeds)
        s = C.c_void_p(stream) if stream is not None else None
        ids = (C.c_int64 * n)() if keep else None
        _check(library().lst_run_events(self._h, hits, seeds, n, 1 if dev else 0, s, ids))
        self.n_events = n
        self.event_ids = list(ids) if keep else None
        return self.event_ids

    def batch_track_candidates(self, out=None):
        """(offsets [n_events + 1], records) of the whole batch in two copies;
        records is a structured array (TC_DTYPE: type, seed, hits[10], pt, eta,
        phi0). out: a TC_DTYPE array to fill (its length is the capacity);
        without it the total is read first and an array of that size made."""
        L = library()
        off = np.zeros(self.n_events + 1, np.int32)
        if out is None:
            _check(L.lst_get_batch_track_candidates(self._h, 0, _ptr(off), None))
            out = np.empty(int(off[-1]), TC_DTYPE)
        cap = len(out)
        _check(L.lst_get_batch_track_candidates(self._h, cap, _ptr(off), _ptr(out) if cap else None))
        return off, out[:min(cap, int(off[-1]))]

    def _batch_args(self, b):
        dev = _input_kind(b, int(b["hit_off"][-1]), int(b["seed_off"][-1]))
        hits = LstHits(_ptr(b["x"]), _ptr(b["y"]), _ptr(b["z"]), _ptr(b["module"]), _ptr(b["side"]),
                       int(b["hit_off"][-1]))
        seeds = LstSeeds(_ptr(b["seeds"]), int(b["seed_off"][-1]))
        ho = np.ascontiguousarray(b["hit_off"], np.int32)
        so = np.ascontiguousarray(b["seed_off"], np.int32)
        return hits, ho, seeds, so, dev

    # -- launch shapes ----------------------------------------------------
    def launch_config(self):
        """[{name, blocks_per_sm, block, tunable, generic}] for every stage of the chain."""
        L = library()
        out = []
        for i in range(L.lst_launch_stage_count()):
            nm = C.c_char_p()
            m, b, f = C.c_int32(), C.c_int32(), C.c_int32()
            _check(L.lst_get_launch_config(self._h, i, C.byref(nm), C.byref(m), C.byref(b), C.byref(f)))
            out.append(dict(name=nm.value.decode(), blocks_per_sm=m.value, block=b.value,
                            tunable=bool(f.value & 1), generic=bool(f.value & 2)))
        return out

    def set_compact_storage(self, enable=True):
        """16-bit copies for the searches' curvature prefilters and the cleaning's eta-phi lists
        (lst_set_compact_storage); the objects do not change."""
        _check(library().lst_set_compact_storage(self._h, 1 if enable else 0))

    def set_fp64_fit(self, enable=True):
        """Refine fits in FP64 instead of float-float on the FP32 pipe (lst_set_fp64_fit)."""
        _check(library().lst_set_fp64_fit(self._h, 1 if enable else 0))

    def set_stage_limits(self, t5=0, pt=0):
        """Survivors a T5 / pT work item stages before re-enumerating (0: the defaults 512 / 256)."""
        _check(library().lst_set_stage_limits(self._h, int(t5), int(pt)))

    def set_launch_config(self, stage, blocks_per_sm=0, block=0):
        """stage: index or name; 0 restores a default."""
        if isinstance(stage, str):
            stage = [c["name"] for c in self.launch_config()].index(stage)
        _check(library().lst_set_launch_config(self._h, int(stage), int(blocks_per_sm), int(block)))

    def autotune(self, batch, reps=3, stream=None):
        """Tune every stage's launch shape on a batch (list of events or a
        pack_events dict); returns (summed stage ms before, after)."""
        b = batch if isinstance(batch, dict) else pack_events(list(batch))
        hits, ho, so_h, so, dev = self._batch_args(b)
        before, after = C.c_float(), C.c_float()
        s = C.c_void_p(stream) if stream is not None else None
        _check(library().lst_autotune(self._h, C.byref(hits), _ptr(ho), C.byref(so_h), _ptr(so), len(ho) - 1,
                                      1 if dev else 0, s, int(reps), C.byref(before), C.byref(after)))
        self.n_events = len(ho) - 1
        return before.value, after.value

    @property
    def launch_count(self):
        return library().lst_last_launch_count(self._h)

    def set_profiling(self, on=True):
        _check(library().lst_set_profiling(self._h, 1 if on else 0))

    def kernel_times(self):
        """[(name, ms)] of every launch of the last batch (profiling must be on)."""
        L = library()
        n = C.c_int32(0)
        names = (C.c_char_p * 64)()
        ms = np.zeros(64, np.float32)
        _check(L.lst_get_kernel_times(self._h, 64, C.byref(n), names, _ptr(ms)))
        return [(names[i].decode(), float(ms[i])) for i in range(n.value)]

    # -- results ----------------------------------------------------------
    def done(self):
        """Non-blocking: has the last batch finished on the device?"""
        return _check(library().lst_query(self._h)) == 1

    @property
    def device_bytes(self):
        return int(library().lst_device_bytes(self._h))

    def set_t5_selection(self, mlp=None, threshold=0.5, prefilter_scale=1.0, capture_features=False):
        """Network-scored T5 selection (mlp: an Mlp) or the hand-set cuts (mlp=None)."""
        self._mlp = mlp
        _check(library().lst_set_t5_selection(self._h, mlp._h if mlp is not None else None, float(threshold),
                                              float(prefilter_scale), 1 if capture_features else 0))

    def set_t3_selection(self, mlp=None, threshold=0.5, capture_features=False):
        """Network pruning of triplets before the T5 and pT3 searches (mlp: an Mlp), or none (mlp=None);
        capture_features computes the triplet features without a network (training)."""
        self._mlp3 = mlp
        _check(library().lst_set_t3_selection(self._h, mlp._h if mlp is not None else None, float(threshold),
                                              1 if capture_features else 0))

    def t3_candidates(self, event=0, features=True):
        """Every T3 of an event: features [n, 48] (when computed), hits [n, 6], score [n] (with a network),
        kept [n]."""
        L = library()
        n = C.c_int32(0)
        _check(L.lst_get_t3_candidates(self._h, int(event), 0, C.byref(n), None, None, None, None))
        k = n.value
        f = np.zeros((k, 48), np.float32) if features else None
        h = np.zeros((k, 6), np.int32)
        has_net = getattr(self, "_mlp3", None) is not None
        sc = np.zeros(k, np.float32) if has_net else None
        kept = np.zeros(k, np.int32)
        _check(L.lst_get_t3_candidates(self._h, int(event), k, C.byref(n), _ptr(f), _ptr(h), _ptr(sc), _ptr(kept)))
        return dict(features=f, hits=h, score=sc, kept=kept.astype(bool))

    def t5_candidates(self, event=0):
        """Every T5 candidate of an event: features [n, 48], hits [n, 10], cut_pass [n], score [n]."""
        L = library()
        n = C.c_int32(0)
        _check(L.lst_get_t5_candidates(self._h, int(event), 0, C.byref(n), None, None, None, None))
        k = n.value
        f = np.zeros((k, 48), np.float32)
        h = np.zeros((k, 10), np.int32)
        cp = np.zeros(k, np.int32)
        sc = np.zeros(k, np.float32)
        _check(L.lst_get_t5_candidates(self._h, int(event), k, C.byref(n), _ptr(f), _ptr(h), _ptr(cp), _ptr(sc)))
        return dict(features=f, hits=h, cut_pass=cp.astype(bool), score=sc)

    def counters(self):
        """Batch-wide device counters (see lst_get_counters)."""
        out = np.zeros(32, np.int32)
        _check(library().lst_get_counters(self._h, _ptr(out), 32))
        return out

    def stats(self, event=0):
        s = LstStats()
        _check(library().lst_get_stats(self._h, int(event), C.byref(s)))
        return dict(counts=dict(zip(STAT_NAMES, list(s.counts))), dropped=dict(zip(STAT_NAMES, list(s.dropped))))

    def track_candidates(self, event=0):
        L = library()
        n = C.c_int32(0)
        _check(L.lst_get_track_candidates(self._h, int(event), 0, C.byref(n), None, None, None, None))
        k = n.value
        t = np.zeros(k, np.int32)
        sd = np.zeros(k, np.int32)
        h = np.zeros((k, 10), np.int32)
        f = np.zeros((k, 3), np.float32)
        _check(L.lst_get_track_candidates(self._h, int(event), k, C.byref(n), _ptr(t), _ptr(sd), _ptr(h), _ptr(f)))
        return dict(n=k, type=t, seed=sd, hits=h, pt=f[:, 0], eta=f[:, 1], phi0=f[:, 2])

    def objects(self, kind, event=0):
        L = library()
        code = KIND_NAMES.index(kind)
        ni, nf = C.c_int32(), C.c_int32()
        _check(L.lst_object_columns(code, C.byref(ni), C.byref(nf)))
        n = C.c_int32(0)
        _check(L.lst_get_objects(self._h, int(event), code, 0, C.byref(n), None, None))
        I = np.zeros((n.value, ni.value), np.int32)
        F = np.zeros((n.value, nf.value), np.float32)
        _check(L.lst_get_objects(self._h, int(event), code, n.value, C.byref(n), _ptr(I), _ptr(F)))
        icol, fcol = COLUMNS[kind]
        rec = {c: I[:, j] for j, c in enumerate(icol)}
        rec.update({c: F[:, j] for j, c in enumerate(fcol)})
        rec["n"] = n.value
        return rec


N_MLP_PARAMS = 9409
N_MLP_INPUTS = 48


class Mlp:
    """The T5 scoring network on a device (parameters, inference, training)."""

    def __init__(self, device=0, max_batch=4096, params=None):
        h = C.c_void_p()
        _check(library().lst_mlp_create(C.byref(h), int(device), int(max_batch)))
        self._h = h
        self.max_batch = max_batch
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "_h", None):
            library().lst_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == N_MLP_PARAMS
        _check(library().lst_mlp_set_params(self._h, _ptr(p)))

    def params(self):
        p = np.zeros(N_MLP_PARAMS, np.float32)
        _check(library().lst_mlp_get_params(self._h, _ptr(p)))
        return p

    def state(self):
        """Training state for a checkpoint: params, Adam moments m and v, step."""
        p, m, v = (np.zeros(N_MLP_PARAMS, np.float32) for _ in range(3))
        step = C.c_int64(0)
        _check(library().lst_mlp_get_state(self._h, _ptr(p), _ptr(m), _ptr(v), C.byref(step)))
        return dict(params=p, m=m, v=v, step=int(step.value))

    def set_state(self, st):
        arr = [np.ascontiguousarray(st[k], np.float32) for k in ("params", "m", "v")]
        for a in arr:
            if a.size != N_MLP_PARAMS:
                raise LstError(f"state arrays hold {N_MLP_PARAMS} floats, not {a.size}")
        _check(library().lst_mlp_set_state(self._h, *[_ptr(a) for a in arr], int(st["step"])))

    def forward(self, features, scores, stream=None):
        """features, scores: CUDA tensors ([n, 48] float32, [n] float32)."""
        n = int(features.shape[0])
        f = _device_array(features, "features", "float32", (n, N_MLP_INPUTS))
        o = _device_array(scores, "scores", "float32", (n,))
        _check(library().lst_mlp_forward(self._h, f, n, o, C.c_void_p(stream) if stream is not None else None))

    def gradient(self, features, labels, stream=None):
        g = np.zeros(N_MLP_PARAMS, np.float32)
        loss = C.c_float(0)
        n = int(features.shape[0])
        f = _device_array(features, "features", "float32", (n, N_MLP_INPUTS))
        y = _device_array(labels, "labels", "float32", (n,))
        _check(library().lst_mlp_gradient(self._h, f, y, n, _ptr(g), C.byref(loss),
                                          C.c_void_p(stream) if stream is not None else None))
        return g, loss.value

    def train_step(self, features, labels, lr=1e-3, want_loss=False, stream=None):
        loss = C.c_float(0)
        n = int(features.shape[0])
        f = _device_array(features, "features", "float32", (n, N_MLP_INPUTS))
        y = _device_array(labels, "labels", "float32", (n,))
        _check(library().lst_mlp_train_step(self._h, f, y, n, float(lr), C.byref(loss) if want_loss else None,
                                            C.c_void_p(stream) if stream is not None else None))
        return loss.value if want_loss else None
