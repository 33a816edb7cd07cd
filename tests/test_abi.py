"""CPU checks of the C ABI: the library loads and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lst_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lst_load_geometry", "lst_run_event", "lst_run_batch", "lst_get_track_candidates", "lst_create",
              "lst_destroy", "lst_get_objects", "lst_get_stats", "lst_release_event", "lst_status_str"):
        assert n in names


def test_result_slot_count_matches_the_header():
    from paper_2209_13711_gb300 import lst
    src = open(os.path.join(ROOT, "include", "lst.h")).read()
    assert int(re.search(r"#define LST_RESULT_SLOTS (\d+)", src).group(1)) == lst.LST_RESULT_SLOTS


def test_setters_refuse_a_null_context_without_device():
    """The context setters answer LST_ERR_ARG for a missing context before touching a device."""
    from paper_2209_13711_gb300 import lst
    L = lst.library()
    assert L.lst_set_fp64_fit(None, 1) == -1
    assert L.lst_set_compact_storage(None, 1) == -1


def test_release_refuses_indices_and_null_without_device():
    from paper_2209_13711_gb300 import lst
    L = lst.library()
    assert L.lst_release_event(None, 1 << 40) == -1
    assert L.lst_release_event(None, 0) == -1


def test_library_exports_every_symbol():
    from paper_2209_13711_gb300 import build
    lib = ctypes.CDLL(build.build())
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_config_defaults_match_input_constants():
    from paper_2209_13711_gb300 import lst
    from synth.config import DEFAULT_CUTS
    c = lst.default_config()
    for f, _ in lst.LstConfig._fields_:
        assert getattr(c, f) == pytest.approx(DEFAULT_CUTS[f]), f


def test_argument_errors_without_device():
    from paper_2209_13711_gb300 import lst
    L = lst.library()
    assert L.lst_create(None, None, None, 0) == -1
    assert L.lst_config_default(None) == -1
    assert L.lst_capacity_default(None, 1) == -1
    ni, nf = ctypes.c_int32(), ctypes.c_int32()
    assert L.lst_object_columns(7, ctypes.byref(ni), ctypes.byref(nf)) == -1
    assert L.lst_object_columns(3, ctypes.byref(ni), ctypes.byref(nf)) == 0 and (ni.value, nf.value) == (2, 7)
    assert L.lst_status_str(-6) == b"batch exceeds the context capacity"


def test_static_md_builder_binding_checks_arguments_without_device():
    """The binding refuses host arrays before any device work, and the library
    answers a missing pointer with LST_ERR_ARG (no CUDA call is made)."""
    import numpy as np
    from paper_2209_13711_gb300 import LstError, build_mini_doublets_static, lst
    cfg = lst.default_config()
    host = np.zeros(4, np.float32)
    with pytest.raises(LstError, match="CUDA tensor"):
        build_mini_doublets_static(cfg, host, 1, host, host, host, host, host, 4, 4, host, host, host, host, host,
                                   host)
    L = lst.library()
    assert L.lst_build_mini_doublets_static(ctypes.byref(cfg), None, 1, *([None] * 5), 0, 0, *([None] * 7),
                                            None) == -1
