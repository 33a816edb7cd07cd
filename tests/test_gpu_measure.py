"""Measurement support on the device (GPU): the calibration probes give
plausible rates, and the candidate-test counts of the device objects equal
those of the oracle's objects."""
import pytest

from paper_2209_13711_gb300 import measure_peaks
from paper_2209_13711_gb300.metrics import candidate_tests
from synth import events as E
from tests.gpu_common import gpu_result, make_context, oracle_result

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    p = measure_peaks(0)
    assert p["sm_count"] > 0
    assert all(m > 0 for m in p["ms"])
    # a GB300-class part: tens of FP32 TFLOP/s, FP64 far below FP32
    assert 10.0 < p["fp32_tflops"] < 400.0
    assert 0.05 < p["fp64_tflops"] < p["fp32_tflops"]
    assert p["atom_warp_gops"] > 0.05 and p["atom_same_gops"] > 0.005 and p["red_lane_gops"] > 0.5


def test_candidate_tests_of_device_objects_equal_oracle(geom_full, maps_full):
    ev = E.pileup_event(20, 5, geom_full)
    ctx = make_context(geom_full, maps_full)
    try:
        ctx.run([ev])
        dev = gpu_result(ctx, 0)
    finally:
        ctx.close()
    ref = oracle_result(geom_full, maps_full, ev)
    n_mod = len(maps_full[0]) - 1
    got = candidate_tests(dev, ev.module, ev.side, *maps_full, n_mod)
    want = candidate_tests(ref, ev.module, ev.side, *maps_full, n_mod)
    assert got == want
    assert all(v > 0 for v in got.values())
