"""Host logic of the occupancy study (CPU): per-module counts follow each
object's innermost MD, and slot memory is modules x cap x bytes."""
import numpy as np

from paper_2209_13711_gb300.occupancy import module_occupancy, slot_bytes


def test_module_occupancy_uses_the_innermost_md():
    obj = {"md": {"mod": np.array([0, 2, 2, 3])},
           "ls": {"md_in": np.array([0, 1, 2, 2]), "md_out": np.array([1, 3, 3, 3])},
           "t3": {"ls_in": np.array([0, 2, 3]), "ls_out": np.array([1, 1, 1])},
           "t5": {"t3_in": np.array([1, 2]), "t3_out": np.array([0, 0])}}
    occ = module_occupancy(obj, 4)
    assert occ["md"].tolist() == [1, 0, 2, 1]
    assert occ["ls"].tolist() == [1, 0, 3, 0]
    assert occ["t3"].tolist() == [1, 0, 2, 0]
    assert occ["t5"].tolist() == [0, 0, 2, 0]


def test_slot_bytes_at_quantiles():
    occ = {k: np.array([[0, 1, 2, 3], [4, 5, 6, 7]]) for k in ("md", "ls", "t3", "t5")}
    r = slot_bytes(occ, {"md": 10, "ls": 1, "t3": 1, "t5": 1}, (100,))["q100"]
    assert r["caps_per_module"]["md"] == 7
    assert r["bytes_per_event"] == 4 * 7 * (10 + 1 + 1 + 1)
    assert r["modules_over_cap_frac"]["t3"] == 0.0
