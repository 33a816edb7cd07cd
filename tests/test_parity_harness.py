"""The parity harness accepts identical results and rejects planted mistakes (CPU)."""
import copy

import numpy as np
import pytest

from synth import events as E
from synth.config import DEFAULT_CUTS
from tests.gpu_common import A_HALF, oracle_result
from tests.parity import compare


@pytest.fixture(scope="module")
def res(geom_full, maps_full):
    return oracle_result(geom_full, maps_full, E.pileup_event(30, 5, geom_full))


def test_identity_passes(res):
    s = compare(res, res, A_HALF, DEFAULT_CUTS)
    assert s["tc"][0] == res["tc"]["n"]


def _drop(rec, i):
    out = {}
    for k, v in rec.items():
        out[k] = np.delete(v, i) if isinstance(v, np.ndarray) and v.ndim >= 1 and len(v) == rec["n"] else v
    out["n"] = rec["n"] - 1
    return out


def test_missing_t5_is_caught(res):
    bad = copy.deepcopy(res)
    # remove the last T5 (nothing downstream indexes it beyond the dropped row if no pT5 uses it)
    used = set(bad["pt5"]["t5"].tolist())
    i = next(j for j in range(bad["t5"]["n"] - 1, -1, -1) if j not in used)
    keep = np.arange(bad["t5"]["n"]) != i
    for k in list(bad["t5"]):
        if isinstance(bad["t5"][k], np.ndarray):
            bad["t5"][k] = bad["t5"][k][keep]
    bad["t5"]["n"] -= 1
    remap = np.cumsum(keep) - 1
    bad["pt5"]["t5"] = remap[bad["pt5"]["t5"]]
    with pytest.raises(AssertionError):
        compare(bad, res, A_HALF, DEFAULT_CUTS, check_tc=False)


def test_perturbed_value_is_caught(res):
    bad = copy.deepcopy(res)
    bad["md"]["dphi"] = bad["md"]["dphi"].copy()
    bad["md"]["dphi"][7] += 1e-4 * bad["md"]["thr_phi"][7]
    with pytest.raises(AssertionError):
        compare(bad, res, A_HALF, DEFAULT_CUTS, check_tc=False)


def test_missing_candidate_is_caught(res):
    bad = copy.deepcopy(res)
    bad["tc"] = _drop(bad["tc"], 0)
    with pytest.raises(AssertionError):
        compare(bad, res, A_HALF, DEFAULT_CUTS)
