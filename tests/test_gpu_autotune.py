"""Launch shapes and the autotuner: results do not depend on the shape (GPU)."""
import pytest

from paper_2209_13711_gb300 import LstError
from synth import events as E
from tests.gpu_common import all_tuples, make_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch(geom_full):
    return [E.pileup_event(pu, 300 + i, geom_full) for i, pu in enumerate((40, 90, 8))]


@pytest.fixture(scope="module")
def reference(geom_full, maps_full, batch):
    ctx = make_context(geom_full, maps_full, max_events=4)
    ctx.run(batch)
    ref = [all_tuples(ctx, i) for i in range(len(batch))]
    ctx.close()
    return ref


def test_launch_config_validation(geom_full, maps_full):
    ctx = make_context(geom_full, maps_full, max_events=1)
    cfg = ctx.launch_config()
    names = [c["name"] for c in cfg]
    assert names[:4] == ["reset", "bin_count", "bin_scan", "bin_scatter"] and names[-1] == "tc_pack"
    assert {"md", "ls", "t3", "t5", "pt5", "pt3", "clean_pls"} <= set(names)
    byname = {c["name"]: c for c in cfg}
    assert not byname["bin_scan"]["tunable"]
    assert byname["t5_gather"]["tunable"] and not byname["t5_gather"]["generic"]
    assert byname["t5"]["tunable"] and not byname["t5"]["generic"]
    assert byname["t5_refine"]["generic"]
    for bad in [("md", 0, 256), ("bin_scan", 2, 0), ("t5_refine", 0, 48), ("t5_refine", 0, 2048),
                ("ls", -1, 0), ("ls", 65, 0)]:
        with pytest.raises(LstError):
            ctx.set_launch_config(*bad)
    with pytest.raises(LstError):
        ctx.set_launch_config(len(cfg), 1, 0)
    ctx.set_launch_config("t5", 3, 0)
    assert {c["name"]: c for c in ctx.launch_config()}["t5"]["blocks_per_sm"] == 3
    ctx.set_launch_config("t5", 0, 0)
    assert {c["name"]: c for c in ctx.launch_config()}["t5"]["blocks_per_sm"] == byname["t5"]["blocks_per_sm"]
    ctx.close()


@pytest.mark.parametrize("bpsm,block", [(1, 64), (16, 512), (3, 96)])
def test_results_independent_of_launch_shape(geom_full, maps_full, batch, reference, bpsm, block):
    ctx = make_context(geom_full, maps_full, max_events=4)
    for c in ctx.launch_config():
        if c["tunable"]:
            try:
                ctx.set_launch_config(c["name"], bpsm, block if c["generic"] else 0)
            except LstError:          # a block the kernel cannot launch
                ctx.set_launch_config(c["name"], bpsm, 0)
    ctx.run(batch)
    for i in range(len(batch)):
        assert all_tuples(ctx, i) == reference[i]
    ctx.close()


def test_autotune_keeps_results(geom_full, maps_full, batch, reference):
    ctx = make_context(geom_full, maps_full, max_events=4)
    before, after = ctx.autotune(batch, reps=1)
    assert before > 0 and after > 0
    # the per-stage choice never takes a shape slower than the default, up to timing noise
    assert after <= 1.25 * before
    for i in range(len(batch)):
        assert all_tuples(ctx, i) == reference[i]       # results of the last tuning run
    ctx.run(batch)                                        # graph captured with the tuned shapes
    for i in range(len(batch)):
        assert all_tuples(ctx, i) == reference[i]
    ctx.close()
