"""The command-line entry points (GPU): a network trained and saved by `train`
attaches to the chain through `run --t3-net` / `run --t5-net`, and prunes the
objects it scores."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _last_json(capsys):
    return json.loads(capsys.readouterr().out.strip().splitlines()[-1])


def _run(capsys, *extra):
    from paper_2209_13711_gb300 import run
    run.main(["--events", "1", "--repeat", "1", "--seed", "3", *extra])
    return _last_json(capsys)


@pytest.mark.parametrize("kind", ["t3", "t5"])
def test_trained_network_attaches_through_run(tmp_path, capsys, kind):
    from paper_2209_13711_gb300 import lst, train
    out = str(tmp_path / f"{kind}.npz")
    train.main(["--kind", kind, "--train-events", "2", "--eval-events", "1", "--epochs", "1", "--out", out])
    res = _last_json(capsys)
    z = np.load(out)
    assert z["params"].shape == (lst.N_MLP_PARAMS,) and np.all(np.isfinite(z["params"]))
    assert float(z["threshold"]) == pytest.approx(res["threshold"])
    base = _run(capsys)
    net = _run(capsys, f"--{kind}-net", out)
    assert net["objects"]["tc"] > 0
    assert sum(net["dropped"].values()) == 0
    assert net["objects"]["t3"] == base["objects"]["t3"]      # both networks act after the T3 stage
    assert net["objects"]["t5"] > 0
    if kind == "t3":
        assert net["objects"]["t5"] < base["objects"]["t5"]    # pruned triplets build no quintuplets
