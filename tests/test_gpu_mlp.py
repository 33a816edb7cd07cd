"""Scoring network on the GPU vs its FP64 reference, and its use in the chain (GPU)."""
import numpy as np
import pytest

from oracle import mlp_oracle as R
from synth import events as E
from synth.config import DEFAULT_CUTS
from synth.mlp_init import init_params
from tests.gpu_common import make_context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, 48)).astype(np.float32)
    X[:, 38:] = 0
    y = (rng.uniform(size=n) < 0.3).astype(np.float32)
    return X, y


@pytest.fixture(scope="module")
def mlp():
    import paper_2209_13711_gb300 as P
    m = P.Mlp(max_batch=4096, params=init_params(7))
    yield m
    m.close()


@pytest.mark.parametrize("n", [1, 17, 1003])
def test_forward_matches_reference(mlp, n):
    X, _ = _data(n, n)
    theta = init_params(7)
    mlp.set_params(theta)
    out = torch.zeros(n, device="cuda")
    mlp.forward(torch.from_numpy(X).cuda(), out)
    torch.cuda.synchronize()
    ref, _ = R.forward(theta.astype(np.float64), X)
    d = np.abs(out.cpu().numpy() - ref)
    # FP32 vs FP64 accumulation may round a hidden activation to the neighbouring
    # BF16 value (2^-8 relative): rare, and bounded well below 5e-3 on the score
    assert d.max() <= 5e-3 and np.mean(d <= 2e-4) >= 0.99 and d.mean() <= 1e-4


def test_gradient_matches_reference(mlp):
    X, y = _data(3000, 11)
    theta = init_params(8)
    mlp.set_params(theta)
    g, loss = mlp.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    gr = R.grad(theta.astype(np.float64), X, y)
    assert abs(loss - R.loss(theta.astype(np.float64), X, y)) < 1e-4
    assert np.linalg.norm(g - gr) <= 1e-2 * np.linalg.norm(gr)
    big = np.abs(gr) > 1e-2 * np.abs(gr).max()
    assert np.allclose(g[big], gr[big], rtol=3e-2, atol=1e-6)


def test_adam_step_matches_reference(mlp):
    X, y = _data(2048, 12)
    theta = init_params(9)
    mlp.set_params(theta)
    mlp.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), lr=1e-3)
    got = mlp.params()
    gr = R.grad(theta.astype(np.float64), X, y)
    want, _, _ = R.adam(theta.astype(np.float64), 0, 0, gr, 1, lr=1e-3)
    big = np.abs(gr) > 1e-2 * np.abs(gr).max()
    assert np.allclose(got[big], want[big], atol=2e-6)
    assert np.all(np.abs(got - theta) <= 1e-3 * 1.0001)


def test_training_reduces_the_loss(mlp):
    X, y = _data(4096, 13)
    y = (X[:, 0] + 0.5 * X[:, 3] > 0.2).astype(np.float32)      # a learnable rule
    mlp.set_params(init_params(10))
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    l0 = mlp.train_step(Xd, yd, lr=3e-3, want_loss=True)
    for _ in range(300):
        mlp.train_step(Xd, yd, lr=3e-3)
    l1 = mlp.train_step(Xd, yd, lr=3e-3, want_loss=True)
    assert l1 < 0.3 * l0


def test_chain_features_match_oracle(geom_full, maps_full):
    from oracle import oracle as O
    ctx = make_context(geom_full, maps_full, max_events=1)
    ctx.set_t5_selection(None, capture_features=True)
    ev = E.pileup_event(30, 77, geom_full)
    ctx.run([ev])
    cand = ctx.t5_candidates(0)
    assert len(cand["hits"]) > 50
    S = O.Setup(geom_full.module_table(), maps_full, DEFAULT_CUTS, ev)
    for i in range(0, len(cand["hits"]), max(1, len(cand["hits"]) // 200)):
        want = S.t5_features(cand["hits"][i])
        got = cand["features"][i].astype(np.float64)
        assert np.all(np.abs(got - want) <= 1e-5 * np.maximum(np.abs(want), 1.0)), i
    ctx.close()


def test_chain_with_the_network(geom_full, maps_full):
    import paper_2209_13711_gb300 as P
    m = P.Mlp(max_batch=64, params=init_params(3))
    ctx = make_context(geom_full, maps_full, max_events=1)
    ev = E.pileup_event(30, 78, geom_full)
    ctx.set_t5_selection(m, threshold=0.0, prefilter_scale=2.0)
    ctx.run([ev])
    st = ctx.stats(0)
    cand = ctx.t5_candidates(0)
    kappa_ok = np.abs(cand["features"][:, 27]) <= 1.05 + 1e-6
    assert st["counts"]["t5"] == int(kappa_ok.sum()) > 0
    # scores are the network's on the captured features
    ref, _ = R.forward(init_params(3).astype(np.float64), cand["features"])
    d = np.abs(cand["score"] - ref)
    assert d.max() <= 5e-3 and np.mean(d <= 2e-4) >= 0.99
    ctx.set_t5_selection(m, threshold=1.5, prefilter_scale=2.0)
    ctx.run([ev])
    assert ctx.stats(0)["counts"]["t5"] == 0
    ctx.set_t5_selection(None)
    ctx.run([ev])
    assert ctx.stats(0)["counts"]["t5"] == int(cand["cut_pass"].sum())
    ctx.close()
    m.close()


def test_trained_network_beats_the_cuts(geom_full):
    """At the cut-based efficiency, the trained network keeps far fewer fakes."""
    import paper_2209_13711_gb300 as P
    from paper_2209_13711_gb300 import train as T
    from synth import maps as M
    ctx = P.Context(geom_full.module_table(), M.load_maps(geom_full), cfg=DEFAULT_CUTS,
                    capacity=P.default_capacity(8))
    ctx.set_t5_selection(None, prefilter_scale=3.0, capture_features=True)
    tr = T.collect(ctx, [E.pu200_event(30000 + i, geom_full) for i in range(8)], batch=8)
    va = T.collect(ctx, [E.pu200_event(31000 + i, geom_full) for i in range(3)], batch=8)
    m = P.Mlp(max_batch=4096, params=init_params(1))
    T.train(m, tr["X"], tr["y"], epochs=3)
    res = T.evaluate(m, va)
    assert res["network"]["efficiency"] >= res["cut"]["efficiency"]
    assert res["network"]["fake_rate"] < 0.5 * res["cut"]["fake_rate"]
    ctx.close()
    m.close()


def test_resume_from_checkpoint_matches_uninterrupted_training(tmp_path):
    """Two epochs in one run against one epoch, a checkpoint (parameters, Adam moments and step) into a fresh
    network, and the second epoch: identical parameters and moments. Resuming from the parameters alone (Adam
    reset) ends elsewhere, so the moments are what the checkpoint must carry."""
    torch = pytest.importorskip("torch")
    import paper_2209_13711_gb300 as P
    from paper_2209_13711_gb300 import train as T
    rng = np.random.default_rng(3)
    n = 4096 * 6
    X = rng.normal(0.0, 1.0, (n, 48)).astype(np.float32)
    X[:, 38:] = 0.0
    y = (X[:, 0] + 0.5 * X[:, 3] - X[:, 7] > 0).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()

    full = P.Mlp(max_batch=4096, params=init_params(2))
    T.train(full, Xd, y, epochs=2, seed=5)
    want = full.state()

    first = P.Mlp(max_batch=4096, params=init_params(2))
    ck = str(tmp_path / "ck.npz")
    T.train(first, Xd, y, epochs=1, seed=5, checkpoint=ck)
    resumed = P.Mlp(max_batch=4096)
    done, hist = T.load_checkpoint(ck, resumed)
    assert done == 1 and len(hist) == 1
    T.train(resumed, Xd, y, epochs=2, seed=5, start_epoch=done, hist=hist)
    got = resumed.state()
    assert got["step"] == want["step"] == 12
    for k in ("params", "m", "v"):
        assert np.array_equal(got[k], want[k]), k

    reset = P.Mlp(max_batch=4096, params=np.load(ck)["params"])
    T.train(reset, Xd, y, epochs=2, seed=5, start_epoch=1)
    assert not np.array_equal(reset.params(), want["params"])


def test_t3_features_match_the_oracle(geom_full, maps_full):
    """FP32 triplet features on the device against the FP64 oracle's, for a sample of an event's T3s."""
    from oracle import oracle as O
    ev = E.pileup_event(60, 8, geom_full)
    ctx = make_context(geom_full, maps_full, max_events=1)
    ctx.set_t3_selection(None, capture_features=True)
    ctx.run([ev])
    c = ctx.t3_candidates(0)
    assert len(c["hits"]) > 10000 and c["kept"].all()
    S = O.Setup(geom_full.module_table(), maps_full, DEFAULT_CUTS, ev)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(c["hits"]), 400, replace=False):
        want = S.t3_features(c["hits"][i])
        got = c["features"][i]
        assert np.all(np.abs(got - want) <= 0.02 + 2e-3 * np.abs(want)), (i, np.nonzero(
            np.abs(got - want) > 0.02 + 2e-3 * np.abs(want))[0])
    ctx.close()


def test_t3_network_prunes_triplets_and_keeps_the_track_candidates(geom_full, maps_full):
    """A network trained on 6 PU200 events' triplets, at the threshold that keeps 99 % of true T3s, prunes
    most of the fake ones; the T5 searches then see fewer candidates and the track-candidate efficiency on
    other events stays within 1 % of the hand-set cuts' alone."""
    import paper_2209_13711_gb300 as P
    from paper_2209_13711_gb300 import metrics as MT
    from paper_2209_13711_gb300 import train as T
    ctx = make_context(geom_full, maps_full, max_events=2)
    ctx.set_t3_selection(None, capture_features=True)
    tr = T.collect_t3(ctx, [E.pu200_event(40000 + i, geom_full) for i in range(6)], batch=2, max_per_event=150000)
    va = T.collect_t3(ctx, [E.pu200_event(41000 + i, geom_full) for i in range(2)], batch=2, device=False)
    m = P.Mlp(max_batch=4096, params=init_params(4))
    T.train(m, tr["X"], tr["y"], epochs=3)
    s = T.scores_of(m, va["X"])
    thr = T.threshold_keeping(s, va["y"], 0.99)
    fake = va["y"] < 0.5
    pruned = float(np.mean(s[fake] < thr))
    assert pruned > 0.5, pruned
    evs = [E.pu200_event(42000 + i, geom_full) for i in range(2)]
    res = {}
    for mode in ("cuts", "network"):
        ctx.set_t3_selection(m if mode == "network" else None, threshold=thr)
        ctx.run(evs)
        rates = [MT.rates(ctx.track_candidates(e), ev.pid, ev.seed_pid, ev.tracks) for e, ev in enumerate(evs)]
        res[mode] = (MT.combine(rates), int(ctx.counters()[21]))
    assert res["network"][0]["efficiency"] >= res["cuts"][0]["efficiency"] - 0.01
    assert res["network"][1] < 0.8 * res["cuts"][1]           # T5 search survivors
    ctx.close()
