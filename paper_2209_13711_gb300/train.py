"""Training and evaluation of the T5 scoring network on the device.

The chain runs with feature capture and a widened T5 prefilter; every T5
candidate of the training events becomes a sample (features from the FP64
refine kernel, label 1 when all ten hits come from one generated particle).
The network is trained with the library's own forward, backward and Adam
kernels. Evaluation compares, on separate events, the hand-set cut selection
with the network at the threshold that matches the cut efficiency.

    python -m paper_2209_13711_gb300.train --train-events 100 --eval-events 8 --out t5_mlp.npz
    python -m paper_2209_13711_gb300.train --kind t3 --train-events 16 --eval-events 4 --out t3_mlp.npz

A T5 file holds the parameters and the threshold that matches the cut
efficiency (`run --t5-net` attaches it). --kind t3 trains the learned triplet
selection instead: every T3 of the training events is a sample (label 1 when
its six hits come from one particle), and the saved file holds the parameters
and the threshold that keeps 99 % of the true T3s of the evaluation events
(`run --t3-net` attaches it).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import lst as L


def label_candidates(cand, pid):
    """1 when all ten hits of a candidate belong to one generated particle."""
    h = cand["hits"]
    p = pid[h]
    true = (p[:, 0] >= 0) & np.all(p == p[:, :1], axis=1)
    return true, np.where(true, p[:, 0], -1)


def collect(ctx, events, batch=16, stream=None, device=False):
    """Features, labels, cut decisions and particle ids of every T5 candidate.

    events: a list of events or an iterable of them (a generator keeps only one
    batch of events on the host). device=True moves each event's features to
    the GPU as it is read, so the training set is held in device memory and
    the host holds one event's features at a time."""
    import itertools
    X, y, cut, part, ev_idx = [], [], [], [], []
    it, b0 = iter(events), 0
    while True:
        chunk = list(itertools.islice(it, batch))
        if not chunk:
            break
        ctx.run(chunk, stream=stream)
        for j, ev in enumerate(chunk):
            c = ctx.t5_candidates(j)
            t, p = label_candidates(c, ev.pid)
            if device:
                import torch
                X.append(torch.from_numpy(c["features"]).cuda())
            else:
                X.append(c["features"])
            y.append(t.astype(np.float32))
            cut.append(c["cut_pass"])
            part.append(p)
            ev_idx.append(np.full(len(t), b0 + j))
        b0 += len(chunk)
    cat = np.concatenate
    if device:
        import torch
        Xc = torch.cat(X)
        X.clear()
    else:
        Xc = cat(X)
    return dict(X=Xc, y=cat(y), cut=cat(cut), particle=cat(part), event=cat(ev_idx))


def collect_t3(ctx, events, batch=8, stream=None, device=True, max_per_event=None, seed=0):
    """Features and labels of the T3s of some events (the learned triplet selection's training set): label 1
    when all six hits come from one generated particle. max_per_event keeps a random subset of each event's
    T3s (a PU200 event holds about 4e5)."""
    import itertools
    rng = np.random.default_rng(seed)
    X, y = [], []
    it = iter(events)
    while True:
        chunk = list(itertools.islice(it, batch))
        if not chunk:
            break
        ctx.run(chunk, stream=stream)
        for j, ev in enumerate(chunk):
            c = ctx.t3_candidates(j)
            p = ev.pid[c["hits"]]
            true = (p[:, 0] >= 0) & np.all(p == p[:, :1], axis=1)
            f = c["features"]
            if max_per_event and len(true) > max_per_event:
                k = rng.choice(len(true), max_per_event, replace=False)
                f, true = f[k], true[k]
            if device:
                import torch
                X.append(torch.from_numpy(f).cuda())
            else:
                X.append(f)
            y.append(true.astype(np.float32))
    if device:
        import torch
        return dict(X=torch.cat(X), y=np.concatenate(y))
    return dict(X=np.concatenate(X), y=np.concatenate(y))


def threshold_keeping(scores, y, keep=0.99):
    """Largest threshold that keeps at least `keep` of the true candidates."""
    s = np.sort(np.asarray(scores)[np.asarray(y) > 0.5])
    if len(s) == 0:
        return 0.0
    k = int(np.floor((1.0 - keep) * len(s)))
    return float(s[k]) if k < len(s) else 0.0


def save_checkpoint(path, mlp, epoch, hist):
    """The network's whole training state (parameters, Adam moments and step) after `epoch` epochs."""
    st = mlp.state()
    np.savez(path, params=st["params"], m=st["m"], v=st["v"], step=st["step"], epoch=epoch,
             hist=np.asarray(hist, np.float64))


def load_checkpoint(path, mlp):
    """Restore a checkpoint into mlp; returns (epochs done, loss history)."""
    z = np.load(path)
    mlp.set_state(dict(params=z["params"], m=z["m"], v=z["v"], step=int(z["step"])))
    return int(z["epoch"]), [float(h) for h in z["hist"]]


def train(mlp, X, y, epochs=4, batch=4096, lr=2e-3, seed=0, log=None, start_epoch=0, checkpoint=None,
          hist=None):
    """Adam over shuffled batches. Epoch ep shuffles with its own generator (seed, ep), so a run resumed
    at start_epoch from a checkpoint continues exactly as the uninterrupted run; with `checkpoint` (a path)
    the state is saved after every epoch."""
    import torch
    n = len(y)
    Xd = X if torch.is_tensor(X) else torch.from_numpy(np.ascontiguousarray(X)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    hist = list(hist or [])
    for ep in range(start_epoch, epochs):
        perm = torch.from_numpy(np.random.default_rng([seed, ep]).permutation(n)).cuda()
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = Xd.index_select(0, idx).contiguous()
            yb = yd.index_select(0, idx).contiguous()
            want = (b0 // batch) % 50 == 0
            l = mlp.train_step(xb, yb, lr=lr, want_loss=want)
            if want:
                losses.append(l)
        hist.append(float(np.mean(losses)) if losses else float("nan"))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
        if checkpoint:
            save_checkpoint(checkpoint, mlp, ep + 1, hist)
    return hist


def scores_of(mlp, X):
    import torch
    Xd = X if torch.is_tensor(X) else torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = torch.zeros(len(X), device="cuda")
    mlp.forward(Xd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def selection_metrics(sel, data):
    """Efficiency over particles with at least one true candidate; fake fraction of the selection."""
    true = data["y"] > 0.5
    key = data["event"].astype(np.int64) * 10 ** 7 + data["particle"]
    findable = np.unique(key[true])
    found = np.unique(key[true & sel])
    eff = len(found) / max(1, len(findable))
    fake = float((sel & ~true).sum()) / max(1, int(sel.sum()))
    return dict(efficiency=eff, fake_rate=fake, selected=int(sel.sum()))


def matched_threshold(scores, data, target_eff):
    """Largest threshold whose efficiency reaches the target."""
    lo, hi = 0.0, 1.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if selection_metrics(scores >= mid, data)["efficiency"] >= target_eff:
            lo = mid
        else:
            hi = mid
    return lo


def evaluate(mlp, data):
    s = scores_of(mlp, data["X"])
    cut = selection_metrics(data["cut"], data)
    thr = matched_threshold(s, data, cut["efficiency"])
    net = selection_metrics(s >= thr, data)
    return dict(cut=cut, network=net, threshold=thr)


def main_t3(args):
    """Train and save the learned triplet selection (parameters and threshold)."""
    from synth import events as E, geometry as G, maps as M
    from synth.config import DEFAULT_CUTS
    from synth.mlp_init import init_params
    geom = G.make_geometry(barrel_only=False)
    maps = M.load_maps(geom)
    ctx = L.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=L.default_capacity(4))
    ctx.set_t3_selection(None, capture_features=True)
    t0 = time.time()
    tr = collect_t3(ctx, (E.pu200_event(43000 + i, geom) for i in range(args.train_events)), batch=4,
                    max_per_event=200000)
    va = collect_t3(ctx, [E.pu200_event(44000 + i, geom) for i in range(args.eval_events)], batch=4, device=False)
    ctx.close()
    mlp = L.Mlp(max_batch=4096, params=init_params(args.seed))
    hist = train(mlp, tr["X"], tr["y"], epochs=args.epochs, seed=args.seed)
    s = scores_of(mlp, va["X"])
    thr = threshold_keeping(s, va["y"], args.keep)
    fake = va["y"] < 0.5
    np.savez(args.out, params=mlp.params(), threshold=thr)
    mlp.close()
    print(json.dumps(dict(samples_train=int(len(tr["y"])), loss_history=hist, threshold=thr,
                          true_kept=float(np.mean(s[~fake] >= thr)), fake_pruned=float(np.mean(s[fake] < thr)),
                          seconds=round(time.time() - t0, 1))))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", choices=("t5", "t3"), default="t5")
    ap.add_argument("--keep", type=float, default=0.99, help="t3: fraction of true T3s the threshold keeps")
    ap.add_argument("--train-events", type=int, default=100)
    ap.add_argument("--eval-events", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--prefilter-scale", type=float, default=3.0)
    ap.add_argument("--out", default="t5_mlp.npy")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--checkpoint", default=None, help="save the training state here after every epoch")
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    if args.kind == "t3":
        return main_t3(args)
    from synth import events as E, geometry as G, maps as M
    from synth.config import DEFAULT_CUTS
    from synth.mlp_init import init_params
    geom = G.make_geometry(barrel_only=False)
    maps = M.load_maps(geom)
    ctx = L.Context(geom.module_table(), maps, cfg=DEFAULT_CUTS, capacity=L.default_capacity(16))
    ctx.set_t5_selection(None, prefilter_scale=args.prefilter_scale, capture_features=True)
    t0 = time.time()
    tr = collect(ctx, (E.pu200_event(10000 + i, geom) for i in range(args.train_events)), device=True)
    va = collect(ctx, [E.pu200_event(20000 + i, geom) for i in range(args.eval_events)])
    print(f"samples: train {len(tr['y'])} ({tr['y'].mean():.3f} true), eval {len(va['y'])}; "
          f"{time.time() - t0:.1f} s", flush=True)
    mlp = L.Mlp(max_batch=4096, params=init_params(args.seed))
    start, hist0 = 0, []
    if args.resume and args.checkpoint and os.path.exists(args.checkpoint):
        start, hist0 = load_checkpoint(args.checkpoint, mlp)
    t1 = time.time()
    hist = train(mlp, tr["X"], tr["y"], epochs=args.epochs, seed=args.seed, log=lambda m: print(m, flush=True),
                 start_epoch=start, checkpoint=args.checkpoint, hist=hist0)
    print(f"training: {time.time() - t1:.1f} s", flush=True)
    res = evaluate(mlp, va)
    res["loss_history"] = hist
    res["train_events"], res["eval_events"] = args.train_events, args.eval_events
    res["samples_train"], res["samples_eval"] = int(len(tr["y"])), int(len(va["y"]))
    np.savez(args.out, params=mlp.params(), threshold=res["threshold"], prefilter_scale=args.prefilter_scale)
    mlp.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
