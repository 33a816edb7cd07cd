"""Pins of the FP64 scoring-network reference and of the feature definition (CPU)."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as R
from oracle import oracle as O
from synth.mlp_init import init_params
from synth import geometry as G
from tests.helix_points import on_cylinder


def _data(n=37, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, R.N_IN)).astype(np.float32)
    X[:, 38:] = 0
    y = (rng.uniform(size=n) < 0.4).astype(np.float64)
    return X, y


def test_parameter_count():
    assert R.N_PARAMS == 9409


def test_gradient_matches_finite_differences():
    X, y = _data()
    theta = init_params(3).astype(np.float64) * 0.7
    g = R.grad(theta, X, y, rounding=False)
    rng = np.random.default_rng(1)
    for i in rng.choice(R.N_PARAMS, 60, replace=False):
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (R.loss(tp, X, y, rounding=False) - R.loss(tm, X, y, rounding=False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-4, abs(fd)) + 1e-9, i


def test_zero_weights_closed_form():
    X, y = _data(50, 2)
    theta = np.zeros(R.N_PARAMS)
    theta[-1] = 0.3                      # b4
    s, _ = R.forward(theta, X)
    sig = 1 / (1 + math.exp(-0.3))
    assert np.allclose(s, sig)
    bce = -np.mean(y * math.log(sig) + (1 - y) * math.log(1 - sig))
    assert abs(R.loss(theta, X, y) - bce) < 1e-12
    g = R.grad(theta, X, y)
    assert abs(g[-1] - np.mean(sig - y)) < 1e-12
    assert np.all(g[:-1] == 0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0, 10, 2000), [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0, 65504.0]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(R.bf16(x), want)


def test_adam_first_step():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    t1, m, v = R.adam(theta, np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # step 1: bias-corrected moments are g and g^2, the update is lr g / (|g| + eps)
    assert np.allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8))


def _features(pt, q, eta, phi0, z0, smear=None):
    """Features of a T5 built from noiseless barrel helix hits (barrel layers 1-5)."""
    from synth import geometry as G, maps as M
    from synth.config import DEFAULT_CUTS
    from synth.events import Event
    geom = G.make_geometry(barrel_only=True)
    xs, ys, zs, mods, sides = [], [], [], [], []
    ds = float(np.float32(G.DSEP))
    for li in range(5):
        for side, r in ((0, G.BARREL_R[li]), (1, G.BARREL_R[li] + ds)):
            p, _ = on_cylinder(pt, q, eta, phi0, z0, r)
            xs.append(p[0]); ys.append(p[1]); zs.append(p[2]); sides.append(side)
        m = int(geom.locate_barrel(np.array([li]), math.atan2(ys[-2], xs[-2]), zs[-2])[0])
        mods += [m, m]
    ev = Event(x=np.array(xs, np.float32), y=np.array(ys, np.float32), z=np.array(zs, np.float32),
               module=np.array(mods, np.int32), side=np.array(sides, np.uint8), pid=np.zeros(10, np.int32),
               seeds=np.zeros((0, 3, 3), np.float32), seed_pid=np.zeros(0, np.int32), tracks=None)
    S = O.Setup(geom.module_table(), M.load_maps(geom), DEFAULT_CUTS, ev)
    return S.t5_features(list(range(10))), ev


def test_features_of_a_helix():
    for q in (-1.0, 1.0):
        f, ev = _features(2.5, q, 0.4, 1.0, 0.0)
        ks = -q * 0.3 * 3.8 / (100 * 2.5)
        two_a = 2 * 0.3 * 3.8 / (200 * 0.8)
        # lower hits sit on the fitted circle and line (float32 inputs: ~1e-3 pulls at most)
        assert np.all(np.abs(f[0:10:2]) < 0.05) and np.all(np.abs(f[10:20:2]) < 0.05)
        assert abs(f[27] - ks / two_a) < 1e-4
        assert abs(f[25] - ks / two_a) < 1e-3 and abs(f[26] - ks / two_a) < 1e-3
        assert abs(f[32] - 0.4) < 1e-4
        r = np.hypot(ev.x[0::2].astype(np.float64), ev.y[0::2].astype(np.float64))
        assert np.allclose(f[20:25], r / 100)
        assert np.allclose(f[33:38], np.arange(1, 6) / 11)
        assert np.all(f[38:] == 0)
        # beta of each triplet has the bending sign
        assert np.sign(f[30]) == np.sign(ks) and np.sign(f[31]) == np.sign(ks)


def _t3_event(geom, pt, q, eta, phi0, layers, shift=0.0):
    """Three barrel MDs of one noiseless helix (lower and upper hits); the middle upper hit moved by `shift`
    along phi-hat."""
    import math
    from types import SimpleNamespace
    from tests.helix_points import barrel_module, on_cylinder
    xs, mods, sides = [], [], []
    for li in layers:
        r = G.BARREL_R[li]
        for side, rr in ((0, r), (1, r + float(np.float32(G.DSEP)))):
            p, _ = on_cylinder(pt, q, eta, phi0, 0.0, rr)
            if side == 1 and li == layers[1]:
                ph = math.atan2(p[1], p[0]) + shift / rr
                p = np.array([rr * math.cos(ph), rr * math.sin(ph), p[2]])
            xs.append(p)
            mods.append(barrel_module(geom, li, xs[-2] if side == 1 else p))
            sides.append(side)
    xs = np.array(xs)
    return SimpleNamespace(x=xs[:, 0], y=xs[:, 1], z=xs[:, 2], module=np.array(mods, np.int32),
                           side=np.array(sides, np.uint8), seeds=np.zeros((0, 3, 3), np.float32))


def test_t3_features_closed_forms(geom_full, maps_full, cuts):
    """Noiseless helix: every pull 0, curvature and eta of the helix, the anchors' radii, beta of the circle,
    and zeros in the slots a triplet does not fill. One upper hit moved by delta in r-phi: its pull is
    delta / sigma_rphi (hits are stored in FP32, hence the tolerances)."""
    import math
    from oracle import oracle as O
    from synth import geometry as G_
    pt, q, eta = 2.5, -1.0, 0.4
    ev = _t3_event(geom_full, pt, q, eta, 0.9, (1, 2, 3))
    S = O.Setup(geom_full.module_table(), maps_full, cuts, ev)
    f = S.t3_features([0, 1, 2, 3, 4, 5])
    two_a = 2 * 0.3 * 3.8 / (200 * 0.8)
    ks = -q * float(G_.curvature_of_pt(pt))
    assert np.all(np.abs(f[0:6]) < 0.05) and np.all(np.abs(f[10:16]) < 0.05)
    assert abs(f[25] - ks / two_a) < 1e-4 * abs(ks / two_a) and abs(f[27] - f[25]) < 1e-6
    assert abs(f[32] - eta) < 1e-5
    assert np.allclose(f[20:23], np.array([G_.BARREL_R[1], G_.BARREL_R[2], G_.BARREL_R[3]]) / 100, atol=1e-6)
    R = 1 / abs(ks)
    a, b, c = (np.array([ev.x[i], ev.y[i]], float) for i in (0, 2, 4))
    beta = math.copysign(math.asin(np.linalg.norm(b - a) / (2 * R)) + math.asin(np.linalg.norm(c - b) / (2 * R)), ks)
    assert abs(f[30] - 10 * beta) < 1e-4
    assert np.allclose(f[33:36], np.array([2, 3, 4]) / 11.0)
    zero = [6, 7, 8, 9, 16, 17, 18, 19, 23, 24, 26, 31] + list(range(36, 48))
    assert np.all(f[zero] == 0.0)
    delta = 3 * 0.009 / math.sqrt(12)
    g = S.__class__(geom_full.module_table(), maps_full, cuts, _t3_event(geom_full, pt, q, eta, 0.9, (1, 2, 3),
                                                                          shift=delta)).t3_features(range(6))
    assert abs(abs(g[3]) - 3.0) < 0.05
    assert np.all(np.abs(np.delete(g[0:6], 3)) < 0.05)
