"""Host checks of the pT3 search's curvature window (the device's ks_window and
float_order_key, restated here): every triplet curvature that can pass the
search's curvature prefilter lies inside the window, so binary-searching a
curvature-ordered view loses nothing; and the integer key orders floats as
their values do."""
import numpy as np

f32 = np.float32


def prefilter_pass(k, s, kt, st, n, rel):
    """|k - kt| <= 1.01 n sqrt(s^2 + st^2) + rel (|k| + |kt|) + 1e-7, in FP32 as the search evaluates it."""
    thr = f32(n) * np.sqrt(f32(s) * f32(s) + f32(st) * f32(st), dtype=f32)
    rhs = thr * f32(1.01) + f32(rel) * (np.abs(f32(k)) + np.abs(f32(kt))) + f32(1e-7)
    return np.abs(f32(k) - f32(kt)) <= rhs


def window(k, s, smax, n, rel):
    return (f32(1.01) * f32(n) * (f32(s) + f32(smax)) + f32(2 * rel) * np.abs(f32(k)) + f32(1e-7)) / f32(1 - rel) \
        * f32(1.001) + f32(1e-7)


def order_key(v):
    u = np.asarray(v, f32).view(np.uint32)
    return np.where(u & np.uint32(0x80000000), ~u, u | np.uint32(0x80000000))


def test_every_passing_curvature_lies_in_the_window():
    rng = np.random.default_rng(7)
    m = 400000
    for rel in (1e-5, 1e-3):                     # FP32 and compact (FP16) storage slack
        k = rng.uniform(-0.015, 0.015, m).astype(f32)
        s = (10 ** rng.uniform(-6, -2.5, m)).astype(f32)
        smax = (10 ** rng.uniform(-6, -2.5, m)).astype(f32)
        st = (smax * rng.uniform(0, 1, m)).astype(f32)
        # curvatures spread around the pass boundary, both sides
        reach = 1.01 * 3.0 * np.sqrt(s.astype(float) ** 2 + st.astype(float) ** 2) + rel * 2 * np.abs(k) + 1e-7
        kt = (k + rng.choice([-1, 1], m) * reach * rng.uniform(0.5, 1.5, m)).astype(f32)
        ok = prefilter_pass(k, s, kt, st, 3.0, rel)
        assert ok.sum() > m // 4
        w = window(k, s, smax, 3.0, rel)
        inside = np.abs(kt.astype(float) - k.astype(float)) <= w.astype(float)
        assert np.all(inside[ok])


def test_order_key_sorts_as_the_values():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.normal(0, 1e-3, 5000), rng.normal(0, 1e3, 5000),
                        [0.0, -0.0, np.inf, -np.inf, 1e-40, -1e-40]]).astype(f32)
    order = np.argsort(order_key(v), kind="stable")
    assert np.all(np.diff(v[order].astype(float)) >= 0)
