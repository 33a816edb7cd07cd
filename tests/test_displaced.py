"""Displaced tracks (CPU): helices from a displaced production vertex, the
muon-gun sample of Section 2.2 (vertices uniform in a 5 cm cube), and the
connection map that covers them."""
import math

import numpy as np
import pytest

from synth import events as E
from synth import geometry as G
from synth import maps as M
from synth.helix import cross_cylinder, cross_cylinder_from, cross_plane, cross_plane_from, position_at

D0_MAX = 2.5 * math.sqrt(2.0)      # the corner of the 5 cm cube's transverse square


@pytest.fixture(scope="module")
def maps_displaced(geom_full):
    return M.load_maps(geom_full, M.MapParams(d0_max=D0_MAX))


def _tracks(rng, n):
    return dict(ks=rng.uniform(-1, 1, n) * float(G.curvature_of_pt(0.8)), th=rng.uniform(-math.pi, math.pi, n),
                tl=rng.uniform(-3, 3, n), x0=rng.uniform(-2.5, 2.5, n), y0=rng.uniform(-2.5, 2.5, n),
                z0=rng.uniform(-2.5, 2.5, n))


def test_from_the_beam_line_equals_the_prompt_helix():
    t = _tracks(np.random.default_rng(0), 5000)
    z = np.zeros(5000)
    for r in (23.0, 51.0, 108.0):
        a = cross_cylinder(t["ks"], t["th"], t["tl"], t["z0"], r)
        b = cross_cylinder_from(t["ks"], t["th"], t["tl"], z, z, t["z0"], r)
        assert np.array_equal(a[0], b[0])
        m = a[0]
        assert np.abs(a[1][m] - b[1][m]).max() < 1e-9
        assert np.abs(np.angle(np.exp(1j * (a[2][m] - b[2][m])))).max() < 1e-11
    a = cross_plane(t["ks"], t["th"], t["tl"], t["z0"], 156.0)
    b = cross_plane_from(t["ks"], t["th"], t["tl"], z, z, t["z0"], 156.0)
    m = a[0] & b[0]
    assert np.array_equal(a[0], b[0]) and np.abs(a[3][m] - b[3][m]).max() < 1e-9


def test_displaced_crossing_is_the_first_point_at_radius_r():
    """On the cylinder, on the helix (the closed-form position after arc length s), and no point of the path
    before s is outside r (brute force along the path)."""
    t = _tracks(np.random.default_rng(1), 3000)
    ok, s, phi, z = cross_cylinder_from(t["ks"], t["th"], t["tl"], t["x0"], t["y0"], t["z0"], 36.0)
    assert ok.mean() > 0.9
    x, y = position_at(t["ks"], t["th"], t["x0"], t["y0"], s)
    assert np.abs(np.hypot(x, y)[ok] - 36.0).max() < 1e-9
    assert np.allclose(z[ok], (t["z0"] + s * t["tl"])[ok])
    for i in np.nonzero(ok)[0][:200]:
        ss = np.linspace(0.0, s[i], 2000)[:-1]
        xx, yy = position_at(np.full_like(ss, t["ks"][i]), t["th"][i], t["x0"][i], t["y0"][i], ss)
        assert np.hypot(xx, yy).max() < 36.0 + 1e-9


def test_impact_parameter_by_brute_force():
    rng = np.random.default_rng(2)
    tr = E.sample_muon_gun(rng, 500)
    d0 = tr.d0
    ss = np.linspace(0.0, 2 * math.pi, 2000001)
    for i in range(0, 500, 25):
        R = 1.0 / abs(tr.kappa_s[i])
        x, y = position_at(np.full_like(ss, tr.kappa_s[i]), tr.phi0[i], tr.x0[i], tr.y0[i], ss * R)
        assert abs(np.hypot(x, y).min() - d0[i]) < 1e-5
    assert np.all(E.sample_pileup_tracks(rng, 10).d0 == 0)


def test_muon_gun_event_shape(geom_full):
    ev = E.muon_gun_event(3, geom_full, n=50)
    d0 = ev.tracks.d0
    assert d0.max() > 1.5 and d0.max() <= D0_MAX + 1e-9
    assert np.all(np.abs(ev.tracks.z0) <= 2.5)
    assert ev.n_seeds == 50 and np.all(ev.pid >= 0)
    assert ev.n_hits > 50 * 10


def test_displaced_connection_map_complete(geom_full, maps_full, maps_displaced):
    """Every consecutive module transition of 1e4 noiseless pT >= pT_min helices from vertices in the 5 cm cube
    is in the displaced map, which also holds every prompt connection."""
    co, ct = maps_displaced[0], maps_displaced[1]
    conn = [set(ct[co[i]:co[i + 1]].tolist()) for i in range(geom_full.n_mod)]
    pco, pct = maps_full[0], maps_full[1]
    for i in range(0, geom_full.n_mod, 7):
        assert set(pct[pco[i]:pco[i + 1]].tolist()) <= conn[i]
    rng = np.random.default_rng(777)
    n = 10000
    tr = E.Tracks(pt=np.exp(rng.uniform(math.log(0.8), math.log(50.0), n)), eta=rng.uniform(-2.6, 2.6, n),
                  phi0=rng.uniform(-math.pi, math.pi, n), q=rng.choice([-1.0, 1.0], n),
                  z0=rng.uniform(-2.5, 2.5, n), x0=rng.uniform(-2.5, 2.5, n), y0=rng.uniform(-2.5, 2.5, n))
    _, S, _, _, MOD = M._crossings_from(geom_full, tr)
    order = np.argsort(S, axis=0)
    Ms, Ss = np.take_along_axis(MOD, order, axis=0), np.take_along_axis(S, order, axis=0)
    checked = 0
    for a in range(Ms.shape[0] - 1):
        good = np.isfinite(Ss[a]) & np.isfinite(Ss[a + 1])
        for m1, m2 in zip(Ms[a][good], Ms[a + 1][good]):
            assert int(m2) in conn[int(m1)], (int(m1), int(m2))
            checked += 1
    assert checked > 30000
