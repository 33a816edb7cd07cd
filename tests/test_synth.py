"""Pins of the seeded input producer (geometry, helices, maps)."""
import math

import numpy as np
import pytest

from synth import events as E
from synth import geometry as G
from synth import maps as M
from synth.helix import cross_cylinder, cross_plane


def test_module_count(geom_full, geom_barrel):
    assert geom_barrel.n_mod == 960
    assert geom_full.n_mod == 13260     # 960 barrel + 10 disks x 1230


def test_locate_roundtrip(geom_full):
    g = geom_full
    rng = np.random.default_rng(0)
    for m in rng.integers(0, g.n_mod, 500):
        phi = 0.5 * (g.phi_lo[m] + g.phi_hi[m])
        ell = 0.5 * (g.lo[m] + g.hi[m])
        if g.subdet[m] == 0:
            got = g.locate_barrel(np.array([g.layer[m] - 1]), phi, ell)[0]
        else:
            got = g.locate_endcap(np.array([g.side[m]]), g.layer[m] - 1, phi, ell)[0]
        assert got == m


def test_noiseless_hits_on_surfaces(geom_full):
    rng = np.random.default_rng(1)
    tr = E.sample_pileup_tracks(rng, 300)
    ev = E.make_event(geom_full, tr, rng, n_noise=0, smear=False, shuffle=False)
    g = geom_full
    m = ev.module
    r = np.hypot(ev.x.astype(np.float64), ev.y.astype(np.float64))
    barrel = g.subdet[m] == 0
    r_exp = g.surf[m] + ev.side * g.dsep[m]
    assert np.allclose(r[barrel], r_exp[barrel], rtol=2e-7)
    z_exp = g.surf[m] + np.sign(g.surf[m]) * ev.side * g.dsep[m]
    assert np.allclose(ev.z[~barrel], z_exp[~barrel], rtol=1e-7)


@pytest.mark.parametrize("pt", [0.8, 1.7, 12.0, 95.0])
def test_three_point_radius_is_pt_over_03B(pt):
    """Circumradius of three noiseless helix points is pT / (0.3 B) (FP64)."""
    for q in (-1.0, 1.0):
        ks = -q * float(G.curvature_of_pt(pt))
        pts = []
        for r in (23.0, 51.0, 88.0):
            ok, s, phi, z = cross_cylinder(np.array([ks]), 0.3, 0.5, 1.0, r)
            pts.append(np.array([r * math.cos(phi[0]), r * math.sin(phi[0])]))
        a, b, c = pts
        la, lb, lc = np.linalg.norm(b - c), np.linalg.norm(c - a), np.linalg.norm(a - b)
        area2 = abs((b - a)[0] * (c - a)[1] - (b - a)[1] * (c - a)[0])
        R = la * lb * lc / (2 * area2)
        assert abs(R - 100.0 * pt / (0.3 * 3.8)) / R < 1e-9


def test_z_linear_in_arc_length():
    ks = np.array([0.009])
    s_all, z_all = [], []
    for r in (23.0, 36.0, 51.0, 68.0):
        ok, s, phi, z = cross_cylinder(ks, 0.0, 1.2, -3.0, r)
        s_all.append(s[0]); z_all.append(z[0])
    for zp in (131.0, 156.0):
        ok, s, phi, rr = cross_plane(ks, 0.0, 1.2, -3.0, zp)
        if ok[0]:
            s_all.append(s[0]); z_all.append(zp)
    s_all, z_all = np.array(s_all), np.array(z_all)
    slope = np.diff(z_all) / np.diff(s_all)
    assert np.allclose(slope, 1.2, rtol=1e-12)


def _random_transitions(geom, p, n, seed, eta_max):
    rng = np.random.default_rng(seed)
    ks = rng.uniform(-1, 1, n) * p.kappa_max
    phi0 = rng.uniform(-math.pi, math.pi, n)
    eta = rng.uniform(-eta_max, eta_max, n)
    z0 = rng.uniform(-p.z_lumi, p.z_lumi, n)
    _, S, PHI, ELL, MOD = M._crossings_all(geom, ks, phi0, np.sinh(eta), z0)
    order = np.argsort(S, axis=0)
    return ks, phi0, eta, np.take_along_axis(MOD, order, axis=0), np.take_along_axis(S, order, axis=0)


def test_connection_map_complete(geom_full, maps_full):
    """Every consecutive module transition of 1e4 noiseless pT >= pT_min helices is in the map."""
    co, ct, so, st = maps_full
    p = M.MapParams()
    _, _, _, Ms, Ss = _random_transitions(geom_full, p, 10000, 12345, 2.6)
    conn = [set(ct[co[i]:co[i + 1]].tolist()) for i in range(geom_full.n_mod)]
    n = 0
    for a in range(Ms.shape[0] - 1):
        good = np.isfinite(Ss[a]) & np.isfinite(Ss[a + 1])
        for m1, m2 in zip(Ms[a][good], Ms[a + 1][good]):
            assert int(m2) in conn[int(m1)]
            n += 1
    assert n > 30000


def test_superbin_map_complete(geom_full, maps_full):
    """The first two modules crossed by a helix are listed under its superbin."""
    co, ct, so, st = maps_full
    p = M.MapParams()
    ks, phi0, eta, Ms, Ss = _random_transitions(geom_full, p, 10000, 54321, 2.6)
    sb = M.superbin_index(eta, phi0, -np.sign(ks), p)
    n = 0
    for i in range(len(ks)):
        lst = set(st[so[sb[i]]:so[sb[i] + 1]].tolist())
        for a in (0, 1):
            if np.isfinite(Ss[a, i]):
                assert int(Ms[a, i]) in lst
                n += 1
    assert n > 15000


def test_event_shapes():
    ev = E.tiny_event(0)
    assert ev.n_hits == 140 and ev.n_seeds == 10
    assert ev.x.dtype == np.float32 and ev.module.dtype == np.int32 and ev.side.dtype == np.uint8
    assert (ev.pid < 0).sum() == 20
