"""FP64 helix points for the closed-form pins (test helper)."""
import math

import numpy as np

from synth import geometry as G
from synth.helix import cross_cylinder, cross_plane


def kappa_s(pt, q):
    return -q * float(G.curvature_of_pt(pt))


def on_cylinder(pt, q, eta, phi0, z0, r):
    ok, s, phi, z = cross_cylinder(np.array([kappa_s(pt, q)]), phi0, math.sinh(eta), z0, r)
    assert ok[0]
    return np.array([r * math.cos(phi[0]), r * math.sin(phi[0]), z[0]]), float(s[0])


def on_plane(pt, q, eta, phi0, z0, zp):
    ok, s, phi, r = cross_plane(np.array([kappa_s(pt, q)]), phi0, math.sinh(eta), z0, zp)
    assert ok[0]
    return np.array([r[0] * math.cos(phi[0]), r[0] * math.sin(phi[0]), zp]), float(s[0])


def barrel_module(geom, li, p):
    return int(geom.locate_barrel(np.array([li]), math.atan2(p[1], p[0]), p[2])[0])


def endcap_module(geom, side, di, p):
    return int(geom.locate_endcap(np.array([side]), di, math.atan2(p[1], p[0]), math.hypot(p[0], p[1]))[0])


def row(p, srphi, sz, sr):
    return [p[0], p[1], p[2], srphi, sz, sr]
