"""Helix propagation in a uniform solenoidal field (input producer).

A track starts at (0, 0, z0) with transverse direction phi0, signed curvature
kappa_s (1/cm, positive = counter-clockwise seen from +z; a positive charge in
Bz > 0 bends clockwise, so kappa_s = -q / R) and tanl = dz/ds = sinh(eta),
where s is the transverse arc length. Along the helix

    position angle  phi(s) = phi0 + kappa_s * s / 2
    radius          r(s)   = 2 sin(|kappa| s / 2) / |kappa|
    z(s)                   = z0 + s * tanl

Only the outgoing half turn (|kappa| s <= pi) is ever recorded.
"""
from __future__ import annotations

import numpy as np


def _safe_kappa(kappa_abs):
    return np.where(kappa_abs > 0, kappa_abs, 1.0)


def cross_cylinder(kappa_s, phi0, tanl, z0, r):
    """Crossing of the helix with the cylinder of radius r (outgoing half).

    Returns (valid, s, phi, z). `valid` is False when the helix never reaches r.
    """
    kappa_s = np.asarray(kappa_s, dtype=np.float64)
    ka = np.abs(kappa_s)
    x = r * ka / 2.0
    valid = x < 1.0
    xs = np.minimum(x, 1.0)
    s = np.where(ka > 0, 2.0 * np.arcsin(xs) / _safe_kappa(ka), r)
    phi = phi0 + kappa_s * s / 2.0
    z = z0 + s * tanl
    return valid, s, phi, z


def cross_plane(kappa_s, phi0, tanl, z0, zp):
    """Crossing of the helix with the plane z = zp (outgoing half turn only).

    Returns (valid, s, phi, r).
    """
    kappa_s = np.asarray(kappa_s, dtype=np.float64)
    tanl = np.asarray(tanl, dtype=np.float64)
    ka = np.abs(kappa_s)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (zp - z0) / np.where(tanl != 0, tanl, np.nan)
    valid = np.isfinite(s) & (s > 0) & (ka * np.nan_to_num(s, nan=0.0) <= np.pi)
    s = np.where(valid, s, 0.0)
    r = np.where(ka > 0, 2.0 * np.sin(ka * s / 2.0) / _safe_kappa(ka), s)
    phi = phi0 + kappa_s * s / 2.0
    return valid, s, phi, r


def wrap_phi(phi):
    return np.mod(np.asarray(phi) + np.pi, 2 * np.pi) - np.pi
