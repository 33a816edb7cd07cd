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


def _start_frame(kappa_s, theta0, x0, y0):
    """Centre of the transverse circle of a track leaving (x0, y0) in direction theta0 with signed
    curvature kappa_s (positive: counter-clockwise), and its radius; None-safe for kappa_s = 0."""
    ka = np.abs(kappa_s)
    R = np.where(ka > 0, 1.0 / np.where(ka > 0, ka, 1.0), np.inf)
    sgn = np.where(kappa_s >= 0, 1.0, -1.0)
    cx = x0 - sgn * R * np.sin(theta0)
    cy = y0 + sgn * R * np.cos(theta0)
    return cx, cy, R, sgn


def position_at(kappa_s, theta0, x0, y0, s):
    """Transverse position after arc length s from (x0, y0) in direction theta0."""
    kappa_s = np.asarray(kappa_s, dtype=np.float64)
    ka = np.abs(kappa_s)
    small = ka * np.abs(s) < 1e-9
    k = np.where(small, 1.0, kappa_s)
    x = np.where(small, x0 + s * np.cos(theta0), x0 + (np.sin(theta0 + kappa_s * s) - np.sin(theta0)) / k)
    y = np.where(small, y0 + s * np.sin(theta0), y0 - (np.cos(theta0 + kappa_s * s) - np.cos(theta0)) / k)
    return x, y


def cross_cylinder_from(kappa_s, theta0, tanl, x0, y0, z0, r):
    """First crossing of a helix that starts at (x0, y0, z0) with transverse direction theta0 with the
    cylinder of radius r (a start inside the cylinder, |kappa| s <= pi). Returns (valid, s, phi, z), phi the
    position angle of the crossing. With x0 = y0 = 0 it agrees with cross_cylinder (theta0 = phi0)."""
    kappa_s = np.asarray(kappa_s, dtype=np.float64)
    x0 = np.asarray(x0, dtype=np.float64) + 0.0 * kappa_s
    y0 = np.asarray(y0, dtype=np.float64) + 0.0 * kappa_s
    r2s = x0 * x0 + y0 * y0
    ux, uy = np.cos(theta0), np.sin(theta0)
    # straight line: |p0 + s u| = r
    b = x0 * ux + y0 * uy
    s_lin = -b + np.sqrt(np.maximum(b * b - (r2s - r * r), 0.0))
    # circle of centre c and radius R against the circle |p| = r: the points at distance q along c-hat
    # from the origin, q = (r^2 - R^2 + d^2) / (2d), and +-h = sqrt(r^2 - q^2) across it
    cx, cy, R, sgn = _start_frame(kappa_s, theta0, x0, y0)
    finite = np.isfinite(R)
    Rf = np.where(finite, R, 1.0)
    cxf, cyf = np.where(finite, cx, 1.0), np.where(finite, cy, 0.0)
    d = np.hypot(cxf, cyf)
    q = (r * r - Rf * Rf + d * d) / (2.0 * d)
    h2 = r * r - q * q
    ok_c = finite & (h2 >= 0.0)
    h = np.sqrt(np.maximum(h2, 0.0))
    ex, ey = cxf / d, cyf / d
    sx0, sy0 = x0 - cxf, y0 - cyf                  # start point seen from the centre
    best = np.full(kappa_s.shape, np.inf)
    for sg in (1.0, -1.0):
        px, py = q * ex - sg * h * ey, q * ey + sg * h * ex
        vx, vy = px - cxf, py - cyf
        ang = np.arctan2(sx0 * vy - sy0 * vx, sx0 * vx + sy0 * vy)   # counter-clockwise angle start -> point
        turn = np.mod(sgn * ang, 2 * np.pi)
        best = np.minimum(best, turn)
    s_circ = best * Rf
    s = np.where(finite, s_circ, s_lin)
    valid = np.where(finite, ok_c & (best <= np.pi), b * b - (r2s - r * r) >= 0.0) & (r2s < r * r)
    s = np.where(valid, s, 0.0)
    x, y = position_at(kappa_s, theta0, x0, y0, s)
    return valid, s, np.arctan2(y, x), z0 + s * tanl


def cross_plane_from(kappa_s, theta0, tanl, x0, y0, z0, zp):
    """Crossing of that helix with the plane z = zp (|kappa| s <= pi). Returns (valid, s, phi, r)."""
    kappa_s = np.asarray(kappa_s, dtype=np.float64)
    tanl = np.asarray(tanl, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (zp - z0) / np.where(tanl != 0, tanl, np.nan)
    valid = np.isfinite(s) & (s > 0) & (np.abs(kappa_s) * np.nan_to_num(s, nan=0.0) <= np.pi)
    s = np.where(valid, s, 0.0)
    x, y = position_at(kappa_s, theta0, x0, y0, s)
    return valid, s, np.arctan2(y, x), np.hypot(x, y)


def wrap_phi(phi):
    return np.mod(np.asarray(phi) + np.pi, 2 * np.pi) - np.pi
