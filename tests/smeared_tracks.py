"""Prompt helices crossing chosen surfaces, with Gaussian-smeared copies (test helper).

Used by the pull and chi2-distribution pins of the oracle's resolution terms.
A point is smeared exactly as the event generator smears hits: by the module's
r-phi resolution along phi-hat, and by its resolution along the strip (z in
the barrel, r in the endcap); pixel points by sig_pix in r-phi and z. Nothing
here computes a cut quantity.
"""
import math

import numpy as np

from synth import geometry as G
from synth.helix import cross_cylinder, cross_plane


def draw_tracks(rng, n, pt_range, eta_range, sigma_z0=5.0):
    """n tracks: pT log-uniform in pt_range, eta uniform in eta_range, phi0 uniform, random charge."""
    lo, hi = pt_range
    pt = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    return dict(pt=pt, q=rng.choice([-1.0, 1.0], n), eta=rng.uniform(eta_range[0], eta_range[1], n),
                phi0=rng.uniform(-math.pi, math.pi, n), z0=rng.normal(0.0, sigma_z0, n))


def crossing(geom, tr, surf, upper=False):
    """Unsmeared crossing of every track with surface surf = ('b', layer index) | ('e', disk index) |
    ('p', radius) (a pixel cylinder); upper selects the module's upper sensor. Returns (xyz [n,3], module
    id [n], valid [n]); the endcap side follows the sign of eta; pixel points carry module -1."""
    ks = -tr["q"] * G.curvature_of_pt(tr["pt"])
    tl = np.sinh(tr["eta"])
    kind, idx = surf
    n = len(ks)
    if kind in ("b", "p"):
        r = G.BARREL_R[idx] if kind == "b" else float(idx)
        if upper:
            r += G.DSEP
        ok, s, phi, z = cross_cylinder(ks, tr["phi0"], tl, tr["z0"], r)
        rr = np.full(n, r)
        if kind == "b":
            mod = geom.locate_barrel(np.full(n, idx), phi, z)
        else:
            mod = np.full(n, -1)
    else:
        side = np.where(tr["eta"] > 0, 1.0, -1.0)
        zp = side * (G.DISK_Z[idx] + (G.DSEP if upper else 0.0))
        ok, s, phi, rr = cross_plane(ks, tr["phi0"], tl, tr["z0"], zp)
        z = zp
        mod = geom.locate_endcap(side.astype(np.int64), idx, phi, rr)
    xyz = np.stack([rr * np.cos(phi), rr * np.sin(phi), np.broadcast_to(z, rr.shape)], axis=-1)
    valid = ok & ((mod >= 0) | (kind == "p"))
    return xyz, mod, valid


def smear(geom, xyz, mod, rng, sig_pix=0.001):
    """Generator-like Gaussian smearing of points xyz [n,3] on modules mod (-1: pixel point)."""
    r = np.hypot(xyz[:, 0], xyz[:, 1])
    phi = np.arctan2(xyz[:, 1], xyz[:, 0])
    z = xyz[:, 2].copy()
    pix = mod < 0
    m = np.where(pix, 0, mod)
    srphi = np.where(pix, sig_pix, geom.sig_rphi[m])
    slong = np.where(pix, sig_pix, geom.sig_long[m])
    barrel = pix | (geom.subdet[m] == G.SUBDET_BARREL)
    phi = phi + rng.normal(0.0, 1.0, len(r)) * srphi / r
    dl = rng.normal(0.0, 1.0, len(r)) * slong
    z = np.where(barrel, z + dl, z)
    r = np.where(barrel, r, r + dl)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1)


def rows(geom, xyz, mod, sig_pix=0.001):
    """(x, y, z, sig_rphi, sig_z, sig_r) rows as the oracle's point tables take them."""
    pix = mod < 0
    m = np.where(pix, 0, mod)
    barrel = geom.subdet[m] == G.SUBDET_BARREL
    srphi = np.where(pix, sig_pix, geom.sig_rphi[m].astype(np.float32).astype(np.float64))
    slong = geom.sig_long[m].astype(np.float32).astype(np.float64)
    sz = np.where(pix, sig_pix, np.where(barrel, slong, 0.0))
    sr = np.where(pix, 0.0, np.where(barrel, 0.0, slong))
    return np.column_stack([xyz, srphi, sz, sr])


def chain(geom, rng, n, surfs, pt_range, eta_range, sigma_z0=5.0):
    """Tracks that cross every surface of surfs on a module (pixel cylinders always count).
    Returns (tracks, truth rows [n, k, 6], smeared rows [n, k, 6], modules [n, k])."""
    tr_all, xs, ms = [], [], []
    got = 0
    for _ in range(200):
        if got >= n:
            break
        tr = draw_tracks(rng, 4 * n, pt_range, eta_range, sigma_z0)
        pts = [crossing(geom, tr, s) for s in surfs]
        ok = np.logical_and.reduce([v for _, _, v in pts])
        tr_all.append({k: v[ok] for k, v in tr.items()})
        xs.append(np.stack([p[0][ok] for p in pts], axis=1))
        ms.append(np.stack([p[1][ok] for p in pts], axis=1))
        got += int(ok.sum())
    if got < n:
        raise ValueError(f"only {got} of {n} tracks cross every surface of {surfs}")
    tr = {k: np.concatenate([t[k] for t in tr_all])[:n] for k in tr_all[0]}
    xyz = np.concatenate(xs)[:n]
    mod = np.concatenate(ms)[:n]
    k = len(surfs)
    truth = np.stack([rows(geom, xyz[:, j], mod[:, j]) for j in range(k)], axis=1)
    sm = np.stack([rows(geom, smear(geom, xyz[:, j], mod[:, j], rng), mod[:, j]) for j in range(k)], axis=1)
    return tr, truth, sm, mod


def expected_chi2_unweighted(truth):
    """First-order E[chi2_rphi] of an unweighted circle fit through points truth [n, 6] (x, y, z, sig_rphi,
    sig_z, sig_r) that lie on one circle, each with its own error along the circle normal.

    Linearised geometric model: a point's distance to the circle moves by n_i . dP_i - n_i . dc - dR for a
    change (dc, dR) of centre and radius (n_i: the unit normal at point i). Least squares with equal weights
    gives residuals (I - H) y with H = X (X^T X)^-1 X^T, X_i = (n_ix, n_iy, 1), y_i = n_i . dP_i of variance
    s_i^2 = (sig_rphi n_i.phi-hat)^2 + (sig_r n_i.r-hat)^2, so E[sum r_i^2 / s_i^2] =
    sum_i [(I - H) diag(s^2) (I - H)^T]_ii / s_i^2, which is n - 3 when all s_i are equal.
    """
    p = truth[:, :2]
    a, b, c = p[0], p[len(p) // 2], p[-1]
    M = 2.0 * np.array([b - a, c - a])
    centre = np.linalg.solve(M, np.array([b @ b - a @ a, c @ c - a @ a]))
    nrm = (p - centre) / np.linalg.norm(p - centre, axis=1)[:, None]
    rhat = p / np.linalg.norm(p, axis=1)[:, None]
    phat = np.stack([-rhat[:, 1], rhat[:, 0]], axis=1)
    s2 = np.maximum((truth[:, 3] * np.sum(nrm * phat, 1)) ** 2 + (truth[:, 5] * np.sum(nrm * rhat, 1)) ** 2,
                    (0.01 * truth[:, 3]) ** 2)
    X = np.column_stack([nrm, np.ones(len(p))])
    Q = np.eye(len(p)) - X @ np.linalg.solve(X.T @ X, X.T)
    return float(np.sum(np.diag(Q @ np.diag(s2) @ Q.T) / s2))
