"""Seeded synthetic events shaped like the paper's workloads (input producer).

Every event is a set of outer-tracker hits (x, y, z as float32, the module id
and the sensor side: 0 = lower / nearer the interaction point, 1 = upper) plus
pixel seeds (three float32 space points per seed at r = 5, 10, 15 cm). The
generator also keeps the truth (particle id of each hit and seed) for
efficiency studies. Random numbers come from numpy's PCG64 (`default_rng`).

Workload recipes (the paper's CMS samples are not available; these stand in):

* ``tiny``: barrel-only geometry, 10 prompt tracks from (0,0,0), pT uniform in
  1-10 GeV, |eta| < 0.8, phi uniform, charge +-1, 20 uniform noise hits.
* ``pu200``: full geometry, 8000 prompt tracks from a Gaussian beamspot
  (sigma_z = 5 cm), dN/dpT ~ pT^-3 above 0.5 GeV, |eta| < 2.4, plus 12 jet-like
  tracks with pT uniform in 5-100 GeV; noise hits are 2 % of all hits.
* ``pileup(pu)``: 40 * pu tracks drawn like ``pu200`` (full geometry,
  beamspot, power-law pT, |eta| < 2.4), 2 % noise: used for batches and the
  serving loop with pu uniform in the stated ranges.

Hits are the helix-sensor intersections, Gaussian-smeared by pitch/sqrt(12)
in r-phi and by strip-length/sqrt(12) along the strip (z in the barrel, r in
the endcap). The module of a hit is the tile containing the unsmeared
crossing. Pixel space points are smeared by 10 um in r-phi and z. The hit
order is shuffled so that nothing downstream may rely on it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import geometry as G
from .helix import cross_cylinder, cross_cylinder_from, cross_plane, cross_plane_from

PIXEL_R = (5.0, 10.0, 15.0)
PIXEL_SIGMA = 0.001   # 10 um


@dataclass
class Tracks:
    pt: np.ndarray
    eta: np.ndarray
    phi0: np.ndarray        # transverse direction at the production vertex
    q: np.ndarray
    z0: np.ndarray
    x0: np.ndarray = None   # transverse production vertex (None: the beam line)
    y0: np.ndarray = None

    @property
    def n(self):
        return len(self.pt)

    @property
    def displaced(self):
        return self.x0 is not None and (np.any(self.x0 != 0) or np.any(self.y0 != 0))

    @property
    def d0(self):
        """Unsigned transverse distance of closest approach of each track's circle to the beam line."""
        if self.x0 is None:
            return np.zeros(self.n)
        ks = self.kappa_s
        ka = np.abs(ks)
        R = 1.0 / np.where(ka > 0, ka, 1.0)
        sg = np.where(ks >= 0, 1.0, -1.0)
        cx = self.x0 - sg * R * np.sin(self.phi0)
        cy = self.y0 + sg * R * np.cos(self.phi0)
        straight = np.abs(self.x0 * np.sin(self.phi0) - self.y0 * np.cos(self.phi0))
        return np.where(ka > 0, np.abs(np.hypot(cx, cy) - R), straight)

    @property
    def kappa_s(self):
        return -self.q * G.curvature_of_pt(self.pt)

    @property
    def tanl(self):
        return np.sinh(self.eta)

    @staticmethod
    def concat(parts):
        t = Tracks(*[np.concatenate([getattr(p, f) for p in parts]) for f in ("pt", "eta", "phi0", "q", "z0")])
        if any(p.x0 is not None for p in parts):
            t.x0 = np.concatenate([p.x0 if p.x0 is not None else np.zeros(p.n) for p in parts])
            t.y0 = np.concatenate([p.y0 if p.y0 is not None else np.zeros(p.n) for p in parts])
        return t


@dataclass
class Event:
    x: np.ndarray          # float32
    y: np.ndarray
    z: np.ndarray
    module: np.ndarray     # int32
    side: np.ndarray       # uint8
    pid: np.ndarray        # int32 particle id, -1 for noise
    seeds: np.ndarray      # float32 [n_seed, 3 points, 3 coords]
    seed_pid: np.ndarray   # int32
    tracks: Tracks

    @property
    def n_hits(self):
        return len(self.x)

    @property
    def n_seeds(self):
        return len(self.seeds)


# --------------------------------------------------------------------------
# track samplers
# --------------------------------------------------------------------------
def sample_tiny_tracks(rng, n=10):
    return Tracks(
        pt=rng.uniform(1.0, 10.0, n),
        eta=rng.uniform(-0.8, 0.8, n),
        phi0=rng.uniform(-math.pi, math.pi, n),
        q=rng.choice([-1.0, 1.0], n),
        z0=np.zeros(n),
    )


def sample_pileup_tracks(rng, n, n_jet=0, eta_max=2.4, sigma_z=5.0):
    u = rng.uniform(0.0, 1.0, n)
    pt = 0.5 / np.sqrt(1.0 - u)              # dN/dpT ~ pT^-3 above 0.5 GeV
    soft = Tracks(
        pt=pt,
        eta=rng.uniform(-eta_max, eta_max, n),
        phi0=rng.uniform(-math.pi, math.pi, n),
        q=rng.choice([-1.0, 1.0], n),
        z0=rng.normal(0.0, sigma_z, n),
    )
    if n_jet == 0:
        return soft
    jets = Tracks(
        pt=rng.uniform(5.0, 100.0, n_jet),
        eta=rng.uniform(-eta_max, eta_max, n_jet),
        phi0=rng.uniform(-math.pi, math.pi, n_jet),
        q=rng.choice([-1.0, 1.0], n_jet),
        z0=rng.normal(0.0, sigma_z, n_jet),
    )
    return Tracks.concat([soft, jets])


# --------------------------------------------------------------------------
# hits
# --------------------------------------------------------------------------
def sensor_surfaces(geom):
    """(kind, value, layer_idx, side_sign, sensor) for every sensor surface.

    kind 0: barrel cylinder of radius value; kind 1: disk plane at z = value.
    """
    out = []
    for li, r in enumerate(G.BARREL_R):
        out.append((0, r, li, 0, 0))
        out.append((0, r + G.DSEP, li, 0, 1))
    if not geom.barrel_only:
        for di, zd in enumerate(G.DISK_Z):
            for sgn in (-1, +1):
                out.append((1, sgn * zd, di, sgn, 0))
                out.append((1, sgn * (zd + G.DSEP), di, sgn, 1))
    return out


def true_crossings(geom, tr: Tracks):
    """All valid (track, sensor) crossings as flat arrays (unsmeared)."""
    ks, tl = tr.kappa_s, tr.tanl
    cols = {k: [] for k in ("tid", "module", "side", "r", "phi", "z", "kind")}
    tids = np.arange(tr.n)
    disp = tr.displaced
    for kind, val, li, sgn, sensor in sensor_surfaces(geom):
        if kind == 0:
            ok, s, phi, z = (cross_cylinder_from(ks, tr.phi0, tl, tr.x0, tr.y0, tr.z0, val) if disp
                             else cross_cylinder(ks, tr.phi0, tl, tr.z0, val))
            r = np.full_like(s, val)
            mid = geom.locate_barrel(np.full(tr.n, li), phi, z)
        else:
            ok, s, phi, r = (cross_plane_from(ks, tr.phi0, tl, tr.x0, tr.y0, tr.z0, val) if disp
                             else cross_plane(ks, tr.phi0, tl, tr.z0, val))
            z = np.full_like(s, val)
            mid = geom.locate_endcap(np.full(tr.n, sgn), li, phi, r)
        ok = ok & (mid >= 0)
        cols["tid"].append(tids[ok])
        cols["module"].append(mid[ok])
        cols["side"].append(np.full(ok.sum(), sensor))
        cols["r"].append(r[ok])
        cols["phi"].append(phi[ok])
        cols["z"].append(z[ok])
        cols["kind"].append(np.full(ok.sum(), kind))
    return {k: np.concatenate(v) for k, v in cols.items()}


def _noise_hits(geom, rng, n):
    area = geom.area()
    p = area / area.sum()
    mid = rng.choice(geom.n_mod, size=n, p=p)
    side = rng.integers(0, 2, n)
    phi = rng.uniform(geom.phi_lo[mid], geom.phi_hi[mid])
    barrel = geom.subdet[mid] == G.SUBDET_BARREL
    # barrel: uniform z; endcap: uniform in area (r^2 uniform)
    zb = rng.uniform(geom.lo[mid], geom.hi[mid])
    rb = geom.surf[mid] + side * geom.dsep[mid]
    u = rng.uniform(0.0, 1.0, n)
    re = np.sqrt(np.abs(geom.lo[mid] ** 2 + u * (geom.hi[mid] ** 2 - geom.lo[mid] ** 2)))
    ze = geom.surf[mid] + np.sign(geom.surf[mid]) * side * geom.dsep[mid]
    r = np.where(barrel, rb, re)
    z = np.where(barrel, zb, ze)
    return mid, side, r, phi, z


def make_event(geom, tracks: Tracks, rng, n_noise=None, noise_frac=None, smear=True, with_seeds=True,
               shuffle=True):
    c = true_crossings(geom, tracks)
    n_sig = len(c["tid"])
    r, phi, z = c["r"].copy(), c["phi"].copy(), c["z"].copy()
    mid = c["module"]
    if smear:
        srphi = geom.sig_rphi[mid]
        slong = geom.sig_long[mid]
        barrel = c["kind"] == 0
        phi = phi + rng.normal(0.0, 1.0, n_sig) * srphi / r
        dl = rng.normal(0.0, 1.0, n_sig) * slong
        r_s = np.where(barrel, r, r + dl)
        z = np.where(barrel, z + dl, z)
        r = r_s
    if n_noise is None:
        n_noise = 0 if noise_frac is None else int(round(noise_frac / (1.0 - noise_frac) * n_sig))
    nm, ns, nr, nphi, nz = _noise_hits(geom, rng, n_noise)
    mod = np.concatenate([mid, nm]).astype(np.int32)
    side = np.concatenate([c["side"], ns]).astype(np.uint8)
    rr = np.concatenate([r, nr])
    pp = np.concatenate([phi, nphi])
    zz = np.concatenate([z, nz])
    pid = np.concatenate([c["tid"], np.full(n_noise, -1)]).astype(np.int32)
    x = (rr * np.cos(pp)).astype(np.float32)
    y = (rr * np.sin(pp)).astype(np.float32)
    zz = zz.astype(np.float32)
    if shuffle:
        perm = rng.permutation(len(x))
        x, y, zz, mod, side, pid = x[perm], y[perm], zz[perm], mod[perm], side[perm], pid[perm]
    seeds, seed_pid = (make_seeds(tracks, rng, smear=smear) if with_seeds
                       else (np.zeros((0, 3, 3), np.float32), np.zeros(0, np.int32)))
    return Event(x=x, y=y, z=zz, module=mod, side=side, pid=pid, seeds=seeds, seed_pid=seed_pid, tracks=tracks)


def make_seeds(tracks: Tracks, rng, smear=True):
    """Three pixel space points per track at r = 5, 10, 15 cm (one seed per track)."""
    ks, tl = tracks.kappa_s, tracks.tanl
    pts = []
    ok_all = np.ones(tracks.n, dtype=bool)
    for r in PIXEL_R:
        ok, s, phi, z = (cross_cylinder_from(ks, tracks.phi0, tl, tracks.x0, tracks.y0, tracks.z0, r)
                         if tracks.displaced else cross_cylinder(ks, tracks.phi0, tl, tracks.z0, r))
        ok_all &= ok
        if smear:
            phi = phi + rng.normal(0.0, PIXEL_SIGMA, tracks.n) / r
            z = z + rng.normal(0.0, PIXEL_SIGMA, tracks.n)
        pts.append(np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1))
    seeds = np.stack(pts, axis=1)[ok_all].astype(np.float32)
    return seeds, np.nonzero(ok_all)[0].astype(np.int32)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def tiny_event(seed=0, geom=None, smear=True):
    geom = geom or G.make_geometry(barrel_only=True)
    rng = np.random.default_rng(seed)
    tr = sample_tiny_tracks(rng, 10)
    return make_event(geom, tr, rng, n_noise=20 if smear else 0, smear=smear)


def pu200_event(seed=0, geom=None, n_tracks=8000, n_jet=12):
    geom = geom or G.make_geometry(barrel_only=False)
    rng = np.random.default_rng(seed)
    tr = sample_pileup_tracks(rng, n_tracks, n_jet=n_jet)
    return make_event(geom, tr, rng, noise_frac=0.02)


def sample_muon_gun(rng, n, pt_range=(2.0, 10.0), eta_max=2.4, cube=5.0):
    """Muons from vertices uniform in a cube of side `cube` cm centred on the interaction point (the
    displaced-track sample of Section 2.2): pT uniform in pt_range, |eta| < eta_max, phi uniform."""
    h = 0.5 * cube
    return Tracks(
        pt=rng.uniform(pt_range[0], pt_range[1], n),
        eta=rng.uniform(-eta_max, eta_max, n),
        phi0=rng.uniform(-math.pi, math.pi, n),
        q=rng.choice([-1.0, 1.0], n),
        z0=rng.uniform(-h, h, n),
        x0=rng.uniform(-h, h, n),
        y0=rng.uniform(-h, h, n),
    )


def muon_gun_event(seed, geom=None, n=20, pt_range=(2.0, 10.0), cube=5.0):
    """Zero-pileup event of n displaced muons (sample_muon_gun), one pixel seed per muon, no noise."""
    geom = geom or G.make_geometry(barrel_only=False)
    rng = np.random.default_rng(seed)
    tr = sample_muon_gun(rng, n, pt_range, cube=cube)
    return make_event(geom, tr, rng, n_noise=0)


def pileup_event(pu, seed, geom=None):
    geom = geom or G.make_geometry(barrel_only=False)
    rng = np.random.default_rng(seed)
    tr = sample_pileup_tracks(rng, int(40 * pu))
    return make_event(geom, tr, rng, noise_frac=0.02)
