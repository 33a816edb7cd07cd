"""Module connectivity map and pixel-seed superbin map (input data).

Both maps are lookup tables handed, unchanged, to the device library and to
the oracle; the method only reads them.

Connectivity map (Section 2.1, Fig. CompModules): for every module m1, the
modules m2 on the NEXT lower-sensor surface that a helix can cross after m1,
for helices from (0, 0, z0) with |z0| <= z_lumi, either charge and transverse
momentum at or above the threshold (|kappa| <= 2a, a = 1/(2 R_min)). The scan
samples, for each module, a grid of points on its lower sensor (edges
included) times a grid of curvatures and the two z0 extremes, propagates to
the next surface crossed, and keeps the bounding box (in phi and in z or r)
of the crossings on each next surface, widened by a safety margin; every
module tile that overlaps a box is connected. The crossings of the true
tracks of a few generated events are added, as the paper adds transitions
seen in simulated tracks.

Superbin map (Section 2.1, pixel line segments): a pixel seed falls into
superbin (eta bin, phi0 bin, charge). For each superbin the map lists the
modules of the first two lower-sensor surfaces that helices from that bin
(pT >= pT_min (1 - tol), |z0| <= z_lumi) cross. Built with the same scan.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass

import numpy as np

from . import geometry as G
from .helix import cross_cylinder, cross_cylinder_from, cross_plane, cross_plane_from, wrap_phi


@dataclass
class MapParams:
    pt_min: float = 0.8
    z_lumi: float = 20.0
    n_eta: int = 120          # superbin eta bins over [-eta_max, eta_max]
    eta_max: float = 3.0
    n_phi: int = 72           # superbin phi0 bins over [-pi, pi)
    pt_tol: float = 0.05      # pLS keep pT >= pt_min (1 - pt_tol)
    margin_cm: float = 1.0    # widening of every bounding box (cm)
    sim_events: int = 4       # generated events whose true transitions are added
    d0_max: float = 0.0       # transverse vertex displacement the connection map also covers (cm)

    @property
    def kappa_max(self):
        return float(G.curvature_of_pt(self.pt_min))


@dataclass
class ConnMap:
    offsets: np.ndarray   # int32 [n_mod + 1]
    targets: np.ndarray   # int32


def lower_surfaces(geom):
    """Lower-sensor surfaces: (kind, value, layer_idx, side)."""
    out = [(0, r, li, 0) for li, r in enumerate(G.BARREL_R)]
    if not geom.barrel_only:
        for sgn in (-1, +1):
            for di, zd in enumerate(G.DISK_Z):
                out.append((1, sgn * zd, di, sgn))
    return out


def _crossings_all(geom, ks, phi0, tanl, z0):
    """For every sample, crossing (valid, s, phi, ell) with each lower surface.

    ell is z on barrel surfaces and r on disks; module ids are resolved too.
    """
    surfs = lower_surfaces(geom)
    n = len(ks)
    ns = len(surfs)
    S = np.full((ns, n), np.inf)
    PHI = np.zeros((ns, n))
    ELL = np.zeros((ns, n))
    MOD = np.full((ns, n), -1, dtype=np.int64)
    for j, (kind, val, li, sgn) in enumerate(surfs):
        if kind == 0:
            ok, s, phi, z = cross_cylinder(ks, phi0, tanl, z0, val)
            mid = geom.locate_barrel(np.full(n, li), phi, z)
            ell = z
        else:
            ok, s, phi, r = cross_plane(ks, phi0, tanl, z0, val)
            mid = geom.locate_endcap(np.full(n, sgn), li, phi, r)
            ell = r
        ok = ok & (mid >= 0)
        S[j] = np.where(ok, s, np.inf)
        PHI[j] = phi
        ELL[j] = ell
        MOD[j] = np.where(ok, mid, -1)
    return surfs, S, PHI, ELL, MOD


def _crossings_from(geom, tr):
    """As _crossings_all, for tracks with transverse production vertices (tr.x0, tr.y0)."""
    surfs = lower_surfaces(geom)
    n = tr.n
    S = np.full((len(surfs), n), np.inf)
    PHI = np.zeros((len(surfs), n))
    ELL = np.zeros((len(surfs), n))
    MOD = np.full((len(surfs), n), -1, dtype=np.int64)
    for j, (kind, val, li, sgn) in enumerate(surfs):
        if kind == 0:
            ok, s, phi, z = cross_cylinder_from(tr.kappa_s, tr.phi0, tr.tanl, tr.x0, tr.y0, tr.z0, val)
            mid = geom.locate_barrel(np.full(n, li), phi, z)
            ell = z
        else:
            ok, s, phi, r = cross_plane_from(tr.kappa_s, tr.phi0, tr.tanl, tr.x0, tr.y0, tr.z0, val)
            mid = geom.locate_endcap(np.full(n, sgn), li, phi, r)
            ell = r
        ok = ok & (mid >= 0)
        S[j] = np.where(ok, s, np.inf)
        PHI[j] = phi
        ELL[j] = ell
        MOD[j] = np.where(ok, mid, -1)
    return surfs, S, PHI, ELL, MOD


def _surface_of_module(geom):
    surfs = lower_surfaces(geom)
    idx = {}
    for j, (kind, val, li, sgn) in enumerate(surfs):
        idx[(kind, li, sgn)] = j
    kind = (geom.subdet == G.SUBDET_ENDCAP).astype(int)
    return np.array([idx[(int(k), int(l) - 1, int(s))] for k, l, s in zip(kind, geom.layer, geom.side)])


def _tiles_in_box(geom, surf, phi_lo, phi_hi, ell_lo, ell_hi):
    """Module ids on surface `surf` whose tile overlaps the (phi, ell) box."""
    kind, val, li, sgn = surf
    out = []
    if phi_hi - phi_lo >= 2 * math.pi:
        phi_lo, phi_hi = -math.pi, math.pi - 1e-12
    if kind == 0:
        dz = 2 * G.BARREL_ZMAX / G.N_Z_BARREL
        iz0 = max(0, int(math.floor((ell_lo + G.BARREL_ZMAX) / dz)))
        iz1 = min(G.N_Z_BARREL - 1, int(math.floor((ell_hi + G.BARREL_ZMAX) / dz)))
        dphi = 2 * math.pi / G.N_PHI_BARREL
        ip0 = int(math.floor((phi_lo + math.pi) / dphi))
        ip1 = int(math.floor((phi_hi + math.pi) / dphi))
        ips = sorted({ip % G.N_PHI_BARREL for ip in range(ip0, ip1 + 1)})
        for iz in range(iz0, iz1 + 1):
            for ip in ips:
                out.append(int(geom.barrel_base[li] + iz * G.N_PHI_BARREL + ip))
    else:
        k0 = max(0, int(math.floor((ell_lo - G.DISK_RMIN) / G.RING_WIDTH)))
        k1 = min(G.N_RING - 1, int(math.floor((ell_hi - G.DISK_RMIN) / G.RING_WIDTH)))
        s = 1 if sgn > 0 else 0
        for k in range(k0, k1 + 1):
            nphi = int(geom.ring_nphi[k])
            dphi = 2 * math.pi / nphi
            ip0 = int(math.floor((phi_lo + math.pi) / dphi))
            ip1 = int(math.floor((phi_hi + math.pi) / dphi))
            ips = sorted({ip % nphi for ip in range(ip0, ip1 + 1)})
            for ip in ips:
                out.append(int(geom.ring_base[s, li, k] + ip))
    return out


class _Boxes:
    """Per (group, surface) bounding boxes of crossings, in phi relative to a
    per-group reference angle and in ell (z on barrel surfaces, r on disks)."""

    def __init__(self, n_groups, n_surf, phi_ref):
        self.ns = n_surf
        self.phi_ref = phi_ref
        self.dmin = np.full(n_groups * n_surf, np.inf)
        self.dmax = np.full(n_groups * n_surf, -np.inf)
        self.lmin = np.full(n_groups * n_surf, np.inf)
        self.lmax = np.full(n_groups * n_surf, -np.inf)

    def add(self, group, surf_idx, phi, ell):
        key = group * self.ns + surf_idx
        d = wrap_phi(phi - self.phi_ref[group])
        np.minimum.at(self.dmin, key, d)
        np.maximum.at(self.dmax, key, d)
        np.minimum.at(self.lmin, key, ell)
        np.maximum.at(self.lmax, key, ell)

    def lists(self, geom, margin):
        surfs = lower_surfaces(geom)
        n_groups = len(self.dmin) // self.ns
        out = [set() for _ in range(n_groups)]
        for u in np.nonzero(np.isfinite(self.dmin))[0]:
            g, j = divmod(int(u), self.ns)
            kind, val, li, sgn = surfs[j]
            lmin, lmax = self.lmin[u], self.lmax[u]
            rr = val if kind == 0 else max(G.DISK_RMIN, lmin - margin)
            mphi = margin / rr
            out[g].update(_tiles_in_box(geom, surfs[j], self.phi_ref[g] + self.dmin[u] - mphi,
                                        self.phi_ref[g] + self.dmax[u] + mphi, lmin - margin, lmax + margin))
        return out


def _to_csr(lists):
    off = np.zeros(len(lists) + 1, dtype=np.int64)
    for i, l in enumerate(lists):
        off[i + 1] = off[i] + len(l)
    tgt = np.concatenate([np.array(sorted(l), dtype=np.int64) for l in lists]) if off[-1] else np.zeros(0, np.int64)
    return off.astype(np.int32), tgt.astype(np.int32)


def _displaced_next(geom, M, ks, phi1, r1, z1, tanl, p: MapParams, turns=(-1.0, -0.5, 0.5, 1.0)):
    """Next-surface crossings of helices through the module points (phi1, r1, z1) whose direction there is
    turned from the prompt helix's by up to asin(d0_max / r1): a vertex displaced by d0 <= d0_max turns a
    track's direction at radius r by at most that angle. Returns (module, surface index, phi, ell)."""
    x1, y1 = r1 * np.cos(phi1), r1 * np.sin(phi1)
    ka = np.abs(ks)
    s1 = np.where(ka > 0, 2.0 * np.arcsin(np.minimum(r1 * ka / 2.0, 1.0)) / np.where(ka > 0, ka, 1.0), r1)
    theta_prompt = phi1 + ks * s1 / 2.0
    dmax = np.arcsin(np.minimum(1.0, p.d0_max / r1))
    surfs = lower_surfaces(geom)
    outs = []
    for f in turns:
        th = theta_prompt + f * dmax
        best = np.full(len(M), np.inf)
        best_j = np.full(len(M), -1)
        best_phi = np.zeros(len(M))
        best_ell = np.zeros(len(M))
        for j, (kind, val, li, sgn) in enumerate(surfs):
            if kind == 0:
                ok, s, phi, z = cross_cylinder_from(ks, th, tanl, x1, y1, z1, val)
                mid = geom.locate_barrel(np.full(len(M), li), phi, z)
                ell = z
            else:
                ok, s, phi, r = cross_plane_from(ks, th, tanl, x1, y1, z1, val)
                mid = geom.locate_endcap(np.full(len(M), sgn), li, phi, r)
                ell = r
            take = ok & (mid >= 0) & (s > 1e-6) & (s < best)
            best = np.where(take, s, best)
            best_j = np.where(take, j, best_j)
            best_phi = np.where(take, phi, best_phi)
            best_ell = np.where(take, ell, best_ell)
        good = best_j >= 0
        outs.append((M[good], best_j[good], best_phi[good], best_ell[good]))
    return [np.concatenate(c) for c in zip(*outs)]


def _module_samples(geom, p: MapParams, mods, n_grid=5, kappas=(-1.0, -0.5, 0.0, 0.5, 1.0)):
    """Helices through a grid of points of the lower sensor of modules `mods`."""
    kmax = p.kappa_max
    u = np.linspace(0.0, 1.0, n_grid)
    uu, vv = np.meshgrid(u, u, indexing="ij")
    uu, vv = uu.ravel(), vv.ravel()
    kk = np.array(kappas) * kmax
    z0s = np.array([-p.z_lumi, p.z_lumi])
    M, P, K, Z = np.meshgrid(mods, np.arange(len(uu)), np.arange(len(kk)), np.arange(len(z0s)), indexing="ij")
    M, P, K, Z = M.ravel(), P.ravel(), K.ravel(), Z.ravel()
    phi1 = geom.phi_lo[M] + uu[P] * (geom.phi_hi[M] - geom.phi_lo[M])
    l1 = geom.lo[M] + vv[P] * (geom.hi[M] - geom.lo[M])
    barrel = geom.subdet[M] == G.SUBDET_BARREL
    r1 = np.where(barrel, geom.surf[M], l1)
    z1 = np.where(barrel, l1, geom.surf[M])
    ks = kk[K]
    z0 = z0s[Z]
    ka = np.abs(ks)
    x = np.minimum(r1 * ka / 2.0, 1.0)
    s1 = np.where(ka > 0, 2.0 * np.arcsin(x) / np.where(ka > 0, ka, 1.0), r1)
    ok = (r1 * ka / 2.0 < 1.0) & (ka * s1 <= math.pi) & (z1 != z0)
    phi0 = phi1 - ks * s1 / 2.0
    tanl = (z1 - z0) / s1
    if p.d0_max > 0:
        return M[ok], ks[ok], phi0[ok], tanl[ok], z0[ok], s1[ok], (phi1[ok], r1[ok], z1[ok])
    return M[ok], ks[ok], phi0[ok], tanl[ok], z0[ok], s1[ok], None


def _next_after(S, s1):
    """Index of the surface crossed next after arc length s1 (or -1)."""
    Sx = np.where(S > s1[None, :] * (1 + 1e-9) + 1e-9, S, np.inf)
    j = np.argmin(Sx, axis=0)
    ok = np.isfinite(Sx[j, np.arange(S.shape[1])])
    return np.where(ok, j, -1)


def build_connection_map(geom, p: MapParams | None = None, sim_events=None, chunk=1500) -> ConnMap:
    p = p or MapParams()
    ns = len(lower_surfaces(geom))
    boxes = _Boxes(geom.n_mod, ns, 0.5 * (geom.phi_lo + geom.phi_hi))
    for c0 in range(0, geom.n_mod, chunk):
        mods = np.arange(c0, min(geom.n_mod, c0 + chunk))
        M, ks, phi0, tanl, z0, s1, pts = _module_samples(geom, p, mods)
        _, S, PHI, ELL, MOD = _crossings_all(geom, ks, phi0, tanl, z0)
        j = _next_after(S, s1)
        ok = j >= 0
        cols = np.arange(len(M))[ok]
        jj = j[ok]
        boxes.add(M[ok], jj, PHI[jj, cols], ELL[jj, cols])
        if pts is not None:
            Md, jd, phid, elld = _displaced_next(geom, M, ks, pts[0], pts[1], pts[2], tanl, p)
            boxes.add(Md, jd, phid, elld)
    lists = boxes.lists(geom, p.margin_cm)
    # transitions of the true tracks of generated events
    n_sim = p.sim_events if sim_events is None else sim_events
    if n_sim:
        from .events import sample_pileup_tracks, sample_tiny_tracks
        for e in range(n_sim):
            rng = np.random.default_rng(1000 + e)
            tr = (sample_tiny_tracks(rng, 2000) if geom.barrel_only
                  else sample_pileup_tracks(rng, 8000, n_jet=12))
            _, S2, _, _, MOD2 = _crossings_all(geom, tr.kappa_s, tr.phi0, tr.tanl, tr.z0)
            if p.d0_max > 0 and not geom.barrel_only:
                from .events import sample_muon_gun
                mu = sample_muon_gun(np.random.default_rng(2000 + e), 8000, pt_range=(p.pt_min, 20.0),
                                     cube=2.0 * p.d0_max / math.sqrt(2.0))
                _, S3, _, _, MOD3 = _crossings_from(geom, mu)
                S2 = np.concatenate([S2, S3], axis=1)
                MOD2 = np.concatenate([MOD2, MOD3], axis=1)
            order = np.argsort(S2, axis=0)
            Ms = np.take_along_axis(MOD2, order, axis=0)
            Ss = np.take_along_axis(S2, order, axis=0)
            for a in range(Ms.shape[0] - 1):
                good = np.isfinite(Ss[a]) & np.isfinite(Ss[a + 1]) & (Ms[a] >= 0) & (Ms[a + 1] >= 0)
                for m1, m2 in zip(Ms[a][good], Ms[a + 1][good]):
                    lists[int(m1)].add(int(m2))
    off, tgt = _to_csr(lists)
    return ConnMap(offsets=off, targets=tgt)


def superbin_index(eta, phi0, charge, p: MapParams):
    """Superbin of a seed; -1 when eta is outside the binned range."""
    eta = np.asarray(eta, dtype=np.float64)
    de = 2 * p.eta_max / p.n_eta
    ie = np.floor((eta + p.eta_max) / de).astype(np.int64)
    dp = 2 * math.pi / p.n_phi
    ip = np.clip(np.floor((np.asarray(phi0) + math.pi) / dp).astype(np.int64), 0, p.n_phi - 1)
    iq = (np.asarray(charge) > 0).astype(np.int64)
    sb = (ie * p.n_phi + ip) * 2 + iq
    return np.where((ie >= 0) & (ie < p.n_eta), sb, -1)


def build_superbin_map(geom, p: MapParams | None = None, n_eta_s=4, n_phi_s=3,
                       kappas=(0.0, 0.25, 0.5, 0.75, 1.0), z0_frac=(-1.0, -0.5, 0.0, 0.5, 1.0), chunk=1000):
    p = p or MapParams()
    nsb = p.n_eta * p.n_phi * 2
    de = 2 * p.eta_max / p.n_eta
    dp = 2 * math.pi / p.n_phi
    pad = 0.01
    ue = np.linspace(-pad / de, 1 + pad / de, n_eta_s)
    up = np.linspace(-pad / dp, 1 + pad / dp, n_phi_s)
    kmax = p.kappa_max / (1.0 - p.pt_tol)
    ns = len(lower_surfaces(geom))
    phi_ref = -math.pi + (np.arange(nsb) // 2 % p.n_phi + 0.5) * dp
    boxes = _Boxes(nsb, ns, phi_ref)
    for c0 in range(0, nsb, chunk):
        sbs = np.arange(c0, min(nsb, c0 + chunk))
        SB, E, P, K, Z = np.meshgrid(sbs, np.arange(n_eta_s), np.arange(n_phi_s), np.arange(len(kappas)),
                                     np.arange(len(z0_frac)), indexing="ij")
        SB, E, P, K, Z = SB.ravel(), E.ravel(), P.ravel(), K.ravel(), Z.ravel()
        iq = SB % 2
        ip = (SB // 2) % p.n_phi
        ie = SB // (2 * p.n_phi)
        eta = -p.eta_max + (ie + ue[E]) * de
        phi0 = -math.pi + (ip + up[P]) * dp
        q = np.where(iq == 1, 1.0, -1.0)
        ks = -q * np.array(kappas)[K] * kmax
        z0 = np.array(z0_frac)[Z] * p.z_lumi
        _, S, PHI, ELL, MOD = _crossings_all(geom, ks, phi0, np.sinh(eta), z0)
        order = np.argsort(S, axis=0)
        cols = np.arange(len(SB))
        for rank in (0, 1):
            jr = order[rank]
            ok = np.isfinite(S[jr, cols])
            boxes.add(SB[ok], jr[ok], PHI[jr[ok], cols[ok]], ELL[jr[ok], cols[ok]])
    return _to_csr(boxes.lists(geom, p.margin_cm))


# --------------------------------------------------------------------------
# cached construction
# --------------------------------------------------------------------------
_CACHE = {}


def _cache_dir():
    d = os.environ.get("LST_MAP_CACHE", os.path.join(os.path.dirname(os.path.dirname(__file__)), "_build", "maps"))
    os.makedirs(d, exist_ok=True)
    return d


def _version_tag():
    h = hashlib.sha1()
    for fn in ("maps.py", "geometry.py", "helix.py", "events.py"):
        with open(os.path.join(os.path.dirname(__file__), fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def load_maps(geom, p: MapParams | None = None):
    """(conn_offsets, conn_targets, sb_offsets, sb_targets), cached on disk."""
    p = p or MapParams()
    key = (geom.barrel_only, tuple(sorted(vars(p).items())))
    if key in _CACHE:
        return _CACHE[key]
    tag = hashlib.sha1(repr(key).encode()).hexdigest()[:12] + "_" + _version_tag()
    fn = os.path.join(_cache_dir(), f"maps_{tag}.npz")
    if os.path.exists(fn):
        d = np.load(fn)
        out = (d["co"], d["ct"], d["so"], d["st"])
    else:
        cm = build_connection_map(geom, p)
        so, st = build_superbin_map(geom, p)
        out = (cm.offsets, cm.targets, so, st)
        tmp = fn + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, co=out[0], ct=out[1], so=out[2], st=out[3])
        os.replace(tmp, fn)
    _CACHE[key] = out
    return out
