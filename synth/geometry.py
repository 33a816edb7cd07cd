"""Synthetic CMS-like Phase-2 outer-tracker geometry.

This module is an input producer shared by the device path, the CPU oracle,
the tests and the benchmark. It lays out paired-sensor "pT modules" (two
closely spaced sensors per module, Section 2 of the paper) and locates points
on them; it holds none of the Segment Linking arithmetic.

Layout (all lengths in cm):

* Barrel: 6 layers whose lower sensor sits at r = 23, 36, 51, 68, 88, 108 and
  whose upper sensor sits DSEP = 0.26 further out. Each layer is tiled into
  16 phi x 10 z modules over |z| <= 120. Strip length 2.5 (layers 1-3) or
  5 (layers 4-6).
* Endcap: 5 disks per side whose lower sensor sits at |z| = 131, 156, 185,
  220, 267 and whose upper sensor sits 0.26 further from the interaction
  point. Each disk covers 23 <= r <= 110 with 16 rings of width 5.4375; ring
  k is cut into round(2 pi rbar_k / 5.4375) phi tiles, giving 1230 modules per
  disk and 13260 modules with the barrel. Rings whose centre lies below
  r = 60 are pixel-strip modules with 0.15 cm macro-pixels along r (as the CMS
  Phase-2 PS modules); rings above carry 5 cm strips.
* Strip pitch 90 um for every sensor, so the r-phi resolution is pitch/sqrt(12);
  the resolution along the strip (z in the barrel, r in the endcap) is
  strip length/sqrt(12).

Module numbering: barrel first, ordered by (layer, z tile, phi tile); then the
endcap ordered by (side -1 then +1, disk, ring, phi tile). Phi tiles start at
phi = -pi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

K_FIELD = 0.3          # GeV per (tesla * metre): R[m] = pT / (0.3 B)
B_FIELD = 3.8          # tesla, uniform along z
DSEP = 0.26            # sensor separation in a pT module (cm)
PITCH = 0.009          # strip pitch (cm)
BARREL_R = (23.0, 36.0, 51.0, 68.0, 88.0, 108.0)
BARREL_STRIP = (2.5, 2.5, 2.5, 5.0, 5.0, 5.0)
BARREL_ZMAX = 120.0
N_PHI_BARREL = 16
N_Z_BARREL = 10
DISK_Z = (131.0, 156.0, 185.0, 220.0, 267.0)
DISK_RMIN = 23.0
DISK_RMAX = 110.0
N_RING = 16
RING_WIDTH = (DISK_RMAX - DISK_RMIN) / N_RING      # 5.4375
ENDCAP_STRIP_SPLIT_R = 60.0
ENDCAP_STRIP_INNER = 0.15
ENDCAP_STRIP_OUTER = 5.0

SUBDET_BARREL = 0
SUBDET_ENDCAP = 1


def curvature_of_pt(pt):
    """Unsigned curvature 1/R in 1/cm for transverse momentum pt in GeV."""
    return K_FIELD * B_FIELD / (100.0 * np.asarray(pt, dtype=np.float64))


def pt_of_curvature(kappa):
    return K_FIELD * B_FIELD / (100.0 * np.asarray(kappa, dtype=np.float64))


@dataclass
class Geometry:
    barrel_only: bool
    n_mod: int
    subdet: np.ndarray      # int32, 0 barrel / 1 endcap
    layer: np.ndarray       # int32, barrel layer 1..6 or disk 1..5
    side: np.ndarray        # int32, 0 barrel, -1/+1 endcap side
    surf: np.ndarray        # float64, barrel: lower-sensor r; endcap: lower-sensor signed z
    dsep: np.ndarray        # float64, sensor separation
    sig_rphi: np.ndarray    # float64, r-phi resolution
    sig_long: np.ndarray    # float64, barrel: z resolution; endcap: r resolution
    strip: np.ndarray       # float64, strip length
    phi_lo: np.ndarray
    phi_hi: np.ndarray
    lo: np.ndarray          # barrel: z_lo; endcap: r_lo
    hi: np.ndarray          # barrel: z_hi; endcap: r_hi
    # lookup tables
    barrel_base: np.ndarray = field(repr=False, default=None)   # [6] first module id of each layer
    ring_nphi: np.ndarray = field(repr=False, default=None)     # [16]
    ring_base: np.ndarray = field(repr=False, default=None)     # [2 sides, 5 disks, 16 rings]

    # ---- locating points -------------------------------------------------
    def locate_barrel(self, layer_idx, phi, z):
        """Module id of barrel layer `layer_idx` (0-based) at (phi, z); -1 outside."""
        phi = np.asarray(phi, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        layer_idx = np.asarray(layer_idx)
        iphi = np.floor((np.mod(phi + math.pi, 2 * math.pi)) / (2 * math.pi / N_PHI_BARREL)).astype(np.int64)
        iphi = np.clip(iphi, 0, N_PHI_BARREL - 1)
        iz = np.floor((z + BARREL_ZMAX) / (2 * BARREL_ZMAX / N_Z_BARREL)).astype(np.int64)
        ok = (np.abs(z) <= BARREL_ZMAX) & (iz >= 0) & (iz < N_Z_BARREL)
        iz = np.clip(iz, 0, N_Z_BARREL - 1)
        mid = self.barrel_base[layer_idx] + iz * N_PHI_BARREL + iphi
        return np.where(ok, mid, -1)

    def locate_endcap(self, side, disk_idx, phi, r):
        """Module id of disk `disk_idx` (0-based) on `side` (+1/-1) at (phi, r); -1 outside."""
        if self.barrel_only:
            return np.full(np.shape(np.asarray(r)), -1, dtype=np.int64)
        phi = np.asarray(phi, dtype=np.float64)
        r = np.asarray(r, dtype=np.float64)
        ring = np.floor((r - DISK_RMIN) / RING_WIDTH).astype(np.int64)
        ok = (r >= DISK_RMIN) & (r <= DISK_RMAX)
        ring = np.clip(ring, 0, N_RING - 1)
        nphi = self.ring_nphi[ring]
        iphi = np.floor(np.mod(phi + math.pi, 2 * math.pi) / (2 * math.pi / nphi)).astype(np.int64)
        iphi = np.minimum(iphi, nphi - 1)
        s = (np.asarray(side) > 0).astype(np.int64)
        mid = self.ring_base[s, disk_idx, ring] + iphi
        return np.where(ok, mid, -1)

    def area(self):
        """Area of one sensor of each module (cm^2)."""
        a = np.where(
            self.subdet == SUBDET_BARREL,
            self.surf * (self.phi_hi - self.phi_lo) * (self.hi - self.lo),
            0.5 * (self.hi ** 2 - self.lo ** 2) * (self.phi_hi - self.phi_lo),
        )
        return a

    def module_table(self):
        """Columns handed to both the device library and the oracle."""
        return dict(
            subdet=self.subdet.astype(np.int32),
            layer=self.layer.astype(np.int32),
            surf=self.surf.astype(np.float32),
            dsep=self.dsep.astype(np.float32),
            sig_rphi=self.sig_rphi.astype(np.float32),
            sig_long=self.sig_long.astype(np.float32),
        )


def make_geometry(barrel_only: bool = False) -> Geometry:
    cols = {k: [] for k in ("subdet", "layer", "side", "surf", "strip", "phi_lo", "phi_hi", "lo", "hi")}
    barrel_base = np.zeros(len(BARREL_R), dtype=np.int64)
    dphi_b = 2 * math.pi / N_PHI_BARREL
    dz_b = 2 * BARREL_ZMAX / N_Z_BARREL
    mid = 0
    for li, r in enumerate(BARREL_R):
        barrel_base[li] = mid
        for iz in range(N_Z_BARREL):
            for ip in range(N_PHI_BARREL):
                cols["subdet"].append(SUBDET_BARREL)
                cols["layer"].append(li + 1)
                cols["side"].append(0)
                cols["surf"].append(r)
                cols["strip"].append(BARREL_STRIP[li])
                cols["phi_lo"].append(-math.pi + ip * dphi_b)
                cols["phi_hi"].append(-math.pi + (ip + 1) * dphi_b)
                cols["lo"].append(-BARREL_ZMAX + iz * dz_b)
                cols["hi"].append(-BARREL_ZMAX + (iz + 1) * dz_b)
                mid += 1
    ring_nphi = np.array(
        [int(round(2 * math.pi * (DISK_RMIN + (k + 0.5) * RING_WIDTH) / RING_WIDTH)) for k in range(N_RING)],
        dtype=np.int64,
    )
    ring_base = np.full((2, len(DISK_Z), N_RING), -1, dtype=np.int64)
    if not barrel_only:
        for si, side in enumerate((-1, +1)):
            for di, zd in enumerate(DISK_Z):
                for k in range(N_RING):
                    ring_base[si, di, k] = mid
                    r_lo = DISK_RMIN + k * RING_WIDTH
                    r_hi = r_lo + RING_WIDTH
                    rbar = 0.5 * (r_lo + r_hi)
                    n = ring_nphi[k]
                    for ip in range(n):
                        cols["subdet"].append(SUBDET_ENDCAP)
                        cols["layer"].append(di + 1)
                        cols["side"].append(side)
                        cols["surf"].append(side * zd)
                        cols["strip"].append(ENDCAP_STRIP_INNER if rbar < ENDCAP_STRIP_SPLIT_R else ENDCAP_STRIP_OUTER)
                        cols["phi_lo"].append(-math.pi + ip * 2 * math.pi / n)
                        cols["phi_hi"].append(-math.pi + (ip + 1) * 2 * math.pi / n)
                        cols["lo"].append(r_lo)
                        cols["hi"].append(r_hi)
                        mid += 1
    strip = np.array(cols["strip"], dtype=np.float64)
    g = Geometry(
        barrel_only=barrel_only,
        n_mod=mid,
        subdet=np.array(cols["subdet"], dtype=np.int32),
        layer=np.array(cols["layer"], dtype=np.int32),
        side=np.array(cols["side"], dtype=np.int32),
        surf=np.array(cols["surf"], dtype=np.float64),
        dsep=np.full(mid, DSEP, dtype=np.float64),
        sig_rphi=np.full(mid, PITCH / math.sqrt(12.0), dtype=np.float64),
        sig_long=strip / math.sqrt(12.0),
        strip=strip,
        phi_lo=np.array(cols["phi_lo"]),
        phi_hi=np.array(cols["phi_hi"]),
        lo=np.array(cols["lo"]),
        hi=np.array(cols["hi"]),
        barrel_base=barrel_base,
        ring_nphi=ring_nphi,
        ring_base=ring_base,
    )
    return g
