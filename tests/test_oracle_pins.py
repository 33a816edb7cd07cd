"""Closed-form pins of the FP64 oracle's cut arithmetic.

Each test fixes a value by geometry (a noiseless helix, a point set on an
exact circle, a textbook regression identity, an independent numpy routine),
never by re-typing the oracle's own formula.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth import geometry as G
from synth import maps as M
from tests.helix_points import barrel_module, endcap_module, kappa_s, on_cylinder, on_plane, row

A_HALF = 0.3 * 3.8 / (200.0 * 0.8)     # 1 / (2 R_min) for pT_min = 0.8 GeV
DS = float(np.float32(G.DSEP))         # the module table carries the sensor separation as float32


@pytest.fixture(scope="module")
def P(geom_full, maps_full, cuts):
    return O.Predicates(O.Setup(geom_full.module_table(), maps_full, cuts))


def preds(geom, maps, cuts, **over):
    c = dict(cuts)
    c.update(over)
    return O.Predicates(O.Setup(geom.module_table(), maps, c))


# ---------------------------------------------------------------- MD
@pytest.mark.parametrize("li", range(6))
@pytest.mark.parametrize("q", [-1.0, 1.0])
def test_md_barrel_window_is_pt_min_helix(geom_full, maps_full, cuts, li, q):
    """With zero resolution terms the barrel MD window is attained exactly by a pT_min helix."""
    P0 = preds(geom_full, maps_full, cuts, n_md=0.0)
    r = G.BARREL_R[li]
    for scale, expect in ((1.0 + 1e-6, True), (1.0 - 1e-6, False)):
        pt = 0.8 * scale
        L, _ = on_cylinder(pt, q, 0.3, 0.7, 0.0, r)
        U, _ = on_cylinder(pt, q, 0.3, 0.7, 0.0, r + DS)
        m = barrel_module(geom_full, li, L)
        ok, d = P0.md(m, L, U)
        assert ok == expect
    L, _ = on_cylinder(0.8, q, 0.3, 0.7, 0.0, r)
    U, _ = on_cylinder(0.8, q, 0.3, 0.7, 0.0, r + DS)
    ok, d = P0.md(barrel_module(geom_full, li, L), L, U)
    closed = math.asin((r + DS) * A_HALF) - math.asin(r * A_HALF)
    assert abs(abs(d["dphi"]) - closed) < 1e-12
    assert math.copysign(1, d["dphi"]) == -q            # positive charge bends clockwise
    assert abs(d["thr_phi"] - closed) < 1e-12


@pytest.mark.parametrize("li", [0, 3, 5])
def test_md_barrel_dz_straight_track(geom_full, maps_full, cuts, li):
    """A straight track from z0 has dz = -dsep z0 / r; the window edge sits at z0 = z_lumi."""
    P0 = preds(geom_full, maps_full, cuts, n_md=0.0)
    r = G.BARREL_R[li]
    for z0, expect in ((20.0 * (1 - 1e-6), True), (20.0 * (1 + 1e-6), False), (0.0, True)):
        L, _ = on_cylinder(1e7, 1.0, 0.2, 0.4, z0, r)
        U, _ = on_cylinder(1e7, 1.0, 0.2, 0.4, z0, r + DS)
        ok, d = P0.md(barrel_module(geom_full, li, L), L, U)
        assert abs(d["dlong"] + DS * z0 / r) < 1e-12
        assert ok == expect


@pytest.mark.parametrize("di", range(5))
def test_md_endcap_closed_forms(P, geom_full, di):
    """Endcap MD: straight track gives dr = 0; a helix gives dphi = kappa_s dsep / (2 tan(lambda))."""
    zd = G.DISK_Z[di]
    L, _ = on_plane(1e7, 1.0, 1.9, 0.1, 0.0, zd)
    U, _ = on_plane(1e7, 1.0, 1.9, 0.1, 0.0, zd + DS)
    m = endcap_module(geom_full, 1, di, L)
    ok, d = P.md(m, L, U)
    assert ok and abs(d["dlong"]) < 1e-9
    for pt, q, eta, z0 in ((0.8, 1.0, 2.0, 15.0), (1.3, -1.0, 1.7, -19.0), (40.0, 1.0, 2.3, 3.0)):
        L, _ = on_plane(pt, q, eta, -2.0, z0, zd)
        if not (G.DISK_RMIN < math.hypot(L[0], L[1]) < G.DISK_RMAX):
            continue
        U, _ = on_plane(pt, q, eta, -2.0, z0, zd + DS)
        m = endcap_module(geom_full, 1, di, L)
        ok, d = P.md(m, L, U)
        assert ok
        assert abs(d["dphi"] - kappa_s(pt, q) * DS / (2 * math.sinh(eta))) < 1e-11


# ---------------------------------------------------------------- LS
def _md_pair(pt, q, eta, phi0, z0, li):
    r = G.BARREL_R[li]
    L, _ = on_cylinder(pt, q, eta, phi0, z0, r)
    U, _ = on_cylinder(pt, q, eta, phi0, z0, r + DS)
    return L, U


@pytest.mark.parametrize("li", range(5))
def test_ls_pointing_straight(geom_full, maps_full, cuts, li):
    P0 = preds(geom_full, maps_full, cuts, n_ls=0.0)
    for z0, expect in ((20.0 * (1 - 1e-6), True), (20.0 * (1 + 1e-6), False), (-7.0, True)):
        LA, UA = _md_pair(1e12, 1.0, 0.3, 1.0, z0, li)
        LB, UB = _md_pair(1e12, 1.0, 0.3, 1.0, z0, li + 1)
        ok, d = P0.ls(barrel_module(geom_full, li, LA), LA, UA, barrel_module(geom_full, li + 1, LB), LB, UB)
        den = math.hypot(LB[0], LB[1]) - math.hypot(LA[0], LA[1])
        assert abs(d["num"] / den - z0) < 1e-9
        assert abs(d["alpha_in"]) < 1e-9 and abs(d["alpha_out"]) < 1e-9
        assert ok == expect


@pytest.mark.parametrize("li", range(5))
@pytest.mark.parametrize("q", [-1.0, 1.0])
def test_ls_angles_pt_min_helix(geom_full, maps_full, cuts, li, q):
    """Position-angle change and both stub angles of a prompt helix, in closed form."""
    P0 = preds(geom_full, maps_full, cuts, n_ls=0.0)
    rA, rB = G.BARREL_R[li], G.BARREL_R[li + 1]
    ka = float(G.curvature_of_pt(0.8))
    for scale, expect in ((1 + 1e-6, True), (1 - 1e-6, False)):
        LA, UA = _md_pair(0.8 * scale, q, 0.2, -1.1, 0.0, li)
        LB, UB = _md_pair(0.8 * scale, q, 0.2, -1.1, 0.0, li + 1)
        ok, d = P0.ls(barrel_module(geom_full, li, LA), LA, UA, barrel_module(geom_full, li + 1, LB), LB, UB)
        assert ok == expect
    LA, UA = _md_pair(0.8, q, 0.2, -1.1, 0.0, li)
    LB, UB = _md_pair(0.8, q, 0.2, -1.1, 0.0, li + 1)
    ok, d = P0.ls(barrel_module(geom_full, li, LA), LA, UA, barrel_module(geom_full, li + 1, LB), LB, UB)
    asn = lambda r: math.asin(r * ka / 2)
    assert abs(d["dphi"] - (-q) * (asn(rB) - asn(rA))) < 1e-12
    assert abs(d["alpha_in"] - (-q) * (asn(rB) - asn(rA + DS))) < 1e-11
    assert abs(d["alpha_out"] - q * (asn(rB + DS) - asn(rA))) < 1e-11
    assert abs(d["thr_phi"] - (asn(rB) - asn(rA))) < 1e-12


# ---------------------------------------------------------------- three points
def _circle_points(cx, cy, R, thetas, z=None):
    pts = []
    for i, t in enumerate(thetas):
        pts.append([cx + R * math.cos(t), cy + R * math.sin(t), 0.0 if z is None else z[i]])
    return pts


@pytest.mark.parametrize("R", [70.0, 300.0, 5000.0])
@pytest.mark.parametrize("orient", [1, -1])
def test_t3_beta_and_kappa_on_circle(P, R, orient):
    cx, cy = 40.0, R + 10.0
    th0 = -math.pi / 2
    ths = [th0 + orient * d / R for d in (0.0, 14.0, 31.0)]
    pts = _circle_points(cx, cy, R, ths)
    rows = [row(p, 0.0026, 0.7, 0.0) for p in pts]
    ok, d = P.t3(rows)
    ab = math.dist(pts[0][:2], pts[1][:2])
    bc = math.dist(pts[1][:2], pts[2][:2])
    beta = math.asin(ab / (2 * R)) + math.asin(bc / (2 * R))
    assert abs(d["beta"] - orient * beta) < 1e-12
    assert abs(d["kappa"] - orient / R) < 1e-12 / R * 1e3


def test_t3_rz_helix_zero_and_failing(P):
    pts = []
    for r in (23.0, 36.0, 51.0):
        p, _ = on_cylinder(2.0, 1.0, 0.9, 1.3, 5.0, r)
        pts.append(p)
    rows = [row(p, 0.0026, 0.72, 0.0) for p in pts]
    ok, d = P.t3(rows)
    assert ok and abs(d["rz"]) < 1e-9 * d["thr_rz"]
    # move the outer anchor along z until the r-z residual crosses its window
    sB = math.dist(pts[0][:2], pts[1][:2])    # chord ~ arc at this curvature; exact offset found below
    for f, expect in ((0.98, True), (1.02, False)):
        lo, hi = 0.0, 50.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            r2 = [list(x) for x in rows]
            r2[2][2] += mid
            okm, dm = P.t3(r2)
            if abs(dm["rz"]) < dm["thr_rz"]:
                lo = mid
            else:
                hi = mid
        r2 = [list(x) for x in rows]
        r2[2][2] += f * lo
        okf, _ = P.t3(r2)
        assert okf == expect


# ---------------------------------------------------------------- fits
def _fit_rows(pts, srphi=0.0026, sz=0.7, sr=0.0):
    return [row(p, srphi, sz, sr) for p in pts]


@pytest.mark.parametrize("n", [5, 6, 8])
@pytest.mark.parametrize("R", [71.0, 900.0, 1e5])
def test_fit_exact_circle_and_helix(n, R):
    for q in (-1.0, 1.0):
        pt = R * 0.3 * 3.8 / 100.0
        radii = [5.0, 10.0, 15.0, 23.0, 36.0, 51.0, 68.0, 88.0][-n:] if n < 8 else [5.0, 10.0, 15.0, 23.0, 36.0,
                                                                                          51.0, 68.0, 88.0]
        pts = [on_cylinder(pt, q, 0.6, 0.9, -4.0, r)[0] for r in radii]
        kappa, chi2, chi2z, tanl = O.fit(_fit_rows(pts))
        assert abs(kappa - kappa_s(pt, q)) < 1e-9 * abs(kappa_s(pt, q)) + 1e-14
        assert chi2 < 1e-12 and chi2z < 1e-12
        assert abs(tanl - math.sinh(0.6)) < 1e-10


def _noisy_points(seed, n=5):
    rng = np.random.default_rng(seed)
    pts = [on_cylinder(1.7, 1.0, 0.4, 2.1, 1.0, r)[0] for r in (23.0, 36.0, 51.0, 68.0, 88.0, 108.0)[:n]]
    out = []
    for p in pts:
        r = math.hypot(p[0], p[1])
        phi = math.atan2(p[1], p[0]) + rng.normal(0, 0.0026) / r
        out.append([r * math.cos(phi), r * math.sin(phi), p[2] + rng.normal(0, 0.7)])
    return out


def test_fit_solution_matches_lstsq():
    """The circle coefficients are the least-squares solution (checked with numpy lstsq)."""
    for seed in range(5):
        pts = np.array(_noisy_points(seed))
        kappa, _, _, _ = O.fit(_fit_rows(pts))
        O_ = pts[2, :2]
        e = pts[4, :2] - pts[0, :2]
        xh = e / np.linalg.norm(e)
        yh = np.array([-xh[1], xh[0]])
        d = pts[:, :2] - O_
        xi, et = d @ xh, d @ yh
        A = np.stack([xi ** 2 + et ** 2, xi, np.ones_like(xi)], axis=1)
        (g, h, k), *_ = np.linalg.lstsq(A, et, rcond=None)
        # curvature of the circle g(x^2+y^2)+hx+k-y=0: centre (-h/2g, 1/2g), R^2 = |c|^2 - k/g
        cxy = np.array([-h / (2 * g), 1 / (2 * g)])
        R = math.sqrt(cxy @ cxy - k / g)
        assert abs(abs(kappa) - 1 / R) < 1e-9 / R


def test_fit_rotation_invariance():
    pts = _noisy_points(3)
    base = O.fit(_fit_rows(pts))
    for ang in (0.3, 2.0, -2.9):
        c, s = math.cos(ang), math.sin(ang)
        rot = [[c * p[0] - s * p[1], s * p[0] + c * p[1], p[2]] for p in pts]
        got = O.fit(_fit_rows(rot))
        assert np.allclose(got, base, rtol=1e-8, atol=1e-12)


def test_fit_sigma_scaling():
    pts = _noisy_points(4)
    a = O.fit(_fit_rows(pts, srphi=0.0026, sz=0.7))
    b = O.fit(_fit_rows(pts, srphi=0.0052, sz=1.4))
    assert abs(b[1] - a[1] / 4) < 1e-9 * a[1]
    assert abs(b[2] - a[2] / 4) < 1e-9 * a[2]


@pytest.mark.parametrize("j", range(5))
def test_rz_chi2_is_leverage_identity(j):
    """One z displaced by delta on an exact helix: chi2 = delta^2 (1 - h_jj) / sigma^2."""
    radii = (23.0, 36.0, 51.0, 68.0, 88.0)
    pts = [on_cylinder(3.0, -1.0, 0.5, 0.2, 2.0, r)[0] for r in radii]
    ka = abs(kappa_s(3.0, -1.0))
    s = np.array([2 * math.asin(math.dist(p[:2], pts[0][:2]) * ka / 2) / ka for p in pts])
    delta, sig = 0.9, 0.7
    pts[j] = pts[j].copy()
    pts[j][2] += delta
    _, _, chi2z, _ = O.fit(_fit_rows(pts, sz=sig))
    h = 1 / len(s) + (s[j] - s.mean()) ** 2 / ((s - s.mean()) ** 2).sum()
    assert abs(chi2z - delta ** 2 * (1 - h) / sig ** 2) < 1e-9


# ---------------------------------------------------------------- pLS
def _seed(pt, q, eta, phi0, z0):
    return np.array([on_cylinder(pt, q, eta, phi0, z0, r)[0] for r in (5.0, 10.0, 15.0)])


def test_pls_closed_form(P):
    rng = np.random.default_rng(11)
    for _ in range(50):
        pt = float(rng.uniform(0.5, 80)); q = float(rng.choice([-1.0, 1.0]))
        eta = float(rng.uniform(-2.4, 2.4)); phi0 = float(rng.uniform(-3.1, 3.1)); z0 = float(rng.normal(0, 5))
        d = P.pls(_seed(pt, q, eta, phi0, z0))
        assert abs(d["kappa"] - kappa_s(pt, q)) < 1e-9 * abs(kappa_s(pt, q))
        assert abs(d["pt"] - pt) < 1e-8 * pt
        assert abs(d["eta"] - eta) < 1e-9
        assert abs(math.remainder(d["phi0"] - phi0, 2 * math.pi)) < 1e-9
        assert abs(d["z0"] - z0) < 1e-8
        assert d["pass_"] == (pt >= 0.8 * 0.95 and abs(z0) <= 20.0)


def test_pls_window_edges(P):
    edge = 0.8 * (1 - 0.05)
    assert P.pls(_seed(edge * (1 + 1e-6), 1.0, 0.3, 0.1, 0.0))["pass_"]
    assert not P.pls(_seed(edge * (1 - 1e-6), 1.0, 0.3, 0.1, 0.0))["pass_"]
    assert P.pls(_seed(5.0, 1.0, 0.3, 0.1, 20.0 * (1 - 1e-6)))["pass_"]
    assert not P.pls(_seed(5.0, 1.0, 0.3, 0.1, 20.0 * (1 + 1e-6)))["pass_"]


def test_pls_superbin_matches_map_binning(P):
    """The oracle's superbin of a noiseless seed is the map's (independent numpy) binning of the truth."""
    rng = np.random.default_rng(12)
    p = M.MapParams()
    for _ in range(200):
        pt = float(rng.uniform(0.8, 50)); q = float(rng.choice([-1.0, 1.0]))
        eta = float(rng.uniform(-2.9, 2.9)); phi0 = float(rng.uniform(-3.1, 3.1))
        d = P.pls(_seed(pt, q, eta, phi0, 0.0))
        assert d["sb"] == int(M.superbin_index(eta, phi0, q, p))


# ---------------------------------------------------------------- T5 / pT5 / pT3
@pytest.mark.parametrize("pt", [0.81, 2.0, 50.0])
@pytest.mark.parametrize("q", [-1.0, 1.0])
def test_t5_noiseless_helix(P, pt, q):
    rows = []
    for r in (23.0, 36.0, 51.0, 68.0, 88.0):
        p, _ = on_cylinder(pt, q, 0.5, 2.5, -6.0, r)
        rows.append(row(p, 0.0026, 0.72, 0.0))
    ok, d = P.t5(rows)
    assert ok
    assert abs(d["dkappa"]) < 1e-12
    assert abs(d["kappa"] - kappa_s(pt, q)) < 1e-9 * abs(kappa_s(pt, q))
    assert d["chi2_rphi"] < 1e-12 and d["chi2_rz"] < 1e-12
    assert abs(d["eta"] - 0.5) < 1e-10
    assert abs(math.remainder(d["phi0"] - 2.5, 2 * math.pi)) < 1e-10


def test_t5_curvature_mismatch_fails(P):
    """Inner triplet from one helix, outer from another: the curvature-consistency cut rejects."""
    rows = []
    for i, r in enumerate((23.0, 36.0, 51.0, 68.0, 88.0)):
        pt = 2.0 if i <= 2 else 1.2
        p, _ = on_cylinder(pt, 1.0, 0.5, 2.5, 0.0, r)
        rows.append(row(p, 0.0026, 0.72, 0.0))
    ok, d = P.t5(rows)
    assert not ok and abs(d["dkappa"]) > d["thr_dkappa"]


@pytest.mark.parametrize("n_ot", [3, 5])
def test_pixel_objects_noiseless(P, n_ot):
    for q in (-1.0, 1.0):
        pt, eta, phi0, z0 = 3.3, -0.4, -0.6, 4.0
        rows = [row(on_cylinder(pt, q, eta, phi0, z0, r)[0], 0.001, 0.001, 0.0) for r in (5.0, 10.0, 15.0)]
        rows += [row(on_cylinder(pt, q, eta, phi0, z0, r)[0], 0.0026, 0.72, 0.0)
                 for r in (23.0, 36.0, 51.0, 68.0, 88.0)[:n_ot]]
        k = kappa_s(pt, q)
        ok, d = P.pt(rows, k, 1e-4, k, 1e-4)
        assert ok and d["chi2_rphi"] < 1e-12 and d["chi2_rz"] < 1e-12
        assert abs(d["kappa"] - k) < 1e-9 * abs(k)
        ok2, _ = P.pt(rows, k, 1e-5, -k, 1e-5)         # opposite-charge T object
        assert not ok2
