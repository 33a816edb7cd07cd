// Segment Linking (Line Segment Tracking) -- plain FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
// benchmark's CPU-baseline leg may load this library. It is the slow,
// obviously correct restatement of the method against which the device
// library is checked; it shares no code, header or table with it.
//
// The paper (arXiv:2209.13711, Section 2.1 and Fig. KernelFlow) describes the
// object chain qualitatively: stubs (mini-doublets, MD) from hit pairs in one
// pT module inside a 0.8 GeV window (Section 2, Fig. pTModule); segments (LS)
// linking MDs of compatible modules (Fig. CompModules); triplets (T3) from two
// LS sharing an MD and quintuplets (T5) from two T3 sharing an MD, with a
// relative-angle requirement (Fig. GeomReqs); pixel line segments (pLS) linked
// to T3/T5 into pT3/pT5; then cross-cleaning in the paper's order and the
// track-candidate (TC) collection. The paper prints no formula, so every cut
// below is this project's reading, written out once here in the order the
// paper gives the steps, with plain nested loops and no blocking or fusion.
//
// Inputs are the same float32 hits the device sees, widened to double.
// Every cut is evaluated as "v <= thr". A candidate whose every cut passes or
// lies within margin_rel * |thr| of its threshold, with at least one inside
// that margin, is recorded in the level's margin list (its decision may flip
// between FP32 and FP64 arithmetic).
//
// Units: cm, GeV, tesla, radians.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <set>
#include <vector>

namespace {

struct OGeom {
    int32_t n_mod;
    const int32_t* subdet;     // 0 barrel, 1 endcap
    const int32_t* layer;
    const float* surf;         // unused by the cuts; kept for completeness
    const float* dsep;
    const float* sig_rphi;
    const float* sig_long;     // barrel: z resolution, endcap: r resolution
    const int32_t* conn_off;   // [n_mod+1]
    const int32_t* conn_tgt;
    const int32_t* sb_off;     // [n_sb+1]
    const int32_t* sb_tgt;
    int32_t n_sb;
};

struct OCfg {
    double pt_min, k_field, b_field, z_lumi;
    double n_md, n_ls, n_t3, n_t5, n_pt;
    double tol_r;                        // |kappa| <= (1 + tol_r) * 2a
    double chi2_rphi_t5, chi2_rz_t5;
    double chi2_rphi_pt3, chi2_rz_pt3;
    double chi2_rphi_pt5, chi2_rz_pt5;
    double pls_pt_tol, sig_pix;
    double sb_eta_max;
    int32_t sb_n_eta, sb_n_phi;
    double dr_clean;
    double margin_rel;
};

struct OEvent {
    int32_t n_hits;
    const float* x;
    const float* y;
    const float* z;
    const int32_t* module;
    const uint8_t* side;
    int32_t n_seeds;
    const float* seeds;        // [n_seeds][3 points][x,y,z]
};

// A measured space point with its resolutions.
struct Pt {
    double x, y, z, r;
    double srphi;   // along phi-hat
    double sz;      // along z (barrel, pixel)
    double sr;      // along r-hat (endcap)
};

struct MD { int lo, up, mod; Pt a; double dx, dy, dz; double dphi, dlong, thr_phi, thr_long; int margin; };
struct LS { int md_in, md_out; double dphi, thr_phi; int margin; };
struct T3 { int ls_in, ls_out; double beta, thr_beta, kappa, sigk, rz, thr_rz; int margin; };
struct T5 { int t3_in, t3_out; double kappa, chi2_rphi, chi2_rz, eta, phi0, pt, score, sigk; int margin; };
struct PLS { int seed, pass, sb; double kappa, sigk, eta, phi0, z0, pt; int margin; };
struct PT { int seed, obj; double kappa, chi2_rphi, chi2_rz, score, pt; int margin; };
struct TC { int type, seed, obj; int hits[10]; double pt, eta, phi0; };

struct Result {
    std::vector<MD> md;
    std::vector<LS> ls;
    std::vector<T3> t3;
    std::vector<T5> t5;
    std::vector<PLS> pls;
    std::vector<PT> pt3, pt5;
    std::vector<TC> tc;
    std::vector<std::array<int, 2>> m_md, m_ls, m_t3, m_t5, m_pt3, m_pt5;
    std::vector<int> m_pls;
    std::vector<std::array<int, 4>> m_clean;   // (cat, idx, cat, idx)
};

// --------------------------------------------------------------------------
// small helpers
// --------------------------------------------------------------------------
const double PI = 3.14159265358979323846;

inline double sq(double v) { return v * v; }
inline double asinc(double v) { return std::asin(std::min(1.0, std::max(0.0, v))); }
inline double wrap(double p) {
    while (p > PI) p -= 2 * PI;
    while (p <= -PI) p += 2 * PI;
    return p;
}
inline double sgn(double v) { return v < 0 ? -1.0 : 1.0; }

// Transverse arc length along a circle of curvature k subtending chord c.
inline double arc(double c, double k) { return k > 0 ? 2.0 * std::asin(std::min(1.0, c * k / 2.0)) / k : c; }

// One cut "v <= thr": returns false on a clear failure; flags `near` when v
// lies within the margin of thr.
struct Cuts {
    double m;
    bool near = false;
    bool fail = false;
    explicit Cuts(double margin) : m(margin) {}
    // returns the FP64 decision v <= thr
    bool operator()(double v, double thr) {
        if (std::fabs(v - thr) <= m * std::fabs(thr)) near = true;
        else if (v > thr) fail = true;
        return v <= thr;
    }
};

double half_curv_max(const OCfg& c) {   // a = 1/(2 R_min), R_min[cm] = 100 pT_min / (k B)
    return c.k_field * c.b_field / (200.0 * c.pt_min);
}

Pt make_hit_point(const OGeom& g, const OEvent& e, int h) {
    Pt p;
    p.x = e.x[h]; p.y = e.y[h]; p.z = e.z[h];
    p.r = std::hypot(p.x, p.y);
    int m = e.module[h];
    p.srphi = g.sig_rphi[m];
    if (g.subdet[m] == 0) { p.sz = g.sig_long[m]; p.sr = 0.0; }
    else { p.sz = 0.0; p.sr = g.sig_long[m]; }
    return p;
}

Pt make_pixel_point(const OCfg& c, const float* q) {
    Pt p;
    p.x = q[0]; p.y = q[1]; p.z = q[2];
    p.r = std::hypot(p.x, p.y);
    p.srphi = c.sig_pix; p.sz = c.sig_pix; p.sr = 0.0;
    return p;
}

// Error of point P perpendicular to a chord of unit direction (cx, cy).
double sigma_perp(const Pt& P, double cx, double cy) {
    double rx = P.x / P.r, ry = P.y / P.r;
    double along_r = cx * rx + cy * ry;            // chord . r-hat
    double across_r = std::fabs(cx * ry - cy * rx); // |chord x r-hat|
    return std::sqrt(sq(P.srphi * along_r) + sq(P.sr * across_r));
}

// --------------------------------------------------------------------------
// Step 1: mini-doublet (stub) in one pT module (Section 2, Fig. pTModule).
// --------------------------------------------------------------------------
bool md_eval(const OGeom& g, const OCfg& c, int m, const Pt& L, const Pt& U, MD& out, bool& near) {
    const double a = half_curv_max(c);
    double dx = U.x - L.x, dy = U.y - L.y, dz = U.z - L.z;
    double rL = L.r;
    double dsep = g.dsep[m], sl = g.sig_long[m], srphi = g.sig_rphi[m];
    double dphi = std::atan2(L.x * dy - L.y * dx, L.x * U.x + L.y * U.y);
    double dlong, thr_phi, thr_long;
    if (g.subdet[m] == 0) {
        thr_phi = asinc((rL + dsep) * a) - asinc(rL * a) + c.n_md * std::sqrt(2.0) * srphi / rL;
        dlong = dz - dsep * L.z / rL;
        thr_long = c.n_md * std::sqrt(2.0) * sl + dsep * c.z_lumi / rL;
    } else {
        double rU = U.r;
        double az = std::fabs(L.z);
        dlong = (rU - rL) - dsep * rL / az;
        thr_long = c.n_md * std::sqrt(2.0) * sl;
        double ds_max = 1.2 * dsep * (rL + c.n_md * sl) / (az - c.z_lumi);
        thr_phi = a * ds_max + c.n_md * std::sqrt(2.0) * srphi / rL;
    }
    Cuts cut(c.margin_rel);
    bool ok = cut(std::fabs(dphi), thr_phi);
    if (!cut.fail) ok = cut(std::fabs(dlong), thr_long) && ok;
    near = cut.near && !cut.fail;
    out.a = L; out.dx = dx; out.dy = dy; out.dz = dz;
    out.dphi = dphi; out.dlong = dlong; out.thr_phi = thr_phi; out.thr_long = thr_long;
    return !cut.fail && ok;
}

// --------------------------------------------------------------------------
// Step 2: line segment between MDs of connected modules (Fig. CompModules).
// --------------------------------------------------------------------------
bool ls_eval(const OGeom& g, const OCfg& c, const MD& A, const MD& B, double& dphi_out, double& thr_out,
             bool& near, double* diag = nullptr) {
    const double a = half_curv_max(c);
    const Pt& P = A.a;
    const Pt& Q = B.a;
    Cuts cut(c.margin_rel);
    bool ok = true;
    // (i) the r-z line through both anchors points back into the luminous region
    double num = P.z * Q.r - Q.z * P.r;
    double den = Q.r - P.r;
    double sig_num = std::sqrt(sq(Q.r * P.sz) + sq(P.r * Q.sz) + sq(Q.z * P.sr) + sq(P.z * Q.sr));
    double thr_p = c.z_lumi * std::fabs(den) + c.n_ls * sig_num;
    ok = cut(std::fabs(num), thr_p) && ok;
    if (diag) { diag[0] = num; diag[1] = thr_p; }
    // (ii) position-angle change bounded by a pT_min helix from the origin
    double dphi = std::atan2(P.x * Q.y - P.y * Q.x, P.x * Q.x + P.y * Q.y);
    double thr_phi = asinc((Q.r + c.n_ls * Q.sr) * a) - asinc(std::max(0.0, P.r - c.n_ls * P.sr) * a) +
                     c.n_ls * std::sqrt(sq(P.srphi / P.r) + sq(Q.srphi / Q.r));
    if (!cut.fail) ok = cut(std::fabs(dphi), thr_phi) && ok;
    if (diag) { diag[2] = dphi; diag[3] = thr_phi; diag[4] = diag[6] = 0; diag[5] = diag[7] = -1; }
    // (iii) each barrel stub direction agrees with the segment direction
    double ux = Q.x - P.x, uy = Q.y - P.y;
    double lu = std::hypot(ux, uy);
    const MD* ends[2] = {&A, &B};
    for (int i = 0; i < 2 && !cut.fail; ++i) {
        const MD& X = *ends[i];
        if (g.subdet[X.mod] != 0) continue;
        double sx = X.dx, sy = X.dy;
        double ls_ = std::hypot(sx, sy);
        double alpha = std::atan2(sx * uy - sy * ux, sx * ux + sy * uy);
        double thr_a = asinc((Q.r + g.dsep[B.mod] + c.n_ls * Q.sr) * a) -
                       asinc(std::max(0.0, P.r - c.n_ls * P.sr) * a) +
                       c.n_ls * (std::sqrt(2.0) * X.a.srphi / ls_ + (P.sr + Q.sr) / lu);
        ok = cut(std::fabs(alpha), thr_a) && ok;
        if (diag) { diag[4 + 2 * i] = alpha; diag[5 + 2 * i] = thr_a; }
    }
    near = cut.near && !cut.fail;
    dphi_out = dphi;
    thr_out = thr_phi;
    return !cut.fail && ok;
}

// --------------------------------------------------------------------------
// Three-point quantities shared by T3, T5 and pLS (Section 2.1, Fig. GeomReqs)
// --------------------------------------------------------------------------
struct Tri {
    double lu, lv, lw, beta, sig_beta, kappa, sigk;
};

Tri tri(const Pt& A, const Pt& B, const Pt& C) {
    Tri t;
    double ux = B.x - A.x, uy = B.y - A.y;
    double vx = C.x - B.x, vy = C.y - B.y;
    double wx = C.x - A.x, wy = C.y - A.y;
    t.lu = std::hypot(ux, uy);
    t.lv = std::hypot(vx, vy);
    t.lw = std::hypot(wx, wy);
    t.beta = std::atan2(ux * vy - uy * vx, ux * vx + uy * vy);
    double sAu = sigma_perp(A, ux / t.lu, uy / t.lu);
    double sBu = sigma_perp(B, ux / t.lu, uy / t.lu);
    double sBv = sigma_perp(B, vx / t.lv, vy / t.lv);
    double sCv = sigma_perp(C, vx / t.lv, vy / t.lv);
    t.sig_beta = std::sqrt(sq(sAu / t.lu) + sq(sBu / t.lu + sBv / t.lv) + sq(sCv / t.lv));
    t.kappa = 2.0 * (ux * wy - uy * wx) / (t.lu * t.lv * t.lw);
    t.sigk = 2.0 * t.sig_beta / (t.lu + t.lv);
    return t;
}

// --------------------------------------------------------------------------
// Step 3: triplet from two LS sharing the middle MD (Fig. Triplet).
// --------------------------------------------------------------------------
bool t3_eval(const OCfg& c, const Pt& A, const Pt& B, const Pt& C, T3& o, bool& near) {
    const double a = half_curv_max(c);
    Tri t = tri(A, B, C);
    Cuts cut(c.margin_rel);
    double thr_beta = asinc(t.lu * a) + asinc(t.lv * a) + c.n_t3 * t.sig_beta;
    bool ok = cut(std::fabs(t.beta), thr_beta);
    double ka = std::fabs(t.kappa);
    double sB = arc(t.lu, ka), sC = arc(t.lw, ka);
    double d = (B.z - A.z) * sC - (C.z - A.z) * sB;
    double sig_d = std::sqrt(sq((sB - sC) * A.sz) + sq(sC * B.sz) + sq(sB * C.sz) + sq((C.z - B.z) * A.sr) +
                             sq((C.z - A.z) * B.sr) + sq((B.z - A.z) * C.sr));
    double thr_rz = c.n_t3 * sig_d;
    if (!cut.fail) ok = cut(std::fabs(d), thr_rz) && ok;
    near = cut.near && !cut.fail;
    o.beta = t.beta; o.thr_beta = thr_beta; o.kappa = t.kappa; o.sigk = t.sigk; o.rz = d; o.thr_rz = thr_rz;
    return !cut.fail && ok;
}

// --------------------------------------------------------------------------
// Circle fit in the chord frame and r-z line fit (T5, pT3, pT5).
//
// Frame: origin at the middle point P[n/2], x-axis along P[n-1] - P[0].
// The circle g (xi^2 + eta^2) + h xi + k - eta = 0 is the least-squares
// solution of eta_i ~ g rho_i^2 + h xi_i + k (an algebraic, Kasa-type fit
// normalised on the transverse coordinate; exact on an exact circle; to first
// order the unweighted geometric fit, since the algebraic residual of a point
// near the circle is S times its distance). Signed curvature kappa = 2g / S
// with S = sqrt(1 + h^2 - 4gk); residuals are geometric distances to the
// circle; each point's error is projected on the circle normal. The fit does
// not weight the points: where their projected errors differ (endcap strips,
// pixel points with outer-tracker points) chi2 exceeds n - 3 on average, by
// the factor its first-order expectation gives.
// --------------------------------------------------------------------------
struct Fit { double kappa, chi2_rphi, chi2_rz, tanl; };
// circle and line parameters of a fit (for the scoring features)
struct FitParams { double gg, hh, kk, S, xx, xy, ox, oy, c0, t, t_hat; };

bool solve3(double M[3][3], double b[3], double x[3]) {
    double A[3][4];
    for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) A[i][j] = M[i][j]; A[i][3] = b[i]; }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r) if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return false;
        if (piv != col) for (int j = 0; j < 4; ++j) std::swap(A[piv][j], A[col][j]);
        for (int r = col + 1; r < 3; ++r) {
            double f = A[r][col] / A[col][col];
            for (int j = col; j < 4; ++j) A[r][j] -= f * A[col][j];
        }
    }
    for (int i = 2; i >= 0; --i) {
        double s = A[i][3];
        for (int j = i + 1; j < 3; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return true;
}

// Variance of point P's error along the circle normal whose (unnormalised)
// components in the chord frame (x-hat = (xx, xy), y-hat = (-xy, xx)) are
// (nl_x, nl_y): srphi along phi-hat and sr along r-hat, projected; floored at
// (0.01 srphi)^2.
double normal_variance(const Pt& P, double nl_x, double nl_y, double xx, double xy) {
    double nx = nl_x * xx - nl_y * xy, ny = nl_x * xy + nl_y * xx;
    double nn = std::hypot(nx, ny);
    nx /= nn; ny /= nn;
    double rx = P.x / P.r, ry = P.y / P.r;
    double n_phi = -nx * ry + ny * rx;
    double n_r = nx * rx + ny * ry;
    return std::max(sq(P.srphi * n_phi) + sq(P.sr * n_r), sq(0.01 * P.srphi));
}

Fit fit_track(const Pt* P, int n, FitParams* fp = nullptr) {
    Fit f;
    const Pt& O = P[n / 2];
    double ex = P[n - 1].x - P[0].x, ey = P[n - 1].y - P[0].y;
    double le = std::hypot(ex, ey);
    double xx = ex / le, xy = ey / le;     // x-hat
    double yx = -xy, yy = xx;              // y-hat
    double xi[16], et[16], rho2[16];
    double M[3][3] = {{0}}, b[3] = {0};
    for (int i = 0; i < n; ++i) {
        double dx = P[i].x - O.x, dy = P[i].y - O.y;
        xi[i] = dx * xx + dy * xy;
        et[i] = dx * yx + dy * yy;
        rho2[i] = xi[i] * xi[i] + et[i] * et[i];
        double row[3] = {rho2[i], xi[i], 1.0};
        for (int p = 0; p < 3; ++p) {
            for (int q = 0; q < 3; ++q) M[p][q] += row[p] * row[q];
            b[p] += row[p] * et[i];
        }
    }
    double sol[3] = {0, 0, 0};
    if (!solve3(M, b, sol)) {
        f.kappa = 1e30; f.chi2_rphi = 1e30; f.chi2_rz = 1e30; f.tanl = 0;
        if (fp) *fp = FitParams{0, 0, 0, 1, xx, xy, O.x, O.y, 0, 0, 0};
        return f;
    }
    double gg = sol[0], hh = sol[1], kk = sol[2];
    double S = std::sqrt(std::max(0.0, 1.0 + hh * hh - 4.0 * gg * kk));
    f.kappa = 2.0 * gg / S;
    double chi2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double u = gg * rho2[i] + hh * xi[i] + kk - et[i];
        double e = 2.0 * u / (S + std::sqrt(std::max(0.0, S * S + 4.0 * gg * u)));
        chi2 += e * e / normal_variance(P[i], 2.0 * gg * xi[i] + hh, 2.0 * gg * et[i] - 1.0, xx, xy);
    }
    f.chi2_rphi = chi2;
    // r-z: z linear in the transverse arc length s measured from P[0]
    double ka = std::fabs(f.kappa);
    double s[16];
    for (int i = 0; i < n; ++i) s[i] = arc(std::hypot(P[i].x - P[0].x, P[i].y - P[0].y), ka);
    double t_hat = (P[n - 1].z - P[0].z) / s[n - 1];
    double w[16], W = 0, Ws = 0, Wz = 0;
    for (int i = 0; i < n; ++i) {
        w[i] = 1.0 / std::max(1e-12, sq(P[i].sz) + sq(t_hat * P[i].sr));
        W += w[i]; Ws += w[i] * s[i]; Wz += w[i] * P[i].z;
    }
    double sbar = Ws / W, zbar = Wz / W, Sss = 0, Ssz = 0;
    for (int i = 0; i < n; ++i) { Sss += w[i] * sq(s[i] - sbar); Ssz += w[i] * (s[i] - sbar) * (P[i].z - zbar); }
    double t = Ssz / Sss, c0 = zbar - t * sbar, chi2z = 0;
    for (int i = 0; i < n; ++i) chi2z += w[i] * sq(P[i].z - c0 - t * s[i]);
    f.chi2_rz = chi2z;
    f.tanl = t;
    if (fp) *fp = FitParams{gg, hh, kk, S, xx, xy, O.x, O.y, c0, t, t_hat};
    return f;
}

// ----------------------------------------------------------------------------
// Scoring features of a T5 (for an optional learned selection; the paper's
// own selection is the cut set above). Hits H[0..9] = (lower, upper) of the
// five MDs, anchors P = the lower hits; code = layer + 6 subdet.
//   f[0..9]   signed distance of each hit to the fitted circle over its error
//             projected on the circle normal, clipped to [-50, 50]
//   f[10..19] (z - line(s)) sqrt(w) of each hit (s: arc length from P[0] on the
//             fitted circle, w: the r-z fit weight), clipped to [-50, 50]
//   f[20..24] anchor radius / 100
//   f[25..27] inner-triplet, outer-triplet and fitted curvature over 2a
//   f[28..29] log(1 + chi2_rphi), log(1 + chi2_rz)
//   f[30..31] 10 x beta of the inner and outer triplet
//   f[32]     eta of the r-z fit
//   f[33..37] layer code / 11;  f[38..47] = 0
// ----------------------------------------------------------------------------
void t5_features(const OCfg& c, const Pt* P, const Pt* H, const int* code, double* f) {
    FitParams F;
    Fit fit = fit_track(P, 5, &F);
    Tri ti = tri(P[0], P[1], P[2]);
    Tri to = tri(P[2], P[3], P[4]);
    const double ka = std::fabs(fit.kappa);
    const double yx = -F.xy, yy = F.xx;
    auto clip = [](double v) { return std::min(50.0, std::max(-50.0, v)); };
    for (int j = 0; j < 10; ++j) {
        const Pt& Q = H[j];
        double dx = Q.x - F.ox, dy = Q.y - F.oy;
        double xi = dx * F.xx + dy * F.xy, et = dx * yx + dy * yy;
        double u = F.gg * (xi * xi + et * et) + F.hh * xi + F.kk - et;
        double e = 2.0 * u / (F.S + std::sqrt(std::max(0.0, F.S * F.S + 4.0 * F.gg * u)));
        double nlx = 2.0 * F.gg * xi + F.hh, nly = 2.0 * F.gg * et - 1.0;
        double nx = nlx * F.xx + nly * yx, ny = nlx * F.xy + nly * yy;
        double nn = std::hypot(nx, ny);
        nx /= nn; ny /= nn;
        double rx = Q.x / Q.r, ry = Q.y / Q.r;
        double s2 = std::max(sq(Q.srphi * (-nx * ry + ny * rx)) + sq(Q.sr * (nx * rx + ny * ry)), sq(0.01 * Q.srphi));
        f[j] = clip(e / std::sqrt(s2));
        double sj = arc(std::hypot(Q.x - P[0].x, Q.y - P[0].y), ka);
        double w = 1.0 / std::max(1e-12, sq(Q.sz) + sq(F.t_hat * Q.sr));
        f[10 + j] = clip((Q.z - F.c0 - F.t * sj) * std::sqrt(w));
    }
    for (int j = 0; j < 5; ++j) f[20 + j] = P[j].r / 100.0;
    const double two_a = 2.0 * half_curv_max(c);
    f[25] = ti.kappa / two_a;
    f[26] = to.kappa / two_a;
    f[27] = fit.kappa / two_a;
    f[28] = std::log1p(std::min(fit.chi2_rphi, 1e30));
    f[29] = std::log1p(std::min(fit.chi2_rz, 1e30));
    f[30] = 10.0 * ti.beta;
    f[31] = 10.0 * to.beta;
    f[32] = std::asinh(fit.tanl);
    for (int j = 0; j < 5; ++j) f[33 + j] = code[j] / 11.0;
    for (int j = 38; j < 48; ++j) f[j] = 0.0;
}

// ----------------------------------------------------------------------------
// Scoring features of a T3, in the T5's slots with the missing ones zero
// (the optional learned selection scores triplets too). Hits H[0..5] =
// (lower, upper) of the three MDs, anchors P = the lower hits.
//   f[0..5]   r-phi pulls of the six hits to the circle fitted to the three
//             anchors (exact through them), f[6..9] = 0
//   f[10..15] r-z pulls of the six hits to the weighted line of the fit,
//             f[16..19] = 0
//   f[20..22] anchor radius / 100, f[23..24] = 0
//   f[25]     triplet curvature over 2a, f[26] = 0, f[27] fitted curvature / 2a
//   f[28..29] log(1 + chi2_rphi), log(1 + chi2_rz)
//   f[30]     10 x beta, f[31] = 0
//   f[32]     eta of the r-z fit
//   f[33..35] layer code / 11; f[36..47] = 0
// ----------------------------------------------------------------------------
void t3_features(const OCfg& c, const Pt* P, const Pt* H, const int* code, double* f) {
    FitParams F;
    Fit fit = fit_track(P, 3, &F);
    Tri t = tri(P[0], P[1], P[2]);
    const double ka = std::fabs(fit.kappa);
    const double yx = -F.xy, yy = F.xx;
    auto clip = [](double v) { return std::min(50.0, std::max(-50.0, v)); };
    for (int j = 0; j < 48; ++j) f[j] = 0.0;
    for (int j = 0; j < 6; ++j) {
        const Pt& Q = H[j];
        double dx = Q.x - F.ox, dy = Q.y - F.oy;
        double xi = dx * F.xx + dy * F.xy, et = dx * yx + dy * yy;
        double u = F.gg * (xi * xi + et * et) + F.hh * xi + F.kk - et;
        double e = 2.0 * u / (F.S + std::sqrt(std::max(0.0, F.S * F.S + 4.0 * F.gg * u)));
        double s2 = normal_variance(Q, 2.0 * F.gg * xi + F.hh, 2.0 * F.gg * et - 1.0, F.xx, F.xy);
        f[j] = clip(e / std::sqrt(s2));
        double sj = arc(std::hypot(Q.x - P[0].x, Q.y - P[0].y), ka);
        double w = 1.0 / std::max(1e-12, sq(Q.sz) + sq(F.t_hat * Q.sr));
        f[10 + j] = clip((Q.z - F.c0 - F.t * sj) * std::sqrt(w));
    }
    for (int j = 0; j < 3; ++j) f[20 + j] = P[j].r / 100.0;
    const double two_a = 2.0 * half_curv_max(c);
    f[25] = t.kappa / two_a;
    f[27] = fit.kappa / two_a;
    f[28] = std::log1p(std::min(fit.chi2_rphi, 1e30));
    f[29] = std::log1p(std::min(fit.chi2_rz, 1e30));
    f[30] = 10.0 * t.beta;
    f[32] = std::asinh(fit.tanl);
    for (int j = 0; j < 3; ++j) f[33 + j] = code[j] / 11.0;
}

// Direction at the point of closest approach to the beam line, assuming a
// prompt track through P: phi0 = phi(P) + q asin(r |kappa| / 2), q = -sgn(kappa).
double phi0_of(const Pt& P, double kappa) {
    return wrap(std::atan2(P.y, P.x) - sgn(kappa) * asinc(P.r * std::fabs(kappa) / 2.0));
}

double pt_of(const OCfg& c, double kappa) {
    double ka = std::fabs(kappa);
    return ka > 0 ? c.k_field * c.b_field / (100.0 * ka) : 1e30;
}

// --------------------------------------------------------------------------
// Step 4: quintuplet from two T3 sharing an MD (Fig. Quintuplet).
// --------------------------------------------------------------------------
bool t5_eval(const OCfg& c, const Pt* P5, T5& o, bool& near, double* diag = nullptr) {
    const double a = half_curv_max(c);
    Cuts cut(c.margin_rel);
    Tri ti = tri(P5[0], P5[1], P5[2]);
    Tri to = tri(P5[2], P5[3], P5[4]);
    if (diag) { diag[0] = ti.kappa - to.kappa; diag[1] = c.n_t5 * std::sqrt(sq(ti.sigk) + sq(to.sigk)); }
    bool ok = cut(std::fabs(ti.kappa - to.kappa), c.n_t5 * std::sqrt(sq(ti.sigk) + sq(to.sigk)));
    Fit f = fit_track(P5, 5);
    if (!cut.fail) ok = cut(std::fabs(f.kappa), (1.0 + c.tol_r) * 2.0 * a) && ok;
    if (!cut.fail) ok = cut(f.chi2_rphi, c.chi2_rphi_t5) && ok;
    if (!cut.fail) ok = cut(f.chi2_rz, c.chi2_rz_t5) && ok;
    near = cut.near && !cut.fail;
    o.kappa = f.kappa; o.chi2_rphi = f.chi2_rphi; o.chi2_rz = f.chi2_rz;
    o.eta = std::asinh(f.tanl); o.phi0 = phi0_of(P5[0], f.kappa); o.pt = pt_of(c, f.kappa);
    o.score = f.chi2_rphi + f.chi2_rz;
    o.sigk = 0.5 * std::sqrt(sq(ti.sigk) + sq(to.sigk));
    return !cut.fail && ok;
}

// --------------------------------------------------------------------------
// Step 5: pixel line segment from a 3-hit pixel seed (Section 2.1).
// --------------------------------------------------------------------------
void pls_eval(const OCfg& c, const Pt* Q, PLS& o, bool& near) {
    const double a = half_curv_max(c);
    Tri t = tri(Q[0], Q[1], Q[2]);
    double ka = std::fabs(t.kappa);
    double s1 = arc(t.lu, ka), s2 = arc(t.lw, ka);
    // unweighted line z = z_c + tanl * s through (0, z0), (s1, z1), (s2, z2)
    double sbar = (s1 + s2) / 3.0, zbar = (Q[0].z + Q[1].z + Q[2].z) / 3.0;
    double Sss = sq(0 - sbar) + sq(s1 - sbar) + sq(s2 - sbar);
    double Ssz = (0 - sbar) * (Q[0].z - zbar) + (s1 - sbar) * (Q[1].z - zbar) + (s2 - sbar) * (Q[2].z - zbar);
    double tanl = Ssz / Sss;
    double zc = zbar - tanl * sbar;
    double z0 = zc - tanl * arc(Q[0].r, ka);
    o.kappa = t.kappa; o.sigk = t.sigk; o.eta = std::asinh(tanl); o.phi0 = phi0_of(Q[0], t.kappa);
    o.z0 = z0; o.pt = pt_of(c, t.kappa);
    Cuts cut(c.margin_rel);
    bool ok = cut(ka, 2.0 * a / (1.0 - c.pls_pt_tol));
    if (!cut.fail) ok = cut(std::fabs(z0), c.z_lumi) && ok;
    o.pass = (!cut.fail && ok) ? 1 : 0;
    // superbin (eta bin, phi0 bin, charge); charge +1 <=> clockwise <=> kappa < 0
    double de = 2.0 * c.sb_eta_max / c.sb_n_eta;
    double dp = 2.0 * PI / c.sb_n_phi;
    double fe = (o.eta + c.sb_eta_max) / de;
    double fp = (o.phi0 + PI) / dp;
    long ie = (long)std::floor(fe);
    long ip = (long)std::floor(fp);
    if (ip < 0) ip = 0;
    if (ip > c.sb_n_phi - 1) ip = c.sb_n_phi - 1;
    int iq = t.kappa < 0 ? 1 : 0;
    o.sb = (ie >= 0 && ie < c.sb_n_eta) ? (int)((ie * c.sb_n_phi + ip) * 2 + iq) : -1;
    bool sb_near = std::fabs(fe - std::round(fe)) <= c.margin_rel || std::fabs(fp - std::round(fp)) <= c.margin_rel;
    near = (cut.near && !cut.fail) || (o.pass && sb_near);
}

// --------------------------------------------------------------------------
// Step 6: pT5 / pT3 = pLS linked to a T5 / T3 (Figs. PixelQuintuplet, PixelTriplet).
// --------------------------------------------------------------------------
bool pt_eval(const OCfg& c, const Pt* P, int n, double kappa_pls, double sigk_pls, double kappa_t,
             double sigk_t, double chi2_rphi_max, double chi2_rz_max, PT& o, bool& near, double* diag = nullptr) {
    const double a = half_curv_max(c);
    Cuts cut(c.margin_rel);
    if (diag) { diag[0] = kappa_pls - kappa_t; diag[1] = c.n_pt * std::sqrt(sq(sigk_pls) + sq(sigk_t)); }
    bool ok = cut(std::fabs(kappa_pls - kappa_t), c.n_pt * std::sqrt(sq(sigk_pls) + sq(sigk_t)));
    Fit f = fit_track(P, n);
    if (!cut.fail) ok = cut(std::fabs(f.kappa), (1.0 + c.tol_r) * 2.0 * a) && ok;
    if (!cut.fail) ok = cut(f.chi2_rphi, chi2_rphi_max) && ok;
    if (!cut.fail) ok = cut(f.chi2_rz, chi2_rz_max) && ok;
    near = cut.near && !cut.fail;
    o.kappa = f.kappa; o.chi2_rphi = f.chi2_rphi; o.chi2_rz = f.chi2_rz;
    o.score = f.chi2_rphi + f.chi2_rz; o.pt = pt_of(c, f.kappa);
    return !cut.fail && ok;
}

// --------------------------------------------------------------------------
// The chain
// --------------------------------------------------------------------------
struct Chain {
    const OGeom& g;
    const OCfg& c;
    const OEvent& e;
    Result& R;
    std::vector<std::vector<int>> lower, upper;   // hits per module, input order
    std::vector<std::vector<int>> md_of_mod;
    std::vector<std::vector<int>> ls_of_md;       // LS by inner MD
    std::vector<std::vector<int>> t3_of_md;       // T3 by inner MD
    std::vector<std::vector<int>> t5_of_md;       // T5 by inner MD

    Chain(const OGeom& g_, const OCfg& c_, const OEvent& e_, Result& R_) : g(g_), c(c_), e(e_), R(R_) {}

    void bin_hits() {
        lower.assign(g.n_mod, {});
        upper.assign(g.n_mod, {});
        for (int h = 0; h < e.n_hits; ++h) {
            int m = e.module[h];
            if (m < 0 || m >= g.n_mod) continue;
            (e.side[h] == 0 ? lower : upper)[m].push_back(h);
        }
    }

    void build_md() {
        md_of_mod.assign(g.n_mod, {});
        for (int m = 0; m < g.n_mod; ++m) {
            for (int hl : lower[m]) {
                for (int hu : upper[m]) {
                    Pt L = make_hit_point(g, e, hl), U = make_hit_point(g, e, hu);
                    MD md;
                    bool near = false;
                    bool pass = md_eval(g, c, m, L, U, md, near);
                    if (near) R.m_md.push_back({hl, hu});
                    if (!pass) continue;
                    md.lo = hl; md.up = hu; md.mod = m; md.margin = near;
                    md_of_mod[m].push_back((int)R.md.size());
                    R.md.push_back(md);
                }
            }
        }
    }

    void build_ls() {
        ls_of_md.assign(R.md.size(), {});
        for (int ia = 0; ia < (int)R.md.size(); ++ia) {
            int m1 = R.md[ia].mod;
            for (int j = g.conn_off[m1]; j < g.conn_off[m1 + 1]; ++j) {
                int m2 = g.conn_tgt[j];
                for (int ib : md_of_mod[m2]) {
                    double dphi, thr;
                    bool near = false;
                    bool pass = ls_eval(g, c, R.md[ia], R.md[ib], dphi, thr, near);
                    if (near) R.m_ls.push_back({ia, ib});
                    if (!pass) continue;
                    ls_of_md[ia].push_back((int)R.ls.size());
                    R.ls.push_back({ia, ib, dphi, thr, (int)near});
                }
            }
        }
    }

    void build_t3() {
        t3_of_md.assign(R.md.size(), {});
        for (int i1 = 0; i1 < (int)R.ls.size(); ++i1) {
            int mA = R.ls[i1].md_in, mB = R.ls[i1].md_out;
            for (int i2 : ls_of_md[mB]) {
                int mC = R.ls[i2].md_out;
                T3 o;
                bool near = false;
                bool pass = t3_eval(c, R.md[mA].a, R.md[mB].a, R.md[mC].a, o, near);
                if (near) R.m_t3.push_back({i1, i2});
                if (!pass) continue;
                o.ls_in = i1; o.ls_out = i2; o.margin = near;
                t3_of_md[mA].push_back((int)R.t3.size());
                R.t3.push_back(o);
            }
        }
    }

    void t3_anchors(int it, Pt* P) const {
        const T3& t = R.t3[it];
        P[0] = R.md[R.ls[t.ls_in].md_in].a;
        P[1] = R.md[R.ls[t.ls_in].md_out].a;
        P[2] = R.md[R.ls[t.ls_out].md_out].a;
    }
    int t3_inner_md(int it) const { return R.ls[R.t3[it].ls_in].md_in; }
    int t3_outer_md(int it) const { return R.ls[R.t3[it].ls_out].md_out; }

    void t5_anchors(int i5, Pt* P) const {
        t3_anchors(R.t5[i5].t3_in, P);
        Pt Q[3];
        t3_anchors(R.t5[i5].t3_out, Q);
        P[3] = Q[1];
        P[4] = Q[2];
    }

    void build_t5() {
        t5_of_md.assign(R.md.size(), {});
        for (int i1 = 0; i1 < (int)R.t3.size(); ++i1) {
            int mC = t3_outer_md(i1);
            for (int i2 : t3_of_md[mC]) {
                Pt P[5], Q[3];
                t3_anchors(i1, P);
                t3_anchors(i2, Q);
                P[3] = Q[1];
                P[4] = Q[2];
                T5 o;
                bool near = false;
                bool pass = t5_eval(c, P, o, near);
                if (near) R.m_t5.push_back({i1, i2});
                if (!pass) continue;
                o.t3_in = i1; o.t3_out = i2; o.margin = near;
                t5_of_md[t3_inner_md(i1)].push_back((int)R.t5.size());
                R.t5.push_back(o);
            }
        }
    }

    void seed_points(int s, Pt* Q) const {
        for (int j = 0; j < 3; ++j) Q[j] = make_pixel_point(c, e.seeds + 9 * s + 3 * j);
    }

    void build_pls() {
        for (int s = 0; s < e.n_seeds; ++s) {
            Pt Q[3];
            seed_points(s, Q);
            PLS o;
            bool near = false;
            pls_eval(c, Q, o, near);
            o.seed = s; o.margin = near;
            if (near) R.m_pls.push_back(s);
            R.pls.push_back(o);
        }
    }

    // pT5 (launched before pT3, Fig. KernelFlow)
    void build_pt5() {
        for (int s = 0; s < e.n_seeds; ++s) {
            const PLS& p = R.pls[s];
            if (!p.pass || p.sb < 0) continue;
            for (int j = g.sb_off[p.sb]; j < g.sb_off[p.sb + 1]; ++j) {
                int m = g.sb_tgt[j];
                for (int ia : md_of_mod[m]) {
                    for (int i5 : t5_of_md[ia]) {
                        Pt P[8];
                        seed_points(s, P);
                        t5_anchors(i5, P + 3);
                        PT o;
                        bool near = false;
                        bool pass = pt_eval(c, P, 8, p.kappa, p.sigk, R.t5[i5].kappa, R.t5[i5].sigk,
                                            c.chi2_rphi_pt5, c.chi2_rz_pt5, o, near);
                        if (near) R.m_pt5.push_back({s, i5});
                        if (!pass) continue;
                        o.seed = s; o.obj = i5; o.margin = near;
                        R.pt5.push_back(o);
                    }
                }
            }
        }
    }

    void build_pt3() {
        for (int s = 0; s < e.n_seeds; ++s) {
            const PLS& p = R.pls[s];
            if (!p.pass || p.sb < 0) continue;
            for (int j = g.sb_off[p.sb]; j < g.sb_off[p.sb + 1]; ++j) {
                int m = g.sb_tgt[j];
                for (int ia : md_of_mod[m]) {
                    for (int i3 : t3_of_md[ia]) {
                        Pt P[6];
                        seed_points(s, P);
                        t3_anchors(i3, P + 3);
                        Tri tt = tri(P[3], P[4], P[5]);
                        PT o;
                        bool near = false;
                        bool pass = pt_eval(c, P, 6, p.kappa, p.sigk, tt.kappa, tt.sigk, c.chi2_rphi_pt3,
                                            c.chi2_rz_pt3, o, near);
                        if (near) R.m_pt3.push_back({s, i3});
                        if (!pass) continue;
                        o.seed = s; o.obj = i3; o.margin = near;
                        R.pt3.push_back(o);
                    }
                }
            }
        }
    }

    // ---- hit lists of the TC-eligible objects --------------------------
    // OT hits are their input index; the three pixel hits of seed s are
    // n_hits + 3 s + j.
    void md_hits(int imd, std::vector<int>& out) const { out.push_back(R.md[imd].lo); out.push_back(R.md[imd].up); }
    void t3_mds(int it, int* m3) const { m3[0] = t3_inner_md(it); m3[1] = R.ls[R.t3[it].ls_in].md_out; m3[2] = t3_outer_md(it); }
    void t5_mds(int i5, int* m5) const {
        int a[3], b[3];
        t3_mds(R.t5[i5].t3_in, a);
        t3_mds(R.t5[i5].t3_out, b);
        m5[0] = a[0]; m5[1] = a[1]; m5[2] = a[2]; m5[3] = b[1]; m5[4] = b[2];
    }
    std::vector<int> hits_of(int cat, int i) const {
        std::vector<int> h;
        int m[5];
        if (cat == 0) {          // pT5
            for (int j = 0; j < 3; ++j) h.push_back(e.n_hits + 3 * R.pt5[i].seed + j);
            t5_mds(R.pt5[i].obj, m);
            for (int j = 0; j < 5; ++j) md_hits(m[j], h);
        } else if (cat == 1) {   // pT3
            for (int j = 0; j < 3; ++j) h.push_back(e.n_hits + 3 * R.pt3[i].seed + j);
            t3_mds(R.pt3[i].obj, m);
            for (int j = 0; j < 3; ++j) md_hits(m[j], h);
        } else if (cat == 2) {   // T5
            t5_mds(i, m);
            for (int j = 0; j < 5; ++j) md_hits(m[j], h);
        } else {                 // pLS
            for (int j = 0; j < 3; ++j) h.push_back(e.n_hits + 3 * R.pls[i].seed + j);
        }
        return h;
    }

    // ---- cross-cleaning (Section 2.1) ----------------------------------
    void clean_and_build_tc() {
        const int NC = 4;   // 0 pT5, 1 pT3, 2 T5, 3 pLS
        int n_obj[NC] = {(int)R.pt5.size(), (int)R.pt3.size(), (int)R.t5.size(), (int)R.pls.size()};
        std::vector<std::vector<int>> hits[NC];
        std::vector<double> score[NC], eta[NC], phi[NC];
        for (int cat = 0; cat < NC; ++cat) {
            hits[cat].resize(n_obj[cat]);
            for (int i = 0; i < n_obj[cat]; ++i) {
                hits[cat][i] = hits_of(cat, i);
                std::vector<int> sorted = hits[cat][i];
                std::sort(sorted.begin(), sorted.end());
                hits[cat][i] = sorted;
                double sc = 0, et = 0, ph = 0;
                if (cat == 0) { sc = R.pt5[i].score; et = R.pls[R.pt5[i].seed].eta; ph = R.pls[R.pt5[i].seed].phi0; }
                if (cat == 1) { sc = R.pt3[i].score; et = R.pls[R.pt3[i].seed].eta; ph = R.pls[R.pt3[i].seed].phi0; }
                if (cat == 2) { sc = R.t5[i].score; et = R.t5[i].eta; ph = R.t5[i].phi0; }
                if (cat == 3) { et = R.pls[i].eta; ph = R.pls[i].phi0; }
                score[cat].push_back(sc); eta[cat].push_back(et); phi[cat].push_back(ph);
            }
        }
        auto shares = [&](int c1, int i1, int c2, int i2) {
            const auto& a = hits[c1][i1];
            const auto& b = hits[c2][i2];
            size_t p = 0, q = 0;
            while (p < a.size() && q < b.size()) {
                if (a[p] == b[q]) return true;
                if (a[p] < b[q]) ++p; else ++q;
            }
            return false;
        };
        const double thr2 = c.dr_clean * c.dr_clean;
        auto dr2 = [&](int c1, int i1, int c2, int i2) {
            double de = eta[c1][i1] - eta[c2][i2];
            double dp = wrap(phi[c1][i1] - phi[c2][i2]);
            return de * de + dp * dp;
        };
        // a pair compared by the eta-phi distance records a margin if it is
        // within the margin of the threshold (on dR^2 the margin doubles)
        auto close = [&](int c1, int i1, int c2, int i2) {
            if (shares(c1, i1, c2, i2)) return true;
            double d = dr2(c1, i1, c2, i2);
            if (std::fabs(d - thr2) <= 2.0 * c.margin_rel * thr2) R.m_clean.push_back({c1, i1, c2, i2});
            return d < thr2;
        };
        // Step 1: duplicates inside one category: an object is dropped when
        // another object of the same category shares a hit with it and has a
        // smaller key (score, h, sorted hit tuple), h = FNV-1a of the sorted
        // hit tuple taken as 32-bit words (offset basis 2166136261, prime
        // 16777619). Objects whose MDs differ only by an upper hit have the
        // same anchors and hence exactly the same score; h orders them.
        std::vector<char> kept[NC];
        for (int cat = 0; cat < 3; ++cat) {
            kept[cat].assign(n_obj[cat], 1);
            std::vector<uint32_t> fnv(n_obj[cat]);
            for (int i = 0; i < n_obj[cat]; ++i) {
                uint32_t h = 2166136261u;
                for (int v : hits[cat][i]) { h ^= (uint32_t)v; h *= 16777619u; }
                fnv[i] = h;
            }
            std::map<int, std::vector<int>> by_hit;
            for (int i = 0; i < n_obj[cat]; ++i)
                for (int h : hits[cat][i]) by_hit[h].push_back(i);
            for (int i = 0; i < n_obj[cat]; ++i) {
                std::set<int> others;
                for (int h : hits[cat][i]) for (int j : by_hit[h]) if (j != i) others.insert(j);
                for (int j : others) {
                    double si = score[cat][i], sj = score[cat][j];
                    double d = std::fabs(si - sj);
                    if ((d > 0 && d <= c.margin_rel * std::max(std::fabs(si), std::fabs(sj))) ||
                        (d == 0 && fnv[i] == fnv[j]))
                        R.m_clean.push_back({cat, i, cat, j});
                    bool better = sj < si || (sj == si && (fnv[j] < fnv[i] ||
                                                           (fnv[j] == fnv[i] && hits[cat][j] < hits[cat][i])));
                    if (better) kept[cat][i] = 0;
                }
            }
        }
        kept[3].assign(n_obj[3], 1);
        // Step 2: pT3 close to (or sharing a hit with) any kept pT5
        for (int i = 0; i < n_obj[1]; ++i) {
            if (!kept[1][i]) continue;
            for (int j = 0; j < n_obj[0]; ++j)
                if (kept[0][j] && close(1, i, 0, j)) { kept[1][i] = 0; }
        }
        // Step 3: T5 against kept pT5 and cleaned pT3
        for (int i = 0; i < n_obj[2]; ++i) {
            if (!kept[2][i]) continue;
            for (int j = 0; j < n_obj[0]; ++j)
                if (kept[0][j] && close(2, i, 0, j)) kept[2][i] = 0;
            for (int j = 0; j < n_obj[1]; ++j)
                if (kept[1][j] && close(2, i, 1, j)) kept[2][i] = 0;
        }
        // Step 4: pLS used by a kept pT5/pT3 are linked; the remaining
        // passing pLS are cross-cleaned against all kept objects.
        std::vector<char> linked(e.n_seeds, 0);
        for (int j = 0; j < n_obj[0]; ++j) if (kept[0][j]) linked[R.pt5[j].seed] = 1;
        for (int j = 0; j < n_obj[1]; ++j) if (kept[1][j]) linked[R.pt3[j].seed] = 1;
        for (int i = 0; i < n_obj[3]; ++i) {
            if (!R.pls[i].pass || linked[i]) { kept[3][i] = 0; continue; }
            for (int cat = 0; cat < 3; ++cat)
                for (int j = 0; j < n_obj[cat]; ++j)
                    if (kept[cat][j] && close(3, i, cat, j)) kept[3][i] = 0;
        }
        // Track candidates
        for (int cat = 0; cat < NC; ++cat) {
            for (int i = 0; i < n_obj[cat]; ++i) {
                if (!kept[cat][i]) continue;
                TC t;
                t.type = cat; t.obj = i;
                std::fill(t.hits, t.hits + 10, -1);
                int m[5];
                int nm = 0;
                if (cat == 0) { t.seed = R.pt5[i].seed; t5_mds(R.pt5[i].obj, m); nm = 5; t.pt = R.pt5[i].pt; }
                if (cat == 1) { t.seed = R.pt3[i].seed; t3_mds(R.pt3[i].obj, m); nm = 3; t.pt = R.pt3[i].pt; }
                if (cat == 2) { t.seed = -1; t5_mds(i, m); nm = 5; t.pt = R.t5[i].pt; }
                if (cat == 3) { t.seed = i; t.pt = R.pls[i].pt; }
                for (int j = 0; j < nm; ++j) { t.hits[2 * j] = R.md[m[j]].lo; t.hits[2 * j + 1] = R.md[m[j]].up; }
                t.eta = eta[cat][i]; t.phi0 = phi[cat][i];
                R.tc.push_back(t);
            }
        }
    }

    void run(int upto) {
        bin_hits();
        build_md();
        if (upto >= 1) build_ls();
        if (upto >= 2) build_t3();
        if (upto >= 3) build_t5();
        if (upto >= 4) build_pls();
        if (upto >= 5) build_pt5();
        if (upto >= 6) build_pt3();
        if (upto >= 7) clean_and_build_tc();
    }
};

// Per-kind column counts of the flat accessors.
enum { K_MD = 0, K_LS, K_T3, K_T5, K_PLS, K_PT3, K_PT5, K_TC,
       K_M_MD = 10, K_M_LS, K_M_T3, K_M_T5, K_M_PLS, K_M_PT3, K_M_PT5, K_M_CLEAN };

}  // namespace

extern "C" {

// Ints per row / doubles per row of each kind (see oracle.py for the names).
int oracle_ncols(int kind, int want_doubles) {
    static const int ni[] = {4, 3, 3, 3, 4, 3, 3, 13};
    static const int nd[] = {4, 2, 6, 8, 6, 5, 5, 3};
    if (kind >= 0 && kind <= K_TC) return want_doubles ? nd[kind] : ni[kind];
    if (kind == K_M_PLS) return want_doubles ? 0 : 1;
    if (kind == K_M_CLEAN) return want_doubles ? 0 : 4;
    if (kind >= K_M_MD && kind <= K_M_PT5) return want_doubles ? 0 : 2;
    return -1;
}

void* oracle_run(const OGeom* g, const OCfg* c, const OEvent* e, int upto) {
    Result* R = new Result();
    Chain ch(*g, *c, *e, *R);
    ch.run(upto);
    return R;
}

void oracle_free(void* r) { delete (Result*)r; }

int oracle_count(void* rp, int kind) {
    Result& R = *(Result*)rp;
    switch (kind) {
        case K_MD: return (int)R.md.size();
        case K_LS: return (int)R.ls.size();
        case K_T3: return (int)R.t3.size();
        case K_T5: return (int)R.t5.size();
        case K_PLS: return (int)R.pls.size();
        case K_PT3: return (int)R.pt3.size();
        case K_PT5: return (int)R.pt5.size();
        case K_TC: return (int)R.tc.size();
        case K_M_MD: return (int)R.m_md.size();
        case K_M_LS: return (int)R.m_ls.size();
        case K_M_T3: return (int)R.m_t3.size();
        case K_M_T5: return (int)R.m_t5.size();
        case K_M_PLS: return (int)R.m_pls.size();
        case K_M_PT3: return (int)R.m_pt3.size();
        case K_M_PT5: return (int)R.m_pt5.size();
        case K_M_CLEAN: return (int)R.m_clean.size();
    }
    return -1;
}

void oracle_fetch(void* rp, int kind, int32_t* I, double* D) {
    Result& R = *(Result*)rp;
    int ni = oracle_ncols(kind, 0), nd = oracle_ncols(kind, 1);
    int n = oracle_count(rp, kind);
    for (int i = 0; i < n; ++i) {
        int32_t* ir = I + (size_t)i * ni;
        double* dr = D ? D + (size_t)i * nd : nullptr;
        switch (kind) {
            case K_MD: { const MD& o = R.md[i]; ir[0] = o.lo; ir[1] = o.up; ir[2] = o.mod; ir[3] = o.margin;
                dr[0] = o.dphi; dr[1] = o.dlong; dr[2] = o.thr_phi; dr[3] = o.thr_long; break; }
            case K_LS: { const LS& o = R.ls[i]; ir[0] = o.md_in; ir[1] = o.md_out; ir[2] = o.margin;
                dr[0] = o.dphi; dr[1] = o.thr_phi; break; }
            case K_T3: { const T3& o = R.t3[i]; ir[0] = o.ls_in; ir[1] = o.ls_out; ir[2] = o.margin;
                dr[0] = o.beta; dr[1] = o.thr_beta; dr[2] = o.kappa; dr[3] = o.sigk; dr[4] = o.rz; dr[5] = o.thr_rz; break; }
            case K_T5: { const T5& o = R.t5[i]; ir[0] = o.t3_in; ir[1] = o.t3_out; ir[2] = o.margin;
                dr[0] = o.kappa; dr[1] = o.chi2_rphi; dr[2] = o.chi2_rz; dr[3] = o.eta; dr[4] = o.phi0; dr[5] = o.pt;
                dr[6] = o.score; dr[7] = o.sigk; break; }
            case K_PLS: { const PLS& o = R.pls[i]; ir[0] = o.seed; ir[1] = o.pass; ir[2] = o.sb; ir[3] = o.margin;
                dr[0] = o.kappa; dr[1] = o.sigk; dr[2] = o.eta; dr[3] = o.phi0; dr[4] = o.z0; dr[5] = o.pt; break; }
            case K_PT3: case K_PT5: { const PT& o = (kind == K_PT3 ? R.pt3 : R.pt5)[i];
                ir[0] = o.seed; ir[1] = o.obj; ir[2] = o.margin;
                dr[0] = o.kappa; dr[1] = o.chi2_rphi; dr[2] = o.chi2_rz; dr[3] = o.score; dr[4] = o.pt; break; }
            case K_TC: { const TC& o = R.tc[i]; ir[0] = o.type; ir[1] = o.seed; ir[2] = o.obj;
                for (int j = 0; j < 10; ++j) ir[3 + j] = o.hits[j];
                dr[0] = o.pt; dr[1] = o.eta; dr[2] = o.phi0; break; }
            case K_M_MD: ir[0] = R.m_md[i][0]; ir[1] = R.m_md[i][1]; break;
            case K_M_LS: ir[0] = R.m_ls[i][0]; ir[1] = R.m_ls[i][1]; break;
            case K_M_T3: ir[0] = R.m_t3[i][0]; ir[1] = R.m_t3[i][1]; break;
            case K_M_T5: ir[0] = R.m_t5[i][0]; ir[1] = R.m_t5[i][1]; break;
            case K_M_PT3: ir[0] = R.m_pt3[i][0]; ir[1] = R.m_pt3[i][1]; break;
            case K_M_PT5: ir[0] = R.m_pt5[i][0]; ir[1] = R.m_pt5[i][1]; break;
            case K_M_PLS: ir[0] = R.m_pls[i]; break;
            case K_M_CLEAN: for (int j = 0; j < 4; ++j) ir[j] = R.m_clean[i][j]; break;
        }
    }
}

// ---- single-candidate predicates for the brute-force completeness tests ----
// Each builds its MDs from explicit hits (indices into the event) and returns
// 1 when every cut passes. *near receives the margin flag.

static bool md_from_hits(const OGeom* g, const OCfg* c, const OEvent* e, int hl, int hu, MD& md, bool& near) {
    int m = e->module[hl];
    if (e->module[hu] != m || e->side[hl] != 0 || e->side[hu] != 1) return false;
    Pt L = make_hit_point(*g, *e, hl), U = make_hit_point(*g, *e, hu);
    md.lo = hl; md.up = hu; md.mod = m;
    return md_eval(*g, *c, m, L, U, md, near);
}

int oracle_pred_md(const OGeom* g, const OCfg* c, const OEvent* e, int hl, int hu, int* near) {
    MD md;
    bool nr = false;
    bool p = md_from_hits(g, c, e, hl, hu, md, nr);
    *near = nr;
    return p;
}

// hits: 2 per MD (lower, upper), n_md MDs; kind: 1 LS (2 MDs), 2 T3 (3), 3 T5 (5)
int oracle_pred_chain(const OGeom* g, const OCfg* c, const OEvent* e, const int32_t* hits, int kind, int* near) {
    int n_md = kind == 1 ? 2 : (kind == 2 ? 3 : 5);
    MD md[5];
    *near = 0;
    for (int i = 0; i < n_md; ++i) {   // anchors and stubs only: the MD cuts are not applied here
        bool nr = false;
        int m = e->module[hits[2 * i]];
        Pt L = make_hit_point(*g, *e, hits[2 * i]), U = make_hit_point(*g, *e, hits[2 * i + 1]);
        md_eval(*g, *c, m, L, U, md[i], nr);
        md[i].lo = hits[2 * i]; md[i].up = hits[2 * i + 1]; md[i].mod = m;
    }
    bool nr = false;
    if (kind == 1) {
        double dp, th;
        int ok = ls_eval(*g, *c, md[0], md[1], dp, th, nr);
        *near = nr;
        return ok;
    }
    Pt P[5];
    for (int i = 0; i < n_md; ++i) P[i] = md[i].a;
    if (kind == 2) { T3 o; int ok = t3_eval(*c, P[0], P[1], P[2], o, nr); *near = nr; return ok; }
    T5 o;
    int ok = t5_eval(*c, P, o, nr);
    *near = nr;
    return ok;
}

// pLS fields for one seed: out = {pass, sb}, dout = {kappa, sigk, eta, phi0, z0, pt}
void oracle_pls(const OCfg* c, const float* seed9, int32_t* out, double* dout) {
    Pt Q[3];
    for (int j = 0; j < 3; ++j) Q[j] = make_pixel_point(*c, seed9 + 3 * j);
    PLS o;
    bool near = false;
    pls_eval(*c, Q, o, near);
    out[0] = o.pass; out[1] = o.sb; out[2] = near;
    dout[0] = o.kappa; dout[1] = o.sigk; dout[2] = o.eta; dout[3] = o.phi0; dout[4] = o.z0; dout[5] = o.pt;
}

// Fit of n points given as (x, y, z, srphi, sz, sr) rows: out = {kappa, chi2_rphi, chi2_rz, tanl}
void oracle_fit(const double* rows, int n, double* out) {
    Pt P[16];
    for (int i = 0; i < n; ++i) {
        P[i].x = rows[6 * i]; P[i].y = rows[6 * i + 1]; P[i].z = rows[6 * i + 2];
        P[i].r = std::hypot(P[i].x, P[i].y);
        P[i].srphi = rows[6 * i + 3]; P[i].sz = rows[6 * i + 4]; P[i].sr = rows[6 * i + 5];
    }
    Fit f = fit_track(P, n);
    out[0] = f.kappa; out[1] = f.chi2_rphi; out[2] = f.chi2_rz; out[3] = f.tanl;
}

// Three-point quantities of (x, y, z, srphi, sz, sr) rows: {beta, sig_beta, kappa, sigk}
void oracle_tri(const double* rows, double* out) {
    Pt P[3];
    for (int i = 0; i < 3; ++i) {
        P[i].x = rows[6 * i]; P[i].y = rows[6 * i + 1]; P[i].z = rows[6 * i + 2];
        P[i].r = std::hypot(P[i].x, P[i].y);
        P[i].srphi = rows[6 * i + 3]; P[i].sz = rows[6 * i + 4]; P[i].sr = rows[6 * i + 5];
    }
    Tri t = tri(P[0], P[1], P[2]);
    out[0] = t.beta; out[1] = t.sig_beta; out[2] = t.kappa; out[3] = t.sigk;
}


// ---- FP64-input entry points for the closed-form pins ----------------------
static Pt pt_from_row(const double* r) {
    Pt P;
    P.x = r[0]; P.y = r[1]; P.z = r[2]; P.r = std::hypot(P.x, P.y);
    P.srphi = r[3]; P.sz = r[4]; P.sr = r[5];
    return P;
}

static Pt module_point(const OGeom* g, int m, const double* xyz) {
    double row[6] = {xyz[0], xyz[1], xyz[2], g->sig_rphi[m], g->subdet[m] == 0 ? g->sig_long[m] : 0.0,
                     g->subdet[m] == 0 ? 0.0 : g->sig_long[m]};
    return pt_from_row(row);
}

// out = {dphi, dlong, thr_phi, thr_long, near}
int oracle_md_d(const OGeom* g, const OCfg* c, int m, const double* L, const double* U, double* out) {
    MD md;
    bool near = false;
    bool ok = md_eval(*g, *c, m, module_point(g, m, L), module_point(g, m, U), md, near);
    out[0] = md.dphi; out[1] = md.dlong; out[2] = md.thr_phi; out[3] = md.thr_long; out[4] = near;
    return ok;
}

// out = {num, thr_p, dphi, thr_phi, alpha_in, thr_in, alpha_out, thr_out, near}; thr_* = -1 when not applied
int oracle_ls_d(const OGeom* g, const OCfg* c, int mA, const double* LA, const double* UA, int mB,
                const double* LB, const double* UB, double* out) {
    MD A, B;
    bool nr = false;
    md_eval(*g, *c, mA, module_point(g, mA, LA), module_point(g, mA, UA), A, nr);
    md_eval(*g, *c, mB, module_point(g, mB, LB), module_point(g, mB, UB), B, nr);
    A.mod = mA; B.mod = mB;
    double dp, th;
    bool near = false;
    for (int i = 0; i < 8; ++i) out[i] = 0;
    out[5] = out[7] = -1;
    bool ok = ls_eval(*g, *c, A, B, dp, th, near, out);
    out[8] = near;
    return ok;
}

// rows [3][6]; out = {beta, thr_beta, kappa, sigk, rz, thr_rz, near}
int oracle_t3_d(const OCfg* c, const double* rows, double* out) {
    T3 o;
    bool near = false;
    bool ok = t3_eval(*c, pt_from_row(rows), pt_from_row(rows + 6), pt_from_row(rows + 12), o, near);
    out[0] = o.beta; out[1] = o.thr_beta; out[2] = o.kappa; out[3] = o.sigk; out[4] = o.rz; out[5] = o.thr_rz;
    out[6] = near;
    return ok;
}

// rows [5][6]; out = {dkappa, thr_dkappa, kappa, chi2_rphi, chi2_rz, eta, phi0, pt, score, near, sigk}
int oracle_t5_d(const OCfg* c, const double* rows, double* out) {
    Pt P[5];
    for (int i = 0; i < 5; ++i) P[i] = pt_from_row(rows + 6 * i);
    T5 o;
    bool near = false;
    bool ok = t5_eval(*c, P, o, near, out);
    out[2] = o.kappa; out[3] = o.chi2_rphi; out[4] = o.chi2_rz; out[5] = o.eta; out[6] = o.phi0; out[7] = o.pt;
    out[8] = o.score; out[9] = near; out[10] = o.sigk;
    return ok;
}

// seed as doubles [3][3]; iout = {pass, sb, near}; dout = {kappa, sigk, eta, phi0, z0, pt}
void oracle_pls_d(const OCfg* c, const double* q, int32_t* iout, double* dout) {
    Pt Q[3];
    for (int j = 0; j < 3; ++j) {
        double row[6] = {q[3 * j], q[3 * j + 1], q[3 * j + 2], c->sig_pix, c->sig_pix, 0.0};
        Q[j] = pt_from_row(row);
    }
    PLS o;
    bool near = false;
    pls_eval(*c, Q, o, near);
    iout[0] = o.pass; iout[1] = o.sb; iout[2] = near;
    dout[0] = o.kappa; dout[1] = o.sigk; dout[2] = o.eta; dout[3] = o.phi0; dout[4] = o.z0; dout[5] = o.pt;
}

// pT3 (n = 6) / pT5 (n = 8) on rows [n][6] (3 pixel rows first);
// out = {kappa, chi2_rphi, chi2_rz, score, near, dkappa, thr_dkappa}
int oracle_pt_d(const OCfg* c, const double* rows, int n, double kappa_pls, double sigk_pls, double kappa_t,
                double sigk_t, double* out) {
    Pt P[8];
    for (int i = 0; i < n; ++i) P[i] = pt_from_row(rows + 6 * i);
    PT o;
    bool near = false;
    bool ok = pt_eval(*c, P, n, kappa_pls, sigk_pls, kappa_t, sigk_t, n == 8 ? c->chi2_rphi_pt5 : c->chi2_rphi_pt3,
                      n == 8 ? c->chi2_rz_pt5 : c->chi2_rz_pt3, o, near, out + 5);
    out[0] = o.kappa; out[1] = o.chi2_rphi; out[2] = o.chi2_rz; out[3] = o.score; out[4] = near;
    return ok;
}


// Features of the T5 formed by five MDs given as (lower, upper) hit pairs of
// the event: out[48].
void oracle_t5_features(const OGeom* g, const OCfg* c, const OEvent* e, const int32_t* md_hits, double* out) {
    Pt P[5], H[10];
    int code[5];
    for (int j = 0; j < 5; ++j) {
        int hl = md_hits[2 * j], hu = md_hits[2 * j + 1];
        P[j] = make_hit_point(*g, *e, hl);
        H[2 * j] = P[j];
        H[2 * j + 1] = make_hit_point(*g, *e, hu);
        int m = e->module[hl];
        code[j] = g->layer[m] + (g->subdet[m] ? 6 : 0);
    }
    t5_features(*c, P, H, code, out);
}

// Features of the T3 formed by three MDs given as (lower, upper) hit pairs
// of the event: out[48].
void oracle_t3_features(const OGeom* g, const OCfg* c, const OEvent* e, const int32_t* md_hits, double* out) {
    Pt P[3], H[6];
    int code[3];
    for (int j = 0; j < 3; ++j) {
        int hl = md_hits[2 * j], hu = md_hits[2 * j + 1];
        P[j] = make_hit_point(*g, *e, hl);
        H[2 * j] = P[j];
        H[2 * j + 1] = make_hit_point(*g, *e, hu);
        int m = e->module[hl];
        code[j] = g->layer[m] + (g->subdet[m] ? 6 : 0);
    }
    t3_features(*c, P, H, code, out);
}

}  // extern "C"
