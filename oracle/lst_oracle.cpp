// CPU oracle for the Line Segment Tracking hot path (arXiv:2207.08207).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain, FP64 statement of what the GPU path
// computes. Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
// It shares no code, header, table or helper with the CUDA library: every formula here is written
// out from the paper's description and the readings of it listed at the top of each stage.
//
// Stages (paper Sec. 2 and Fig. "GPU implementation flowchart", Sec. 4.2):
//   hit binning by module (Sec. 4.2) -> Mini-Doublets (Sec. 2.2) -> Line Segments (Sec. 2.2)
//   -> Triplets (Sec. 2.3) -> Quintuplets (Sec. 2.3) -> pixel seeds, pT3, pT5 (Sec. 2.4)
//   -> cross-cleaning and Track Candidates (Sec. 2.5) -> track extensions (Sec. 2.5.1).
//
// The paper prints no cut formula or constant; each selection below is the reading fixed for this
// project (anchor hit = lower-sensor hit, cut windows from the pT threshold, luminous region and
// hit resolution, chi2 fits). Every cut is expressed as margin = bound - value >= 0; a candidate
// whose |margin| is within 1e-5 of max(|bound|, |value|) is "borderline" and reported as such.
//
// Parity-pinned by tests/test_oracle_pins.py (closed forms, single-helix invariants, Karimaki fit
// against a geometric least-squares fit) and tests/test_oracle_bruteforce.py (exhaustive all-pairs
// search on small events). Compiled with -O2 -ffp-contract=off (no fused multiply-add, no fast-math).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// constants (the value of each is the float32 literal, promoted to double)
// ---------------------------------------------------------------------------------------------
struct Params {
  double k;             // pT = k * R  [GeV/cm], 0.003 * 3.8 T
  double pt_thr;        // pT threshold, Sec. 2.2 (0.8 GeV)
  double sin_max;       // cap of sin(alpha) in alpha_thr
  double z_lum;         // luminous-region half length [cm]
  double d0_max;        // transverse impact-parameter allowance in MD/LS windows [cm]
  double n_sigma;
  double sigma_rphi;    // hit resolution r-phi [cm]
  double sigma_z;       // barrel hit resolution in z [cm]
  double sigma_r;       // endcap hit resolution in r [cm]
  double chi2_t3;       // T3 r-z chi2 cut
  double chi2_t5_c;     // T5 global circle-fit chi2 cut
  double chi2_t5_rz;    // T5 r-z chi2 cut
  double chi2_pt3_xy, chi2_pt3_rz, chi2_pt5_xy, chi2_pt5_rz;
  double f_t3;          // T3 pT estimate >= f_t3 * pt_thr
  double d0_t3;         // T3 circle impact parameter [cm]
  double c_rel, c_abs;  // T5 inner/outer curvature compatibility
  double dr_min;        // eta-phi cross-cleaning distance
  double pt_cap;        // cap on pT estimates [GeV]
  double pls_dir_err;   // pixel seed direction uncertainty [rad]
  double pls_pt_err;    // pixel seed relative pT uncertainty
  double sigma_floor;   // floor on r-z per-anchor uncertainties [cm]
  int t5_overlap_hits;  // T5 duplicate removal: >= this many shared hits (of 10)
};

// The pixel-bin layout: eta in [-2.5, 2.5) by 0.05 (index 20*eta + 50), phi by 2pi/128, charge.
constexpr int kPixNEta = 100;
constexpr int kPixNPhi = 128;
constexpr double kBorderRel = 1e-5;

Params default_params() {
  Params p;
  p.k = (double)0.0114f;
  p.pt_thr = (double)0.8f;
  p.sin_max = (double)0.95f;
  p.z_lum = (double)15.0f;
  p.d0_max = (double)0.1f;
  p.n_sigma = (double)3.0f;
  p.sigma_rphi = (double)0.003f;
  p.sigma_z = (double)0.1f;
  p.sigma_r = (double)0.1f;
  p.chi2_t3 = (double)9.0f;
  p.chi2_t5_c = (double)20.0f;
  p.chi2_t5_rz = (double)16.0f;
  p.chi2_pt3_xy = (double)16.0f;
  p.chi2_pt3_rz = (double)16.0f;
  p.chi2_pt5_xy = (double)25.0f;
  p.chi2_pt5_rz = (double)25.0f;
  p.f_t3 = (double)0.8f;
  p.d0_t3 = (double)2.0f;
  p.c_rel = (double)0.2f;
  p.c_abs = (double)1.5e-4f;
  p.dr_min = (double)0.01f;
  p.pt_cap = (double)1.0e4f;
  p.pls_dir_err = (double)1.0e-3f;
  p.pls_pt_err = (double)0.01f;
  p.sigma_floor = (double)1.0e-4f;
  p.t5_overlap_hits = 7;
  return p;
}

const double kPi = 3.14159265358979323846;
const double kTwoPi = 6.28318530717958647692;

double wrap_pi(double a) {  // to (-pi, pi]
  while (a > kPi) a -= kTwoPi;
  while (a <= -kPi) a += kTwoPi;
  return a;
}

// Decision bookkeeping for one candidate: pass = every margin >= 0 (the FP64 decision);
// borderline = some margin within kBorderRel of its scale and no other cut fails clearly.
struct Verdict {
  bool all_pass = true;
  bool clear_fail = false;
  bool border = false;
  double min_rel = 1e300;
  void cut(double bound, double value) {  // pass iff value <= bound
    double margin = bound - value;
    if (!(margin >= 0.0)) all_pass = false;  // NaN fails
    double scale = std::max(std::fabs(bound), std::fabs(value));
    double rel = scale > 0.0 ? std::fabs(margin) / scale : 0.0;
    if (!(rel == rel)) rel = 1e300;
    min_rel = std::min(min_rel, rel);
    if (rel <= kBorderRel) border = true;
    else if (!(margin >= 0.0)) clear_fail = true;
  }
  void cut_ge(double bound, double value) { cut(-bound, -value); }  // pass iff value >= bound
  void fail() { all_pass = false; clear_fail = true; }
  bool keep() const { return all_pass || (border && !clear_fail); }
  bool definite() const { return !border || clear_fail; }
};

// ---------------------------------------------------------------------------------------------
// input records (layout of the boundary structs)
// ---------------------------------------------------------------------------------------------
struct ModuleRec {
  int32_t id, subdet, layer, side, type;
  float surf, spacing, phi_lo, phi_hi, w_lo, w_hi;
};
struct PlsRec {
  float pt, eta, phi, x0, y0, z0;
  int32_t charge;
  int32_t pix_hit[4];
  int32_t pad;
};

// ---------------------------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------------------------
struct Hit { double x, y, z, r, phi; int32_t orig; int32_t sensor; int32_t module; int32_t endcap; };
// pass: the object exists under the FP64 decisions (its own cuts pass and every member exists);
// definite: neither it nor any member had a borderline cut. Candidates that fail only through a
// borderline cut are kept (pass = false, definite = false) so that the objects another rounding
// could build from them are known too.
struct MD {
  int32_t lo, up;  // indices into the binned hit list
  int32_t module;
  bool pass, definite;
  double dphichange, pt_est;
};
struct LS { int32_t md_in, md_out; bool pass, definite; double z0, dphi; };
struct T3 {
  int32_t ls_in, ls_out; int32_t md[3];
  bool pass, definite;
  double R, xc, yc, chi2_rz, pt_est;
};
struct T5 {
  int32_t t3_in, t3_out; int32_t md[5];
  bool pass, definite;
  double kappa_in, kappa_out, kappa_fit, chi2_c, chi2_rz, eta, phi, pt;
};
struct PObj {  // pT3 or pT5
  int32_t pls, obj; bool pass, definite; double chi2_xy, chi2_rz, score;
};
struct TC {
  int32_t type, obj;  // type 0 pT5, 1 pT3, 2 T5, 3 pLS; obj = index in its own table
  int32_t hits[14];
  double pt, eta, phi;
};

// Track extension of a track candidate (Sec. 2.5.1): the T3 that continues it outward, or t3 = -1.
struct TCExt {
  int32_t t3 = -1;       // extending T3 (index in the T3 table)
  int32_t n_add = 0;     // MDs added: 2 (the T3 shares the TC's last MD) or 1 (its last two MDs)
  bool definite = true;  // no candidate of this TC had a borderline cut, and its objects are definite
  double chi2_c = 0, chi2_rz = 0;
  int32_t hits[4] = {-1, -1, -1, -1};   // the added MDs' hits (lower, upper), inner -> outer
};

struct Geometry {
  int32_t n_mods;
  std::vector<ModuleRec> mods;
  std::vector<int32_t> conn_off, conn_tgt, pix_off, pix_tgt;
  int32_t n_pix_bins;
};

struct Result {
  std::vector<int32_t> order;    // binned position -> input hit index
  std::vector<int32_t> offsets;  // per sensor, n_sensors + 1
  std::vector<MD> md;
  std::vector<LS> ls;
  std::vector<T3> t3;
  std::vector<T5> t5;
  std::vector<int32_t> pls_bin;
  std::vector<PObj> pt3, pt5;
  std::vector<TC> tc;
  std::vector<uint8_t> t5_kept;   // T5 survives duplicate removal
  std::vector<TCExt> tc_ext;      // per TC row
};

// ---------------------------------------------------------------------------------------------
// hit binning: a stable sort of hits by sensor id (Sec. 4.2, "pre-processing the hits")
// ---------------------------------------------------------------------------------------------
void bin_hits(const Geometry& g, const float* x, const float* y, const float* z,
              const int32_t* sensor, int32_t n, Result& res, std::vector<Hit>& hits) {
  int32_t n_sens = 2 * g.n_mods;
  std::vector<int32_t> idx(n);
  for (int32_t i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int32_t a, int32_t b) { return sensor[a] < sensor[b]; });
  res.order = idx;
  res.offsets.assign(n_sens + 1, 0);
  for (int32_t i = 0; i < n; ++i) res.offsets[sensor[i] + 1] += 1;
  for (int32_t s = 0; s < n_sens; ++s) res.offsets[s + 1] += res.offsets[s];
  hits.resize(n);
  for (int32_t j = 0; j < n; ++j) {
    int32_t i = idx[j];
    Hit h;
    h.x = x[i]; h.y = y[i]; h.z = z[i];
    h.r = std::sqrt(h.x * h.x + h.y * h.y);
    h.phi = std::atan2(h.y, h.x);
    h.orig = i;
    h.sensor = sensor[i];
    h.module = sensor[i] / 2;
    h.endcap = g.mods[h.module].subdet == 1;
    hits[j] = h;
  }
}

double alpha_thr(const Params& P, double r) {
  return std::asin(std::min(r * (P.k / 2.0) / P.pt_thr, P.sin_max));
}

// ---------------------------------------------------------------------------------------------
// Mini-Doublet (Sec. 2.2): a hit pair in the two sensors of one module whose direction is
// consistent with a track of pT >= pT_thr from the luminous region (plus resolution and
// impact-parameter allowances).
// ---------------------------------------------------------------------------------------------
Verdict md_cuts(const Params& P, const ModuleRec& m, const Hit& l, const Hit& u,
                double& dphichange, double& pt_est) {
  Verdict v;
  const double delta = m.spacing;
  const double s2 = std::sqrt(2.0);
  if (m.subdet == 0) {
    // barrel: angle between the radial direction at the lower hit and the hit-pair direction
    dphichange = wrap_pi(std::atan2(u.y - l.y, u.x - l.x) - std::atan2(l.y, l.x));
    double bound = alpha_thr(P, l.r) + P.n_sigma * s2 * P.sigma_rphi / delta + P.d0_max / l.r;
    v.cut(bound, std::fabs(dphichange));
    // z: slope dz/dr between that of a line from z = -z_lum and from z = +z_lum, with the
    // helix stretch factor 1/cos(alpha_thr) allowed
    double a = std::min(l.r * (P.k / 2.0) / P.pt_thr, P.sin_max);
    double gfac = 1.0 / std::sqrt(1.0 - a * a);
    double t1 = (l.z - P.z_lum) / l.r;
    double t2 = (l.z + P.z_lum) / l.r;
    double lo = delta * std::min(t1, gfac * t1) - P.n_sigma * s2 * P.sigma_z;
    double hi = delta * std::max(t2, gfac * t2) + P.n_sigma * s2 * P.sigma_z;
    double dz = u.z - l.z;
    v.cut_ge(lo, dz);
    v.cut(hi, dz);
  } else {
    // endcap: radial step across the sensor gap consistent with a line from the luminous region
    double az = std::fabs(l.z);
    double dr_max = l.r * delta / (az - P.z_lum);
    double dr_min = l.r * delta / (az + P.z_lum);
    double dr = u.r - l.r;
    v.cut_ge(dr_min - P.n_sigma * s2 * P.sigma_r, dr);
    v.cut(dr_max + P.n_sigma * s2 * P.sigma_r, dr);
    double dphi = wrap_pi(u.phi - l.phi);
    double bound = std::asin(std::min((l.r + dr_max) * (P.k / 2.0) / P.pt_thr, P.sin_max)) -
                   alpha_thr(P, l.r) + P.n_sigma * s2 * P.sigma_rphi / l.r;
    v.cut(bound, std::fabs(dphi));
    dphichange = dphi * az / delta;
  }
  pt_est = std::min(P.k * l.r / (2.0 * std::max(std::fabs(std::sin(dphichange)), 1e-9)), P.pt_cap);
  return v;
}

// ---------------------------------------------------------------------------------------------
// Line Segment (Sec. 2.2): two MDs in modules connected by the module map; the anchors must
// point back to the luminous region in r-z and open an azimuth compatible with pT >= pT_thr.
// ---------------------------------------------------------------------------------------------
Verdict ls_cuts(const Params& P, const Hit& a, const Hit& b, double& z0_out, double& dphi_out) {
  Verdict v;
  double r1 = a.r, r2 = b.r, z1 = a.z, z2 = b.z;
  double D = r2 - r1;
  if (D == 0.0) { v.fail(); z0_out = 0; dphi_out = 0; return v; }
  double z0r = (z1 * r2 - z2 * r1) / D;
  double Rthr = P.pt_thr / P.k;
  double s1 = 2.0 * Rthr * std::asin(std::min(r1 / (2.0 * Rthr), 1.0));
  double s2 = 2.0 * Rthr * std::asin(std::min(r2 / (2.0 * Rthr), 1.0));
  double z0s = (s2 != s1) ? (z1 * s2 - z2 * s1) / (s2 - s1) : z0r;
  double sz1 = a.endcap ? 0.0 : P.sigma_z, sz2 = b.endcap ? 0.0 : P.sigma_z;
  double sr1 = a.endcap ? P.sigma_r : 0.0, sr2 = b.endcap ? P.sigma_r : 0.0;
  double var = (r2 / D) * (r2 / D) * sz1 * sz1 + (r1 / D) * (r1 / D) * sz2 * sz2 +
               ((z0r - z2) / D) * ((z0r - z2) / D) * sr1 * sr1 +
               ((z1 - z0r) / D) * ((z1 - z0r) / D) * sr2 * sr2;
  double L = P.z_lum + P.n_sigma * std::sqrt(var);
  double zmin = std::min(z0r, z0s), zmax = std::max(z0r, z0s);
  v.cut(L, zmin);      // [zmin, zmax] intersects [-L, L]
  v.cut_ge(-L, zmax);
  double dphi = wrap_pi(b.phi - a.phi);
  double bound = alpha_thr(P, r2) - alpha_thr(P, r1) +
                 P.n_sigma * P.sigma_rphi * std::sqrt(1.0 / (r1 * r1) + 1.0 / (r2 * r2)) +
                 P.d0_max * (1.0 / r1 + 1.0 / r2);
  v.cut(bound, std::fabs(dphi));
  z0_out = z0r;
  dphi_out = dphi;
  return v;
}

// circle through three points (circumcircle); R = +inf for collinear points
void circumcircle(double ax, double ay, double bx, double by, double cx, double cy, double& xc,
                  double& yc, double& R) {
  double d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by));
  if (d == 0.0) { xc = yc = R = INFINITY; return; }
  double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
  xc = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d;
  yc = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d;
  R = std::sqrt((ax - xc) * (ax - xc) + (ay - yc) * (ay - yc));
}

// arc length from the origin to radius r along a circle of radius R through the origin
double arc_s(double R, double r) {
  if (std::isinf(R)) return r;
  return 2.0 * R * std::asin(std::min(r / (2.0 * R), 1.0));
}

// weighted least-squares line z = a + b s; returns chi2 and the slope b
double line_fit_chi2(int n, const double* s, const double* z, const double* sig, double& b_out) {
  double S = 0, Sx = 0, Sy = 0, Sxx = 0, Sxy = 0;
  for (int i = 0; i < n; ++i) {
    double w = 1.0 / (sig[i] * sig[i]);
    S += w; Sx += w * s[i]; Sy += w * z[i]; Sxx += w * s[i] * s[i]; Sxy += w * s[i] * z[i];
  }
  double den = S * Sxx - Sx * Sx;
  double b = (S * Sxy - Sx * Sy) / den;
  double a = (Sxx * Sy - Sx * Sxy) / den;
  double chi2 = 0;
  for (int i = 0; i < n; ++i) {
    double res = (z[i] - a - b * s[i]) / sig[i];
    chi2 += res * res;
  }
  b_out = b;
  return chi2;
}

// r-z straight-line fit in arc length s for anchors on a circle of radius R (Sec. 2.3):
// barrel anchors carry sigma_z, endcap anchors sigma_r * |b0| with b0 the first-to-last slope.
// Returns false when the arc length does not grow from the first to the last anchor.
bool rz_chi2(const Params& P, int n, const Hit* const* h, double R, double& chi2, double& slope) {
  double s[8], z[8], sig[8];
  for (int i = 0; i < n; ++i) { s[i] = arc_s(R, h[i]->r); z[i] = h[i]->z; }
  if (!(s[n - 1] > s[0])) return false;
  double b0 = (z[n - 1] - z[0]) / (s[n - 1] - s[0]);
  for (int i = 0; i < n; ++i)
    sig[i] = std::max(h[i]->endcap ? P.sigma_r * std::fabs(b0) : P.sigma_z, P.sigma_floor);
  chi2 = line_fit_chi2(n, s, z, sig, slope);
  return true;
}

// ---------------------------------------------------------------------------------------------
// Triplet (Sec. 2.3): two LS sharing an MD; circle through the three anchors for a pT estimate
// and an impact-parameter check; straight-line chi2 in r-z.
// ---------------------------------------------------------------------------------------------
Verdict t3_cuts(const Params& P, const Hit& h1, const Hit& h2, const Hit& h3, T3& t) {
  Verdict v;
  double xc, yc, R;
  circumcircle(h1.x, h1.y, h2.x, h2.y, h3.x, h3.y, xc, yc, R);
  double d0;
  if (std::isinf(R)) {  // straight line: distance of the origin from the line through h1, h3
    double dx = h3.x - h1.x, dy = h3.y - h1.y;
    d0 = std::fabs(h1.x * dy - h1.y * dx) / std::sqrt(dx * dx + dy * dy);
  } else {
    d0 = std::fabs(std::sqrt(xc * xc + yc * yc) - R);
  }
  double pt_est = std::min(P.k * R, P.pt_cap);
  v.cut_ge(P.f_t3 * P.pt_thr, P.k * R);
  v.cut(P.d0_t3, d0);
  const Hit* hh[3] = {&h1, &h2, &h3};
  double chi2 = 0, slope = 0;
  if (!rz_chi2(P, 3, hh, R, chi2, slope)) { v.fail(); chi2 = INFINITY; }
  else v.cut(P.chi2_t3, chi2);
  t.R = R; t.xc = xc; t.yc = yc; t.chi2_rz = chi2; t.pt_est = pt_est;
  return v;
}

// ---------------------------------------------------------------------------------------------
// Karimaki's non-iterative circle fit (V. Karimaki, NIM A305 (1991) 187), equal weights.
// Circle: 1/2 rho (x^2+y^2) - (1 + rho d)(x sin(phi) - y cos(phi)) + 1/2 rho d^2 + d = 0, with
// phi the direction at the point of closest approach d (sin(phi), -cos(phi)) to the origin.
// The sense of phi follows the order of the points (first -> last).
// ---------------------------------------------------------------------------------------------
void karimaki(int n, const double* x, const double* y, double& rho, double& phi, double& d) {
  double mx = 0, my = 0, mxx = 0, mxy = 0, myy = 0, mr2 = 0, mxr = 0, myr = 0, mrr = 0;
  for (int i = 0; i < n; ++i) {
    double r2 = x[i] * x[i] + y[i] * y[i];
    mx += x[i]; my += y[i]; mxx += x[i] * x[i]; mxy += x[i] * y[i]; myy += y[i] * y[i];
    mr2 += r2; mxr += x[i] * r2; myr += y[i] * r2; mrr += r2 * r2;
  }
  mx /= n; my /= n; mxx /= n; mxy /= n; myy /= n; mr2 /= n; mxr /= n; myr /= n; mrr /= n;
  double Cxx = mxx - mx * mx, Cxy = mxy - mx * my, Cyy = myy - my * my;
  double Cxr = mxr - mx * mr2, Cyr = myr - my * mr2, Crr = mrr - mr2 * mr2;
  double q1 = Crr * Cxy - Cxr * Cyr;
  double q2 = Crr * (Cxx - Cyy) - Cxr * Cxr + Cyr * Cyr;
  phi = 0.5 * std::atan2(2.0 * q1, q2);
  if (std::cos(phi) * (x[n - 1] - x[0]) + std::sin(phi) * (y[n - 1] - y[0]) < 0.0) phi += kPi;
  phi = wrap_pi(phi);
  double kap = (std::sin(phi) * Cxr - std::cos(phi) * Cyr) / Crr;
  double del = -kap * mr2 + std::sin(phi) * mx - std::cos(phi) * my;
  double root = std::sqrt(1.0 - 4.0 * del * kap);
  rho = 2.0 * kap / root;
  d = 2.0 * del / (1.0 + root);
}

// geometric residual |p - c| - R of a point from the circle (rho, phi, d); the line p.n - d
// when rho == 0
double circle_residual(double rho, double phi, double d, double x, double y) {
  double nx = std::sin(phi), ny = -std::cos(phi);
  if (rho == 0.0) return x * nx + y * ny - d;
  double cxr = (1.0 / rho + d) * nx, cyr = (1.0 / rho + d) * ny;
  return std::sqrt((x - cxr) * (x - cxr) + (y - cyr) * (y - cyr)) - 1.0 / std::fabs(rho);
}

// ---------------------------------------------------------------------------------------------
// Quintuplet (Sec. 2.3): two T3 sharing an MD; their circle radii must be close; a global circle
// fit of the five anchors (Karimaki) and an r-z line fit, each with a chi2 cut.
// ---------------------------------------------------------------------------------------------
Verdict t5_cuts(const Params& P, const Hit* const* h, double R_in, double R_out, T5& t) {
  Verdict v;
  double kin = std::isinf(R_in) ? 0.0 : 1.0 / R_in;
  double kout = std::isinf(R_out) ? 0.0 : 1.0 / R_out;
  v.cut(P.c_rel * std::max(kin, kout) + P.c_abs, std::fabs(kin - kout));
  double x[5], y[5];
  for (int i = 0; i < 5; ++i) { x[i] = h[i]->x; y[i] = h[i]->y; }
  double rho, phi, d;
  karimaki(5, x, y, rho, phi, d);
  double chi2c = 0;
  for (int i = 0; i < 5; ++i) {
    double res = circle_residual(rho, phi, d, x[i], y[i]) / P.sigma_rphi;
    chi2c += res * res;
  }
  v.cut(P.chi2_t5_c, chi2c);
  double R = (rho == 0.0) ? INFINITY : 1.0 / std::fabs(rho);
  double chi2rz = 0, slope = 0;
  if (!rz_chi2(P, 5, h, R, chi2rz, slope)) { v.fail(); chi2rz = INFINITY; }
  else v.cut(P.chi2_t5_rz, chi2rz);
  t.kappa_in = kin; t.kappa_out = kout; t.kappa_fit = rho; t.chi2_c = chi2c; t.chi2_rz = chi2rz;
  t.eta = std::asinh(slope);
  t.phi = phi;
  t.pt = (rho == 0.0) ? P.pt_cap : std::min(P.k / std::fabs(rho), P.pt_cap);
  return v;
}

// ---------------------------------------------------------------------------------------------
// pixel seeds and pT3 / pT5 (Sec. 2.4): the seed's helix is not refitted; the outer anchors are
// tested against the circle and the r-z line that the seed's (pT, eta, phi, x0, y0, z0) define.
// ---------------------------------------------------------------------------------------------
int32_t pixel_bin(const PlsRec& s) {
  double ie = std::floor((double)s.eta * 20.0 + 50.0);
  if (!(ie >= 0.0 && ie < (double)kPixNEta)) return -1;
  double ph = (double)s.phi;
  if (ph < 0.0) ph = ph + kTwoPi;
  double ip = std::floor(ph * (64.0 / kPi));
  if (ip < 0.0) ip = 0.0;
  if (ip > kPixNPhi - 1) ip = kPixNPhi - 1;
  return ((int32_t)ie * kPixNPhi + (int32_t)ip) * 2 + (s.charge > 0 ? 1 : 0);
}

// The terms one outer anchor contributes: its distance from the seed's circle and the variance of
// that distance (hit resolution plus the seed's direction and curvature uncertainties carried out to
// the anchor's radius), and its z offset from the seed's r-z line with that offset's variance.
struct SeedTerms { double dist, var_xy, dz, var_rz; };

SeedTerms seed_terms(const Params& P, const PlsRec& s, const Hit& a) {
  double R = (double)s.pt / P.k;
  double q = s.charge > 0 ? 1.0 : -1.0;
  double phi = s.phi;
  double cx = (double)s.x0 + q * R * std::sin(phi);
  double cy = (double)s.y0 - q * R * std::cos(phi);
  double cot = std::sinh((double)s.eta);
  SeedTerms t;
  t.dist = std::sqrt((a.x - cx) * (a.x - cx) + (a.y - cy) * (a.y - cy)) - R;
  t.var_xy = P.sigma_rphi * P.sigma_rphi + (a.r * P.pls_dir_err) * (a.r * P.pls_dir_err) +
             (P.pls_pt_err * a.r * a.r / (2.0 * R)) * (P.pls_pt_err * a.r * a.r / (2.0 * R));
  double sa = arc_s(R, a.r);
  double zpred = (double)s.z0 + sa * cot;
  double sz = a.endcap ? P.sigma_r * std::fabs(cot) : P.sigma_z;
  double th = sa * (1.0 + cot * cot) * P.pls_dir_err;
  t.dz = a.z - zpred;
  t.var_rz = sz * sz + th * th;
  return t;
}

Verdict pobj_cuts(const Params& P, const PlsRec& s, int n, const Hit* const* h, double cut_xy,
                  double cut_rz, PObj& o) {
  Verdict v;
  double chi2xy = 0, chi2rz = 0;
  for (int i = 0; i < n; ++i) {
    SeedTerms t = seed_terms(P, s, *h[i]);
    chi2xy += t.dist * t.dist / t.var_xy;
    chi2rz += t.dz * t.dz / t.var_rz;
  }
  v.cut(cut_xy, chi2xy);
  v.cut(cut_rz, chi2rz);
  o.chi2_xy = chi2xy; o.chi2_rz = chi2rz; o.score = chi2xy + chi2rz;
  return v;
}

// ---------------------------------------------------------------------------------------------
// Track extension (Sec. 2.5.1): a track candidate's MDs plus the MDs a T3 adds beyond its outer
// end must be one track. Reading: the T3's circle agrees in curvature with the candidate's (as the
// two T3 of a T5 must), and the extended track's n anchors lie on one r-z line in arc length (the
// Quintuplet's r-z fit) with chi2_rz <= chi2_T5,rz (n - 2) / 3, the T5 cut per degree of freedom
// (equal to it at n = 5). Karimaki's circle fit of the n anchors is evaluated for the ranking of
// candidates and as an output, not cut on: with the r-phi resolution alone as its error it
// rejects about half of the true continuations into the endcap (whose radial hit error it does not
// carry), at unchanged purity.
// ---------------------------------------------------------------------------------------------
Verdict ext_cuts(const Params& P, int n, const Hit* const* h, double kappa_t3, double kappa_tc,
                 double& chi2c, double& chi2rz) {
  Verdict v;
  v.cut(P.c_rel * std::max(kappa_t3, kappa_tc) + P.c_abs, std::fabs(kappa_t3 - kappa_tc));
  double x[8], y[8];
  for (int i = 0; i < n; ++i) { x[i] = h[i]->x; y[i] = h[i]->y; }
  double rho, phi, d;
  karimaki(n, x, y, rho, phi, d);
  chi2c = 0;
  for (int i = 0; i < n; ++i) {
    double res = circle_residual(rho, phi, d, x[i], y[i]) / P.sigma_rphi;
    chi2c += res * res;
  }
  double R = (rho == 0.0) ? INFINITY : 1.0 / std::fabs(rho);
  double slope = 0;
  if (!rz_chi2(P, n, h, R, chi2rz, slope)) { v.fail(); chi2rz = INFINITY; }
  else v.cut(P.chi2_t5_rz * (n - 2) / 3.0, chi2rz);
  return v;
}

// ---------------------------------------------------------------------------------------------
// canonical keys: the sorted hit-index tuple of an object (input hit indices; pixel hits use the
// seed's ids). Ties in every "best" choice are broken by these keys, never by storage order.
// ---------------------------------------------------------------------------------------------
bool key_less(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
  return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end());
}

bool dr_close(const Params& P, double eta_a, double phi_a, double eta_b, double phi_b) {
  // eta and phi are the float32 values both sides store; the difference is taken in double
  double de = eta_a - eta_b;
  double dp = phi_a - phi_b;
  if (dp > kPi) dp = dp - kTwoPi;
  if (dp <= -kPi) dp = dp + kTwoPi;
  double d2 = de * de + dp * dp;
  return d2 < P.dr_min * P.dr_min;
}

struct Runner {
  const Params& P;
  const Geometry& g;
  Result& R;
  std::vector<Hit> hits;
  const PlsRec* pls;
  int32_t n_pls;
  bool brute;

  Runner(const Params& p, const Geometry& gg, Result& r) : P(p), g(gg), R(r) {}

  const Hit& anchor(int32_t md) const { return hits[R.md[md].lo]; }

  bool connected(int32_t A, int32_t B) const {
    for (int32_t k = g.conn_off[A]; k < g.conn_off[A + 1]; ++k)
      if (g.conn_tgt[k] == B) return true;
    return false;
  }

  void add_md(int32_t m, int32_t il, int32_t iu) {
    double dpc, pte;
    Verdict v = md_cuts(P, g.mods[m], hits[il], hits[iu], dpc, pte);
    if (!v.keep()) return;
    MD o{il, iu, m, v.all_pass, v.definite(), dpc, pte};
    R.md.push_back(o);
  }

  void run_md() {
    if (!brute) {
      for (int32_t m = 0; m < g.n_mods; ++m)
        for (int32_t il = R.offsets[2 * m]; il < R.offsets[2 * m + 1]; ++il)
          for (int32_t iu = R.offsets[2 * m + 1]; iu < R.offsets[2 * m + 2]; ++iu) add_md(m, il, iu);
    } else {  // every ordered pair of hits, tested for "same module, lower then upper sensor"
      int32_t n = (int32_t)hits.size();
      for (int32_t il = 0; il < n; ++il)
        for (int32_t iu = 0; iu < n; ++iu) {
          int32_t sl = hits[il].sensor, su = hits[iu].sensor;
          if (sl / 2 == su / 2 && (sl & 1) == 0 && (su & 1) == 1)
            add_md(hits[il].module, il, iu);
        }
    }
  }

  void add_ls(int32_t a, int32_t b) {
    double z0, dphi;
    Verdict v = ls_cuts(P, anchor(a), anchor(b), z0, dphi);
    if (!v.keep()) return;
    LS o{a, b, v.all_pass && R.md[a].pass && R.md[b].pass,
         v.definite() && R.md[a].definite && R.md[b].definite, z0, dphi};
    R.ls.push_back(o);
  }

  void run_ls() {
    int32_t nmd = (int32_t)R.md.size();
    if (!brute) {
      // MDs of each module are contiguous in R.md (built module by module)
      std::vector<int32_t> first(g.n_mods + 1, 0);
      for (int32_t i = 0; i < nmd; ++i) first[R.md[i].module + 1]++;
      for (int32_t m = 0; m < g.n_mods; ++m) first[m + 1] += first[m];
      for (int32_t A = 0; A < g.n_mods; ++A)
        for (int32_t a = first[A]; a < first[A + 1]; ++a)
          for (int32_t k = g.conn_off[A]; k < g.conn_off[A + 1]; ++k) {
            int32_t B = g.conn_tgt[k];
            for (int32_t b = first[B]; b < first[B + 1]; ++b) add_ls(a, b);
          }
    } else {
      for (int32_t a = 0; a < nmd; ++a)
        for (int32_t b = 0; b < nmd; ++b)
          if (connected(R.md[a].module, R.md[b].module)) add_ls(a, b);
    }
  }

  void add_t3(int32_t i, int32_t j) {
    const LS& a = R.ls[i];
    const LS& b = R.ls[j];
    T3 t;
    t.ls_in = i; t.ls_out = j;
    t.md[0] = a.md_in; t.md[1] = a.md_out; t.md[2] = b.md_out;
    Verdict v = t3_cuts(P, anchor(t.md[0]), anchor(t.md[1]), anchor(t.md[2]), t);
    if (!v.keep()) return;
    t.pass = v.all_pass && a.pass && b.pass;
    t.definite = v.definite() && a.definite && b.definite;
    R.t3.push_back(t);
  }

  void run_t3() {
    int32_t nls = (int32_t)R.ls.size();
    if (!brute) {
      std::vector<std::vector<int32_t>> by_in(R.md.size());
      for (int32_t j = 0; j < nls; ++j) by_in[R.ls[j].md_in].push_back(j);
      for (int32_t i = 0; i < nls; ++i)
        for (int32_t j : by_in[R.ls[i].md_out]) add_t3(i, j);
    } else {
      for (int32_t i = 0; i < nls; ++i)
        for (int32_t j = 0; j < nls; ++j)
          if (R.ls[i].md_out == R.ls[j].md_in) add_t3(i, j);
    }
  }

  void add_t5(int32_t i, int32_t j) {
    const T3& a = R.t3[i];
    const T3& b = R.t3[j];
    T5 t;
    t.t3_in = i; t.t3_out = j;
    t.md[0] = a.md[0]; t.md[1] = a.md[1]; t.md[2] = a.md[2]; t.md[3] = b.md[1]; t.md[4] = b.md[2];
    const Hit* h[5];
    for (int k = 0; k < 5; ++k) h[k] = &anchor(t.md[k]);
    Verdict v = t5_cuts(P, h, a.R, b.R, t);
    if (!v.keep()) return;
    t.pass = v.all_pass && a.pass && b.pass;
    t.definite = v.definite() && a.definite && b.definite;
    R.t5.push_back(t);
  }

  void run_t5() {
    int32_t nt3 = (int32_t)R.t3.size();
    if (!brute) {
      std::vector<std::vector<int32_t>> by_first(R.md.size());
      for (int32_t j = 0; j < nt3; ++j) by_first[R.t3[j].md[0]].push_back(j);
      for (int32_t i = 0; i < nt3; ++i)
        for (int32_t j : by_first[R.t3[i].md[2]]) add_t5(i, j);
    } else {
      for (int32_t i = 0; i < nt3; ++i)
        for (int32_t j = 0; j < nt3; ++j)
          if (R.t3[i].md[2] == R.t3[j].md[0]) add_t5(i, j);
    }
  }

  bool in_pixmap(int32_t bin, int32_t module) const {
    for (int32_t k = g.pix_off[bin]; k < g.pix_off[bin + 1]; ++k)
      if (g.pix_tgt[k] == module) return true;
    return false;
  }

  template <class Obj>
  void run_pobj(const std::vector<Obj>& objs, int nmd, double cut_xy, double cut_rz,
                std::vector<PObj>& out) {
    int32_t nobj = (int32_t)objs.size();
    std::vector<std::vector<int32_t>> by_module;
    if (!brute) {
      by_module.resize(g.n_mods);
      for (int32_t j = 0; j < nobj; ++j) by_module[R.md[objs[j].md[0]].module].push_back(j);
    }
    for (int32_t p = 0; p < n_pls; ++p) {
      int32_t bin = R.pls_bin[p];
      if (bin < 0) continue;
      auto eval = [&](int32_t j) {
        const Obj& o = objs[j];
        const Hit* h[5];
        for (int k = 0; k < nmd; ++k) h[k] = &anchor(o.md[k]);
        PObj po;
        po.pls = p; po.obj = j;
        Verdict v = pobj_cuts(P, pls[p], nmd, h, cut_xy, cut_rz, po);
        if (!v.keep()) return;
        po.pass = v.all_pass && o.pass;
        po.definite = v.definite() && o.definite;
        out.push_back(po);
      };
      if (!brute) {
        for (int32_t k = g.pix_off[bin]; k < g.pix_off[bin + 1]; ++k)
          for (int32_t j : by_module[g.pix_tgt[k]]) eval(j);
      } else {
        for (int32_t j = 0; j < nobj; ++j)
          if (in_pixmap(bin, R.md[objs[j].md[0]].module)) eval(j);
      }
    }
  }

  // hits of an object in the fixed output order: pixel hits, then (lower, upper) per MD inner->outer
  void md_hits(const int32_t* md, int n, std::vector<int32_t>& out) const {
    for (int k = 0; k < n; ++k) {
      out.push_back(hits[R.md[md[k]].lo].orig);
      out.push_back(hits[R.md[md[k]].up].orig);
    }
  }
  std::vector<int32_t> sorted_key(std::vector<int32_t> v) const {
    std::sort(v.begin(), v.end());
    return v;
  }

  void run_tc() {
    const int32_t nt5 = (int32_t)R.t5.size();
    // 1. per pixel seed, the best passing pT5 and pT3: lowest (score as float32, key)
    auto best_per_pls = [&](const std::vector<PObj>& objs, bool is_t5) {
      std::vector<int32_t> best(n_pls, -1);
      std::vector<float> best_score(n_pls, 0.f);
      std::vector<std::vector<int32_t>> best_key(n_pls);
      for (int32_t i = 0; i < (int32_t)objs.size(); ++i) {
        const PObj& o = objs[i];
        if (!o.pass) continue;
        float sc = (float)o.score;
        std::vector<int32_t> h(pls[o.pls].pix_hit, pls[o.pls].pix_hit + 4);
        if (is_t5) md_hits(R.t5[o.obj].md, 5, h);
        else md_hits(R.t3[o.obj].md, 3, h);
        std::vector<int32_t> key = sorted_key(h);
        int32_t p = o.pls;
        if (best[p] < 0 || sc < best_score[p] || (sc == best_score[p] && key_less(key, best_key[p]))) {
          best[p] = i; best_score[p] = sc; best_key[p] = key;
        }
      }
      return best;
    };
    std::vector<int32_t> best5 = best_per_pls(R.pt5, true);
    std::vector<int32_t> best3 = best_per_pls(R.pt3, false);

    // 2. T5 duplicate removal (non-greedy): A is dropped iff some passing B shares >= 7 of its 10
    //    hits and has the lower (chi2_c as float32, key)
    std::vector<std::vector<int32_t>> t5hits(nt5), t5key(nt5);
    for (int32_t i = 0; i < nt5; ++i) {
      md_hits(R.t5[i].md, 5, t5hits[i]);
      t5key[i] = sorted_key(t5hits[i]);
    }
    R.t5_kept.assign(nt5, 0);
    std::vector<std::vector<int32_t>> t5_of_hit;
    if (!brute) {
      t5_of_hit.resize(hits.size() + 1);
      for (int32_t b = 0; b < nt5; ++b)
        if (R.t5[b].pass)
          for (int k = 0; k < 5; ++k) {
            t5_of_hit[R.md[R.t5[b].md[k]].lo].push_back(b);
            t5_of_hit[R.md[R.t5[b].md[k]].up].push_back(b);
          }
    }
    auto shared_hits = [&](int32_t a, int32_t b) {
      int shared = 0;
      for (int32_t x : t5hits[a])
        for (int32_t y : t5hits[b])
          if (x == y) ++shared;
      return shared;
    };
    for (int32_t a = 0; a < nt5; ++a) {
      if (!R.t5[a].pass) continue;
      std::vector<int32_t> others;
      if (brute) {
        for (int32_t b = 0; b < nt5; ++b) others.push_back(b);
      } else {  // only T5 sharing at least one hit can share seven
        for (int k = 0; k < 5; ++k) {
          for (int32_t b : t5_of_hit[R.md[R.t5[a].md[k]].lo]) others.push_back(b);
          for (int32_t b : t5_of_hit[R.md[R.t5[a].md[k]].up]) others.push_back(b);
        }
        std::sort(others.begin(), others.end());
        others.erase(std::unique(others.begin(), others.end()), others.end());
      }
      bool drop = false;
      for (int32_t b : others) {
        if (b == a || !R.t5[b].pass) continue;
        if (shared_hits(a, b) < P.t5_overlap_hits) continue;
        float ca = (float)R.t5[a].chi2_c, cb = (float)R.t5[b].chi2_c;
        if (cb < ca || (cb == ca && key_less(t5key[b], t5key[a]))) { drop = true; break; }
      }
      R.t5_kept[a] = drop ? 0 : 1;
    }

    // 3. assemble in the order pT5, pT3, T5, pLS (Sec. 2.5), with eta-phi cross-cleaning
    struct Cand { int32_t type, obj; std::vector<int32_t> hits, key; float pt, eta, phi; };
    std::vector<Cand> acc_pt5, acc_pt3, acc_t5, acc_pls;
    // accepted (eta, phi) points, searched in an eta window: dR < dr_min implies |deta| < dr_min
    struct EtaPhi { float first, second; };
    auto ep_less = [](const EtaPhi& a, const EtaPhi& b) {
      return a.first < b.first || (a.first == b.first && a.second < b.second);
    };
    std::vector<EtaPhi> near_set;
    auto add_near = [&](float eta, float phi) {
      EtaPhi v{eta, phi};
      near_set.insert(std::upper_bound(near_set.begin(), near_set.end(), v, ep_less), v);
    };
    auto is_near = [&](float eta, float phi) {
      if (brute) {
        for (const auto& e : near_set)
          if (dr_close(P, eta, phi, e.first, e.second)) return true;
        return false;
      }
      auto it = std::lower_bound(near_set.begin(), near_set.end(),
                                 EtaPhi{(float)((double)eta - 2.0 * P.dr_min), -1e30f}, ep_less);
      for (; it != near_set.end() && (double)it->first <= (double)eta + P.dr_min; ++it)
        if (dr_close(P, eta, phi, it->first, it->second)) return true;
      return false;
    };
    std::vector<uint8_t> pls_used5(n_pls, 0);
    for (int32_t p = 0; p < n_pls; ++p) {
      if (best5[p] < 0) continue;
      const PObj& o = R.pt5[best5[p]];
      Cand c{0, best5[p], {}, {}, pls[p].pt, pls[p].eta, pls[p].phi};
      c.hits.assign(pls[p].pix_hit, pls[p].pix_hit + 4);
      md_hits(R.t5[o.obj].md, 5, c.hits);
      c.key = sorted_key(c.hits);
      acc_pt5.push_back(c);
      pls_used5[p] = 1;
    }
    for (const Cand& c : acc_pt5) add_near(c.eta, c.phi);
    for (int32_t p = 0; p < n_pls; ++p) {
      if (best3[p] < 0 || pls_used5[p]) continue;
      if (is_near(pls[p].eta, pls[p].phi)) continue;
      const PObj& o = R.pt3[best3[p]];
      Cand c{1, best3[p], {}, {}, pls[p].pt, pls[p].eta, pls[p].phi};
      c.hits.assign(pls[p].pix_hit, pls[p].pix_hit + 4);
      md_hits(R.t3[o.obj].md, 3, c.hits);
      c.key = sorted_key(c.hits);
      acc_pt3.push_back(c);
    }
    for (const Cand& c : acc_pt3) add_near(c.eta, c.phi);
    for (int32_t i = 0; i < nt5; ++i) {
      if (!R.t5_kept[i]) continue;
      float eta = (float)R.t5[i].eta, phi = (float)R.t5[i].phi;
      if (is_near(eta, phi)) continue;
      Cand c{2, i, t5hits[i], t5key[i], (float)R.t5[i].pt, eta, phi};
      acc_t5.push_back(c);
    }
    for (const Cand& c : acc_t5) add_near(c.eta, c.phi);
    std::vector<uint8_t> pls_member(n_pls, 0);
    for (const PObj& o : R.pt3) if (o.pass) pls_member[o.pls] = 1;
    for (const PObj& o : R.pt5) if (o.pass) pls_member[o.pls] = 1;
    for (int32_t p = 0; p < n_pls; ++p) {
      if (pls_member[p]) continue;
      if (is_near(pls[p].eta, pls[p].phi)) continue;
      Cand c{3, p, {}, {}, pls[p].pt, pls[p].eta, pls[p].phi};
      c.hits.assign(pls[p].pix_hit, pls[p].pix_hit + 4);
      c.key = sorted_key(c.hits);
      acc_pls.push_back(c);
    }
    for (auto* lst : {&acc_pt5, &acc_pt3, &acc_t5, &acc_pls}) {
      std::sort(lst->begin(), lst->end(),
                [&](const Cand& a, const Cand& b) { return key_less(a.key, b.key); });
      for (const Cand& c : *lst) {
        TC t;
        t.type = c.type; t.obj = c.obj;
        for (int k = 0; k < 14; ++k) t.hits[k] = k < (int)c.hits.size() ? c.hits[k] : -1;
        t.pt = c.pt; t.eta = c.eta; t.phi = c.phi;
        R.tc.push_back(t);
      }
    }
  }

  // Track extensions (Sec. 2.5.1): for each pT5, pT3 and T5 track candidate, the T3 that continues
  // it outward best: candidates share the candidate's last MD (adding two MDs) or its last two MDs
  // (adding one); the passing one with the lowest (chi2_c + chi2_rz as float32, sorted hit tuple of
  // the T3) is chosen.
  void run_ext() {
    const int32_t nt3 = (int32_t)R.t3.size();
    std::vector<std::vector<int32_t>> by_first;
    if (!brute) {
      by_first.resize(R.md.size());
      for (int32_t j = 0; j < nt3; ++j) by_first[R.t3[j].md[0]].push_back(j);
    }
    R.tc_ext.assign(R.tc.size(), TCExt{});
    for (size_t i = 0; i < R.tc.size(); ++i) {
      const TC& t = R.tc[i];
      std::vector<int32_t> m;
      double kappa_tc = 0;
      bool tc_definite = true;
      if (t.type == 0) {
        const PObj& o = R.pt5[t.obj];
        m.assign(R.t5[o.obj].md, R.t5[o.obj].md + 5);
        kappa_tc = P.k / (double)pls[o.pls].pt;
        tc_definite = o.definite;
      } else if (t.type == 1) {
        const PObj& o = R.pt3[t.obj];
        m.assign(R.t3[o.obj].md, R.t3[o.obj].md + 3);
        kappa_tc = P.k / (double)pls[o.pls].pt;
        tc_definite = o.definite;
      } else if (t.type == 2) {
        m.assign(R.t5[t.obj].md, R.t5[t.obj].md + 5);
        kappa_tc = std::fabs(R.t5[t.obj].kappa_fit);
        tc_definite = R.t5[t.obj].definite;
      } else {
        continue;   // a pixel line segment has no outer-tracker MD to extend from
      }
      const int K = (int)m.size();
      TCExt best;
      bool have = false, any_border = false;
      float best_score = 0.f;
      std::vector<int32_t> best_key;
      for (int overlap = 1; overlap <= 2; ++overlap) {
        const int32_t first = m[K - overlap];
        std::vector<int32_t> cands;
        if (brute) {
          for (int32_t j = 0; j < nt3; ++j) if (R.t3[j].md[0] == first) cands.push_back(j);
        } else {
          cands = by_first[first];
        }
        for (int32_t j : cands) {
          const T3& c3 = R.t3[j];
          if (overlap == 2 && c3.md[1] != m[K - 1]) continue;
          std::vector<int32_t> all = m;
          for (int k = overlap; k < 3; ++k) all.push_back(c3.md[k]);
          const int n = (int)all.size();
          const Hit* h[8];
          for (int k = 0; k < n; ++k) h[k] = &anchor(all[k]);
          double chi2c, chi2rz;
          Verdict v = ext_cuts(P, n, h, std::isinf(c3.R) ? 0.0 : 1.0 / c3.R, kappa_tc, chi2c, chi2rz);
          if (!v.keep()) continue;
          if (!v.definite() || !c3.definite) any_border = true;
          if (!(v.all_pass && c3.pass)) continue;
          float sc = (float)(chi2c + chi2rz);
          std::vector<int32_t> key;
          md_hits(c3.md, 3, key);
          key = sorted_key(key);
          if (!have || sc < best_score || (sc == best_score && key_less(key, best_key))) {
            have = true;
            best_score = sc;
            best_key = key;
            best = TCExt{};
            best.t3 = j;
            best.n_add = 3 - overlap;
            best.chi2_c = chi2c;
            best.chi2_rz = chi2rz;
            std::vector<int32_t> added;
            md_hits(&c3.md[overlap], 3 - overlap, added);
            for (size_t k = 0; k < added.size(); ++k) best.hits[k] = added[k];
          }
        }
      }
      best.definite = !any_border && tc_definite;
      R.tc_ext[i] = best;
    }
  }

  void run(const float* x, const float* y, const float* z, const int32_t* sensor, int32_t n_hits,
           const PlsRec* pl, int32_t np, bool brute_force) {
    pls = pl; n_pls = np; brute = brute_force;
    bin_hits(g, x, y, z, sensor, n_hits, R, hits);
    run_md();
    run_ls();
    run_t3();
    run_t5();
    R.pls_bin.resize(n_pls);
    for (int32_t p = 0; p < n_pls; ++p) R.pls_bin[p] = g.n_pix_bins > 0 ? pixel_bin(pls[p]) : -1;
    run_pobj(R.t3, 3, P.chi2_pt3_xy, P.chi2_pt3_rz, R.pt3);
    run_pobj(R.t5, 5, P.chi2_pt5_xy, P.chi2_pt5_rz, R.pt5);
    run_tc();
    run_ext();
  }
};

struct Handle {
  Result res;
  std::vector<Hit> hits;
};

}  // namespace

// ---------------------------------------------------------------------------------------------
// C interface (ctypes)
// ---------------------------------------------------------------------------------------------
extern "C" {

// constants in the order of lst_config's float fields (k ... sigma_floor), then the overlap count
int orc_constants(double* out, int n) {
  Params p = default_params();
  double v[] = {p.k, p.pt_thr, p.sin_max, p.z_lum, p.d0_max, p.n_sigma, p.sigma_rphi, p.sigma_z,
                p.sigma_r, p.chi2_t3, p.chi2_t5_c, p.chi2_t5_rz, p.chi2_pt3_xy, p.chi2_pt3_rz,
                p.chi2_pt5_xy, p.chi2_pt5_rz, p.f_t3, p.d0_t3, p.c_rel, p.c_abs, p.dr_min,
                p.pt_cap, p.pls_dir_err, p.pls_pt_err, p.sigma_floor, (double)p.t5_overlap_hits};
  int m = (int)(sizeof(v) / sizeof(v[0]));
  for (int i = 0; i < n && i < m; ++i) out[i] = v[i];
  return m;
}

void* orc_run(double pt_thr, const void* mods, int32_t n_mods, const int32_t* conn_off,
              const int32_t* conn_tgt, const int32_t* pix_off, const int32_t* pix_tgt,
              int32_t n_pix_bins, const float* x, const float* y, const float* z,
              const int32_t* sensor, int32_t n_hits, const void* pls, int32_t n_pls,
              int32_t brute_force) {
  Params P = default_params();
  P.pt_thr = pt_thr;
  Geometry g;
  g.n_mods = n_mods;
  const ModuleRec* mr = static_cast<const ModuleRec*>(mods);
  g.mods.assign(mr, mr + n_mods);
  g.conn_off.assign(conn_off, conn_off + n_mods + 1);
  g.conn_tgt.assign(conn_tgt, conn_tgt + g.conn_off[n_mods]);
  g.n_pix_bins = n_pix_bins;
  if (n_pix_bins > 0) {
    g.pix_off.assign(pix_off, pix_off + n_pix_bins + 1);
    g.pix_tgt.assign(pix_tgt, pix_tgt + g.pix_off[n_pix_bins]);
  }
  Handle* h = new Handle();
  Runner r(P, g, h->res);
  r.run(x, y, z, sensor, n_hits, static_cast<const PlsRec*>(pls), n_pls, brute_force != 0);
  h->hits = r.hits;
  return h;
}

void orc_free(void* h) { delete static_cast<Handle*>(h); }

// tables: 0 binned order, 1 sensor offsets, 2 MD, 3 LS, 4 T3, 5 T5, 6 pLS bins, 7 pT3, 8 pT5,
// 9 TC, 10 T5 kept flags, 11 TC extensions (one per TC row)
int64_t orc_count(void* hp, int32_t table) {
  Result& R = static_cast<Handle*>(hp)->res;
  switch (table) {
    case 0: return (int64_t)R.order.size();
    case 1: return (int64_t)R.offsets.size();
    case 2: return (int64_t)R.md.size();
    case 3: return (int64_t)R.ls.size();
    case 4: return (int64_t)R.t3.size();
    case 5: return (int64_t)R.t5.size();
    case 6: return (int64_t)R.pls_bin.size();
    case 7: return (int64_t)R.pt3.size();
    case 8: return (int64_t)R.pt5.size();
    case 9: return (int64_t)R.tc.size();
    case 10: return (int64_t)R.t5_kept.size();
    case 11: return (int64_t)R.tc_ext.size();
  }
  return -1;
}

// integer columns
//  MD: 0 hit_lo(orig) 1 hit_up(orig) 2 module 3 pass 4 definite
//  LS: 0 md_in 1 md_out 2 pass 3 definite
//  T3: 0 ls_in 1 ls_out 2 pass 3 definite 4..6 md[0..2]
//  T5: 0 t3_in 1 t3_out 2 pass 3 definite 4..8 md[0..4]
//  pT3/pT5: 0 pls 1 obj 2 pass 3 definite
//  TC: 0 type 1 obj 2..15 hits
//  TC extension: 0 t3 (-1: none) 1 MDs added 2 definite 3..6 added hits (-1 padded)
int orc_get_i32(void* hp, int32_t table, int32_t col, int32_t* dst) {
  Handle* h = static_cast<Handle*>(hp);
  Result& R = h->res;
  switch (table) {
    case 0: for (size_t i = 0; i < R.order.size(); ++i) dst[i] = R.order[i]; return 0;
    case 1: for (size_t i = 0; i < R.offsets.size(); ++i) dst[i] = R.offsets[i]; return 0;
    case 2:
      for (size_t i = 0; i < R.md.size(); ++i) {
        const MD& o = R.md[i];
        int32_t v[] = {h->hits[o.lo].orig, h->hits[o.up].orig, o.module, o.pass, o.definite};
        if (col < 0 || col > 4) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 3:
      for (size_t i = 0; i < R.ls.size(); ++i) {
        const LS& o = R.ls[i];
        int32_t v[] = {o.md_in, o.md_out, o.pass, o.definite};
        if (col < 0 || col > 3) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 4:
      for (size_t i = 0; i < R.t3.size(); ++i) {
        const T3& o = R.t3[i];
        int32_t v[] = {o.ls_in, o.ls_out, o.pass, o.definite, o.md[0], o.md[1], o.md[2]};
        if (col < 0 || col > 6) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 5:
      for (size_t i = 0; i < R.t5.size(); ++i) {
        const T5& o = R.t5[i];
        int32_t v[] = {o.t3_in, o.t3_out, o.pass, o.definite, o.md[0], o.md[1], o.md[2], o.md[3], o.md[4]};
        if (col < 0 || col > 8) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 6: for (size_t i = 0; i < R.pls_bin.size(); ++i) dst[i] = R.pls_bin[i]; return 0;
    case 7: case 8: {
      const std::vector<PObj>& v = table == 7 ? R.pt3 : R.pt5;
      for (size_t i = 0; i < v.size(); ++i) {
        int32_t c[] = {v[i].pls, v[i].obj, v[i].pass, v[i].definite};
        if (col < 0 || col > 3) return -1;
        dst[i] = c[col];
      }
      return 0;
    }
    case 9:
      for (size_t i = 0; i < R.tc.size(); ++i) {
        if (col == 0) dst[i] = R.tc[i].type;
        else if (col == 1) dst[i] = R.tc[i].obj;
        else if (col >= 2 && col < 16) dst[i] = R.tc[i].hits[col - 2];
        else return -1;
      }
      return 0;
    case 10: for (size_t i = 0; i < R.t5_kept.size(); ++i) dst[i] = R.t5_kept[i]; return 0;
    case 11:
      for (size_t i = 0; i < R.tc_ext.size(); ++i) {
        const TCExt& o = R.tc_ext[i];
        if (col == 0) dst[i] = o.t3;
        else if (col == 1) dst[i] = o.n_add;
        else if (col == 2) dst[i] = o.definite;
        else if (col >= 3 && col < 7) dst[i] = o.hits[col - 3];
        else return -1;
      }
      return 0;
  }
  return -1;
}

// float columns
//  MD: 0 dphichange 1 pt_est 2 x 3 y 4 z 5 r (anchor = lower hit)
//  LS: 0 z0 1 dphi
//  T3: 0 R 1 xc 2 yc 3 chi2_rz 4 pt_est
//  T5: 0 kappa_in 1 kappa_out 2 kappa_fit 3 chi2_c 4 chi2_rz 5 eta 6 phi 7 pt
//  pT3/pT5: 0 chi2_xy 1 chi2_rz 2 score
//  TC: 0 pt 1 eta 2 phi
//  TC extension: 0 chi2_c 1 chi2_rz
int orc_get_f64(void* hp, int32_t table, int32_t col, double* dst) {
  Handle* h = static_cast<Handle*>(hp);
  Result& R = h->res;
  switch (table) {
    case 2:
      for (size_t i = 0; i < R.md.size(); ++i) {
        const MD& o = R.md[i];
        const Hit& a = h->hits[o.lo];
        double v[] = {o.dphichange, o.pt_est, a.x, a.y, a.z, a.r};
        if (col < 0 || col > 5) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 3:
      for (size_t i = 0; i < R.ls.size(); ++i) {
        double v[] = {R.ls[i].z0, R.ls[i].dphi};
        if (col < 0 || col > 1) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 4:
      for (size_t i = 0; i < R.t3.size(); ++i) {
        const T3& o = R.t3[i];
        double v[] = {o.R, o.xc, o.yc, o.chi2_rz, o.pt_est};
        if (col < 0 || col > 4) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 5:
      for (size_t i = 0; i < R.t5.size(); ++i) {
        const T5& o = R.t5[i];
        double v[] = {o.kappa_in, o.kappa_out, o.kappa_fit, o.chi2_c, o.chi2_rz, o.eta, o.phi, o.pt};
        if (col < 0 || col > 7) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 7: case 8: {
      const std::vector<PObj>& v = table == 7 ? R.pt3 : R.pt5;
      for (size_t i = 0; i < v.size(); ++i) {
        double c[] = {v[i].chi2_xy, v[i].chi2_rz, v[i].score};
        if (col < 0 || col > 2) return -1;
        dst[i] = c[col];
      }
      return 0;
    }
    case 9:
      for (size_t i = 0; i < R.tc.size(); ++i) {
        double v[] = {R.tc[i].pt, R.tc[i].eta, R.tc[i].phi};
        if (col < 0 || col > 2) return -1;
        dst[i] = v[col];
      }
      return 0;
    case 11:
      for (size_t i = 0; i < R.tc_ext.size(); ++i) {
        if (col == 0) dst[i] = R.tc_ext[i].chi2_c;
        else if (col == 1) dst[i] = R.tc_ext[i].chi2_rz;
        else return -1;
      }
      return 0;
  }
  return -1;
}

// Exposed closed forms, so the tests can pin them directly.
void orc_circumcircle(const double* p, double* out) {
  circumcircle(p[0], p[1], p[2], p[3], p[4], p[5], out[0], out[1], out[2]);
}
void orc_karimaki(int n, const double* x, const double* y, double* out) {
  karimaki(n, x, y, out[0], out[1], out[2]);
  double chi2 = 0;
  for (int i = 0; i < n; ++i) {
    double r = circle_residual(out[0], out[1], out[2], x[i], y[i]);
    chi2 += r * r;
  }
  out[3] = chi2;
}
double orc_line_fit(int n, const double* s, const double* z, const double* sig, double* slope) {
  return line_fit_chi2(n, s, z, sig, *slope);
}
// The pT3 / pT5 terms of one seed against n anchors (x, y, z; endcap flag): per anchor
// (distance from the seed circle, its variance, z offset from the seed line, its variance) in
// terms[4 n]; chi2[0] = chi2_xy and chi2[1] = chi2_rz summed as the pT3 / pT5 selection sums them.
void orc_seed_terms(const void* seed, int32_t n, const double* x, const double* y, const double* z,
                    const int32_t* endcap, double* terms, double* chi2) {
  Params P = default_params();
  const PlsRec& s = *static_cast<const PlsRec*>(seed);
  chi2[0] = chi2[1] = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    Hit a;
    a.x = x[i]; a.y = y[i]; a.z = z[i];
    a.r = std::sqrt(a.x * a.x + a.y * a.y);
    a.phi = std::atan2(a.y, a.x);
    a.orig = i; a.sensor = 0; a.module = 0;
    a.endcap = endcap[i] != 0;
    SeedTerms t = seed_terms(P, s, a);
    terms[4 * i + 0] = t.dist;
    terms[4 * i + 1] = t.var_xy;
    terms[4 * i + 2] = t.dz;
    terms[4 * i + 3] = t.var_rz;
    chi2[0] += t.dist * t.dist / t.var_xy;
    chi2[1] += t.dz * t.dz / t.var_rz;
  }
}

int32_t orc_pixel_bin(float eta, float phi, int32_t charge) {
  PlsRec s;
  std::memset(&s, 0, sizeof(s));
  s.eta = eta; s.phi = phi; s.charge = charge;
  return pixel_bin(s);
}

}  // extern "C"
