// Shared device-side definitions of the GB300 Line Segment Tracking library.
//
// Precision design. Object storage and the bulk of the cut arithmetic are float32. Every cut is a
// comparison value <= bound. A float32 evaluation decides a candidate only when its margin is
// clear of the threshold by more than a guard band that bounds the float32 error of that formula
// (relative 2^-12 of max(|bound|, |value|) for the Mini-Doublet and Line-Segment windows, which
// are written in forms whose float32 error is ~1e-6 relative: compensated cross products, exact
// hit-coordinate differences, an asin-difference identity). Candidates inside the band are queued
// and decided again in float64. The chi2 cuts (T3, T5, pT3, pT5), whose residuals are tiny
// differences of coordinates of order 100 cm, use float32 only as a conservative pre-filter; every
// candidate that survives it is decided, and its stored floats computed, in double-float
// arithmetic (pairs of floats, ~48 bits, lst_ff.cuh), which runs on the float32 pipes: on GB300
// float64 issues at a small fraction of the float32 rate. The decisions agree with an exact
// evaluation of the cut definitions except within ~1e-12 relative of a threshold.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lst.h"
#include "lst_ff.cuh"

namespace lst {

constexpr int kPixNEta = 100;
constexpr int kPixNPhi = 128;
constexpr double kPiD = 3.14159265358979323846;
constexpr double kTwoPiD = 6.28318530717958647692;
constexpr float kGuardWindow = 1.0f / 4096.0f;   // MD / LS float32 guard (relative)
constexpr float kGuardChi2 = 1.0f / 16.0f;       // chi2 pre-filter guard (relative)
constexpr float kGuardChi2Abs = 0.25f;           // chi2 pre-filter guard (absolute)

// Cut constants in precision T (derived values computed once on the host in double).
template <class T>
struct Cst {
  T k, pt_thr, sin_max, z_lum, d0_max, n_sigma, sigma_rphi, sigma_z, sigma_r;
  T k2p;         // k / 2 / pt_thr: sin(alpha) = r * k2p at the threshold
  T two_rthr;    // 2 R_thr = 2 pt_thr / k
  T tol_rphi;    // n_sigma * sqrt(2) * sigma_rphi
  T tol_z;       // n_sigma * sqrt(2) * sigma_z
  T tol_r;       // n_sigma * sqrt(2) * sigma_r
  T chi2_t3, chi2_t5_c, chi2_t5_rz, chi2_pt3_xy, chi2_pt3_rz, chi2_pt5_xy, chi2_pt5_rz;
  T f_t3, d0_t3, c_rel, c_abs, dr_min, pt_cap, pls_dir_err, pls_pt_err, sigma_floor;
  int t5_overlap_hits;
};

struct Consts {
  Cst<float> f;
  Cst<double> d;
  Cst<ff> x;   // the float64 values as double-float pairs
};

// ---------------------------------------------------------------------------------------------
// precision-generic math
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_asin(float x) { return asinf(x); }
__device__ __forceinline__ double m_asin(double x) { return asin(x); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double m_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double m_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }

// a*d - b*c. float: Kahan's compensated form (error ~1.5 ulp of the result, no cancellation
// loss); double: plain.
__device__ __forceinline__ float diff_prod(float a, float d, float b, float c) {
  float w = b * c;
  float e = fmaf(-b, c, w);
  float f = fmaf(a, d, -w);
  return f + e;
}
__device__ __forceinline__ double diff_prod(double a, double d, double b, double c) {
  return a * d - b * c;
}

// asin(a) - asin(b) for 0 <= a, b < 1 given amb = a - b, in a form without cancellation:
// sin(asin a - asin b) = (a - b) [sqrt(1-b^2) + b (a+b) / (sqrt(1-a^2) + sqrt(1-b^2))].
template <class T>
__device__ __forceinline__ T asin_diff(T a, T b, T amb) {
  T ca = m_sqrt((T(1) - a) * (T(1) + a));
  T cb = m_sqrt((T(1) - b) * (T(1) + b));
  return m_asin(amb * (cb + b * (a + b) / (ca + cb)));
}

// ---------------------------------------------------------------------------------------------
// cut accumulators
// ---------------------------------------------------------------------------------------------
enum Verdict : int { kReject = 0, kAccept = 1, kUnsure = 2 };

// float32 evaluation: decides only outside the guard band
struct Acc32 {
  bool fail = false, unsure = false;
  float g;
  __device__ explicit Acc32(float guard) : g(guard) {}
  __device__ __forceinline__ void cut(float bound, float value) {  // pass iff value <= bound
    float m = bound - value;
    float tol = g * fmaxf(fabsf(bound), fabsf(value)) + 1e-30f;
    if (!(m == m)) unsure = true;
    else if (m < -tol) fail = true;
    else if (m <= tol) unsure = true;
  }
  __device__ __forceinline__ void cut_ge(float bound, float value) { cut(-bound, -value); }
  __device__ __forceinline__ void force_unsure() { unsure = true; }
  __device__ __forceinline__ void reject() { fail = true; }
  __device__ __forceinline__ int verdict() const { return fail ? kReject : (unsure ? kUnsure : kAccept); }
};

// float64 evaluation: the decision (NaN fails)
struct Acc64 {
  bool fail = false;
  __device__ explicit Acc64(double = 0) {}
  __device__ __forceinline__ void cut(double bound, double value) {
    if (!(bound - value >= 0.0)) fail = true;
  }
  __device__ __forceinline__ void cut_ge(double bound, double value) { cut(-bound, -value); }
  __device__ __forceinline__ void force_unsure() {}
  __device__ __forceinline__ void reject() { fail = true; }
  __device__ __forceinline__ int verdict() const { return fail ? kReject : kAccept; }
};

// double-float evaluation: the decision, as in float64 (NaN fails)
struct AccFF {
  bool fail = false;
  __device__ explicit AccFF(ff = ff(0.0f)) {}
  __device__ __forceinline__ void cut(ff bound, ff value) {
    if (!(value <= bound)) fail = true;
  }
  __device__ __forceinline__ void cut_ge(ff bound, ff value) { cut(-bound, -value); }
  __device__ __forceinline__ void force_unsure() {}
  __device__ __forceinline__ void reject() { fail = true; }
  __device__ __forceinline__ int verdict() const { return fail ? kReject : kAccept; }
};

template <class T> struct AccOf;
template <> struct AccOf<float> { using type = Acc32; };
template <> struct AccOf<double> { using type = Acc64; };
template <> struct AccOf<ff> { using type = AccFF; };

// ---------------------------------------------------------------------------------------------
// Mini-Doublet selection (Sec. 2.2). Lower hit l, upper hit u of one module with sensor spacing
// delta.
//   barrel: dPhiChange = angle between the radial direction at l and the direction l -> u;
//           |dPhiChange| <= alpha_thr(r_l) + n_sigma sqrt2 sigma_rphi / delta + d0_max / r_l,
//           alpha_thr(r) = asin(min(r k / (2 pT_thr), sin_max));
//           z_u - z_l within delta * [min(t1, g t1), max(t2, g t2)] -+ n_sigma sqrt2 sigma_z with
//           t1,2 = (z_l -+ z_lum) / r_l and g = 1 / cos(alpha_thr(r_l)).
//   endcap: r_u - r_l within [dr_min, dr_max] -+ n_sigma sqrt2 sigma_r with
//           dr_max,min = r_l delta / (|z_l| -+ z_lum);
//           |phi_u - phi_l| <= alpha(r_l + dr_max) - alpha_thr(r_l) + n_sigma sqrt2 sigma_rphi / r_l;
//           dPhiChange = (phi_u - phi_l) |z_l| / delta.
//   pt_est = k r_l / (2 max(|sin dPhiChange|, 1e-9)), capped.
// ---------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int md_eval(const Cst<T>& c, bool endcap, T delta, T xl, T yl, T zl,
                                       T xu, T yu, T zu, T guard, T& dphic, T& pt_est) {
  typename AccOf<T>::type acc(guard);
  const T rl = m_sqrt(xl * xl + yl * yl);
  if (!endcap) {
    const T dx = xu - xl, dy = yu - yl;
    // angle from (xl, yl) to (dx, dy)
    const T cr = diff_prod(xl, dy, yl, dx);
    const T dt = diff_prod(xl, dx, -yl, dy);
    dphic = m_atan2(cr, dt);
    const T a = m_min(rl * c.k2p, c.sin_max);
    const T bound = m_asin(a) + c.tol_rphi / delta + c.d0_max / rl;
    acc.cut(bound, m_abs(dphic));
    const T g = T(1) / m_sqrt((T(1) - a) * (T(1) + a));
    const T t1 = (zl - c.z_lum) / rl;
    const T t2 = (zl + c.z_lum) / rl;
    const T lo = delta * m_min(t1, g * t1) - c.tol_z;
    const T hi = delta * m_max(t2, g * t2) + c.tol_z;
    const T dz = zu - zl;
    acc.cut_ge(lo, dz);
    acc.cut(hi, dz);
  } else {
    const T ru = m_sqrt(xu * xu + yu * yu);
    const T dx = xu - xl, dy = yu - yl;
    const T dr = (dx * (xu + xl) + dy * (yu + yl)) / (ru + rl);
    const T az = m_abs(zl);
    const T dr_max = rl * delta / (az - c.z_lum);
    const T dr_min = rl * delta / (az + c.z_lum);
    acc.cut_ge(dr_min - c.tol_r, dr);
    acc.cut(dr_max + c.tol_r, dr);
    const T cr = diff_prod(xl, yu, yl, xu);
    const T dt = diff_prod(xl, xu, -yl, yu);
    const T dphi = m_atan2(cr, dt);
    const T a_raw = (rl + dr_max) * c.k2p;
    const T b_raw = rl * c.k2p;
    T adiff;
    if (a_raw < c.sin_max && b_raw < c.sin_max) {
      adiff = asin_diff(a_raw, b_raw, dr_max * c.k2p);
    } else {  // a capped window: the identity's input a - b loses its accuracy in float32
      const T a = m_min(a_raw, c.sin_max), b = m_min(b_raw, c.sin_max);
      adiff = m_asin(a) - m_asin(b);
      acc.force_unsure();
    }
    const T bound = adiff + c.tol_rphi / rl;
    acc.cut(bound, m_abs(dphi));
    dphic = dphi * az / delta;
  }
  pt_est = m_min(c.k * rl / (T(2) * m_max(m_abs(m_sin(dphic)), T(1e-9))), c.pt_cap);
  return acc.verdict();
}

// ---------------------------------------------------------------------------------------------
// Line Segment selection (Sec. 2.2). Anchors (x1,y1,z1) of the inner MD and (x2,y2,z2) of the
// outer MD (anchor = lower-sensor hit).
//   r-z pointing: z0 of the straight line through the anchors, z0_r = (z1 r2 - z2 r1)/(r2 - r1),
//   and of the helix at the threshold radius (r replaced by the arc length s at R_thr); the
//   interval [min, max] must meet [-L, L], L = z_lum + n_sigma sigma_z0 (sigma_z0 propagated from
//   sigma_z of barrel anchors and sigma_r of endcap anchors).
//   r-phi: |phi2 - phi1| <= alpha_thr(r2) - alpha_thr(r1)
//                            + n_sigma sigma_rphi sqrt(1/r1^2 + 1/r2^2) + d0_max (1/r1 + 1/r2).
// ---------------------------------------------------------------------------------------------
// r_i = sqrt(x_i^2 + y_i^2) and s_i = 2 R_thr asin(min(r_i / (2 R_thr), 1)) are passed in (they are
// per-MD quantities).
template <class T>
__device__ __forceinline__ int ls_eval(const Cst<T>& c, T x1, T y1, T z1, T r1, T s1, bool ec1, T x2,
                                       T y2, T z2, T r2, T s2, bool ec2, T guard, T& z0_out,
                                       T& dphi_out) {
  typename AccOf<T>::type acc(guard);
  const T D = r2 - r1;
  z0_out = T(0);
  dphi_out = T(0);
  if (D == T(0)) { acc.reject(); return acc.verdict(); }
  if (m_abs(D) < T(1)) acc.force_unsure();  // float32 z0 loses accuracy when r1 ~ r2
  const T iD = T(1) / D;
  const T z0r = diff_prod(z1, r2, z2, r1) * iD;
  const T z0s = (s2 != s1) ? diff_prod(z1, s2, z2, s1) / (s2 - s1) : z0r;
  const T sz1 = ec1 ? T(0) : c.sigma_z, sz2 = ec2 ? T(0) : c.sigma_z;
  const T sr1 = ec1 ? c.sigma_r : T(0), sr2 = ec2 ? c.sigma_r : T(0);
  const T q1 = r2 * iD * sz1, q2 = r1 * iD * sz2, q3 = (z0r - z2) * iD * sr1, q4 = (z1 - z0r) * iD * sr2;
  const T L = c.z_lum + c.n_sigma * m_sqrt(q1 * q1 + q2 * q2 + q3 * q3 + q4 * q4);
  acc.cut(L, m_min(z0r, z0s));
  acc.cut_ge(-L, m_max(z0r, z0s));
  const T cr = diff_prod(x1, y2, y1, x2);
  const T dt = diff_prod(x1, x2, -y1, y2);
  const T dphi = m_atan2(cr, dt);
  const T a2 = r2 * c.k2p, a1 = r1 * c.k2p;
  T adiff;
  if (a2 < c.sin_max && a1 < c.sin_max) {
    adiff = asin_diff(a2, a1, D * c.k2p);
  } else {
    adiff = m_asin(m_min(a2, c.sin_max)) - m_asin(m_min(a1, c.sin_max));
    acc.force_unsure();
  }
  const T ir1 = T(1) / r1, ir2 = T(1) / r2;
  const T bound = adiff + c.n_sigma * c.sigma_rphi * m_sqrt(ir1 * ir1 + ir2 * ir2) + c.d0_max * (ir1 + ir2);
  acc.cut(bound, m_abs(dphi));
  z0_out = z0r;
  dphi_out = dphi;
  return acc.verdict();
}

// ---------------------------------------------------------------------------------------------
// Circle through three points, in a form that stays accurate for nearly straight tracks.
// u = p2 - p1, v = p3 - p1; signed curvature kappa = 2 (u x v) / (|u| |v| |v - u|); the centre
// is p1 + w with w = (|u|^2 v_perp - |v|^2 u_perp) / (2 u x v), v_perp = (v_y, -v_x).
// The distance of the origin from the circle, |hypot(centre) - R|, is evaluated as
// |2A / (1 + sqrt(1 + 2|kappa| A))| with A = |kappa|/2 |p1|^2 + p1 . n (n = unit vector from p1
// to the centre), which equals it exactly and needs no large cancellation.
// ---------------------------------------------------------------------------------------------
template <class T>
struct Circle3 {
  T kappa;   // signed
  T R;       // 1 / |kappa| (inf for collinear points)
  T xc, yc;  // centre (inf for collinear points)
  T d0;      // distance of the origin from the circle
};

template <class T>
__device__ __forceinline__ Circle3<T> circle3(T x1, T y1, T x2, T y2, T x3, T y3) {
  Circle3<T> o;
  const T ux = x2 - x1, uy = y2 - y1, vx = x3 - x1, vy = y3 - y1;
  const T cr = diff_prod(ux, vy, uy, vx);
  const T uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
  const T wx3 = x3 - x2, wy3 = y3 - y2;
  const T ww = wx3 * wx3 + wy3 * wy3;
  const T rs = m_sqrt(uu * vv * ww);   // 2 R |cr|
  o.kappa = T(2) * cr / rs;
  // direction of the centre from p1 (valid also when cr -> 0)
  const T Nx = uu * vy - vv * uy;
  const T Ny = -uu * vx + vv * ux;
  const T inv_nn = T(1) / m_sqrt(Nx * Nx + Ny * Ny);
  const T sgn = cr >= T(0) ? T(1) : T(-1);
  const T nx = sgn * Nx * inv_nn, ny = sgn * Ny * inv_nn;
  const T ak = m_abs(o.kappa);
  if (cr == T(0)) {
    o.R = T(1) / T(0);
    o.xc = o.yc = T(1) / T(0);
    // straight line through p1 and p3: distance of the origin
    o.d0 = m_abs(diff_prod(x1, vy, y1, vx)) / m_sqrt(vv);
    return o;
  }
  const T inv_2cr = T(1) / (T(2) * cr);
  o.R = m_abs(rs * inv_2cr);
  o.xc = x1 + Nx * inv_2cr;
  o.yc = y1 + Ny * inv_2cr;
  const T A = T(0.5) * ak * (x1 * x1 + y1 * y1) + (x1 * nx + y1 * ny);
  o.d0 = m_abs(T(2) * A / (T(1) + m_sqrt(T(1) + T(2) * ak * A)));
  return o;
}

// arc length from the origin to radius r on a circle of curvature |kappa| through the origin
template <class T>
__device__ __forceinline__ T arc_len(T akappa, T two_r, T r) {   // two_r = 2 / akappa
  const T x = r * akappa * T(0.5);
  if (x <= T(0)) return r;
  if (x >= T(1)) return two_r * T(1.5707963267948966);  // = pi R (the cap of asin at 1)
  return m_asin(x) * two_r;
}
template <class T>
__device__ __forceinline__ T arc_len(T akappa, T r) {
  return arc_len(akappa, T(2) / akappa, r);
}

// The fits below take the first n of their points (n <= NMAX, a runtime count): their loops run to
// the compile-time bound NMAX and skip the points past n, so one copy of the code serves every
// count, with the same operations in the same order as for a fixed count. The fixed-count forms
// (template <T, N>) are the same functions with n = N.

// Weighted straight-line fit z = a + b s; returns chi2 and the slope b (centred sums).
template <class T, int NMAX>
__device__ __forceinline__ T line_chi2_n(const T* s, const T* z, const T* sig, int n, T& slope) {
  T S = 0, Ss = 0, Sz = 0;
  T w[NMAX], isig[NMAX];
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < n) {
      isig[i] = T(1) / sig[i];
      w[i] = isig[i] * isig[i];
      S += w[i]; Ss += w[i] * s[i]; Sz += w[i] * z[i];
    }
  }
  const T iS = T(1) / S;
  const T sm = Ss * iS, zm = Sz * iS;
  T Sss = 0, Ssz = 0;
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < n) {
      const T ds = s[i] - sm;
      Sss += w[i] * ds * ds;
      Ssz += w[i] * ds * (z[i] - zm);
    }
  }
  const T b = Ssz / Sss;
  T chi2 = 0;
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < n) {
      const T r = (z[i] - zm - b * (s[i] - sm)) * isig[i];
      chi2 += r * r;
    }
  }
  slope = b;
  return chi2;
}
template <class T, int N>
__device__ __forceinline__ T line_chi2(const T* s, const T* z, const T* sig, T& slope) {
  return line_chi2_n<T, N>(s, z, sig, N, slope);
}

// r-z chi2 in arc length for n anchors on a circle of curvature |kappa| (Sec. 2.3): barrel anchors
// carry sigma_z, endcap anchors sigma_r |b0| (b0 = first-to-last slope), floored. Returns false
// when the arc length does not grow from the first to the last anchor.
template <class T, int NMAX>
__device__ __forceinline__ bool rz_fit_n(const Cst<T>& c, T akappa, const T* r, const T* z, const bool* ec,
                                         int n, T& chi2, T& slope) {
  T s[NMAX], sig[NMAX];
  const T two_r = T(2) / akappa;
  T s_last = T(0), z_last = T(0);   // of the n-th anchor (carried along: no run-time array index)
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
    if (i < n) {
      s[i] = arc_len(akappa, two_r, r[i]);
      s_last = s[i];
      z_last = z[i];
    }
  if (!(s_last > s[0])) return false;
  const T b0 = (z_last - z[0]) / (s_last - s[0]);
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
    if (i < n) sig[i] = m_max(ec[i] ? c.sigma_r * m_abs(b0) : c.sigma_z, c.sigma_floor);
  chi2 = line_chi2_n<T, NMAX>(s, z, sig, n, slope);
  return true;
}
template <class T, int N>
__device__ __forceinline__ bool rz_fit(const Cst<T>& c, T akappa, const T* r, const T* z,
                                       const bool* ec, T& chi2, T& slope) {
  return rz_fit_n<T, N>(c, akappa, r, z, ec, N, chi2, slope);
}

// ---------------------------------------------------------------------------------------------
// Karimaki's circle fit (V. Karimaki, NIM A305 (1991) 187) with equal weights.
// Circle: 1/2 rho (x^2 + y^2) - (1 + rho d)(x sin phi - y cos phi) + 1/2 rho d^2 + d = 0;
// phi is the direction at the point of closest approach to the origin, oriented first -> last.
// ---------------------------------------------------------------------------------------------
template <class T, int NMAX>
__device__ __forceinline__ void karimaki_n(const T* x, const T* y, int n, T& rho, T& phi, T& d, T& sp, T& cp) {
  T mx = 0, my = 0, mxx = 0, mxy = 0, myy = 0, mr2 = 0, mxr = 0, myr = 0, mrr = 0;
  T x_last = x[0], y_last = y[0];   // of the n-th point (carried along: no run-time array index)
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < n) {
      x_last = x[i];
      y_last = y[i];
      const T r2 = x[i] * x[i] + y[i] * y[i];
      mx += x[i]; my += y[i];
      mxx += x[i] * x[i]; mxy += x[i] * y[i]; myy += y[i] * y[i];
      mr2 += r2; mxr += x[i] * r2; myr += y[i] * r2; mrr += r2 * r2;
    }
  }
  const T inv = T(1) / T((float)n);
  mx *= inv; my *= inv; mxx *= inv; mxy *= inv; myy *= inv; mr2 *= inv; mxr *= inv; myr *= inv; mrr *= inv;
  const T Cxx = mxx - mx * mx, Cxy = mxy - mx * my, Cyy = myy - my * my;
  const T Cxr = mxr - mx * mr2, Cyr = myr - my * mr2, Crr = mrr - mr2 * mr2;
  const T q1 = Crr * Cxy - Cxr * Cyr;
  const T q2 = Crr * (Cxx - Cyy) - Cxr * Cxr + Cyr * Cyr;
  const T dx = x_last - x[0], dy = y_last - y[0];
  if constexpr (std::is_same<T, ff>::value) {
    // phi = atan2(2 q1, q2) / 2 in (-pi/2, pi/2], so cos phi >= 0: its sine and cosine from the
    // double angle's, (cos 2phi, sin 2phi) = (q2, 2 q1) / h, by the half-angle formulas, each in
    // the form free of cancellation; the angle itself (an output only) in float32
    const ff s2 = ff(2.0f) * q1;
    const ff h = m_sqrt(s2 * s2 + q2 * q2);
    if (h.hi == 0.0f) {
      sp = ff(0.0f);
      cp = ff(1.0f);
    } else {
      const ff c2 = q2 / h, sn2 = s2 / h;
      if (c2.hi >= 0.0f) {
        cp = m_sqrt((ff(1.0f) + c2) * ff(0.5f));
        sp = sn2 / (ff(2.0f) * cp);
      } else {
        sp = m_sqrt((ff(1.0f) - c2) * ff(0.5f));
        if (signbit(sn2.hi)) sp = -sp;
        cp = sn2 / (ff(2.0f) * sp);
      }
    }
    if (cp * dx + sp * dy < T(0)) {
      sp = -sp;
      cp = -cp;
    }
    phi = ff(atan2f(sp.hi, cp.hi));
  } else {
    phi = T(0.5) * m_atan2(T(2) * q1, q2);
    if constexpr (sizeof(T) == 4) sincosf(phi, &sp, &cp);
    else sincos(phi, &sp, &cp);
    if (cp * dx + sp * dy < T(0)) {
      phi += T(kPiD);
      sp = -sp;
      cp = -cp;
    }
    if (phi > T(kPiD)) phi -= T(kTwoPiD);
    if (phi <= -T(kPiD)) phi += T(kTwoPiD);
  }
  const T kap = (sp * Cxr - cp * Cyr) / Crr;
  const T del = -kap * mr2 + sp * mx - cp * my;
  const T root = m_sqrt(T(1) - T(4) * del * kap);
  rho = T(2) * kap / root;
  d = T(2) * del / (T(1) + root);
}
template <class T, int N>
__device__ __forceinline__ void karimaki(const T* x, const T* y, T& rho, T& phi, T& d, T& sp, T& cp) {
  karimaki_n<T, N>(x, y, N, rho, phi, d, sp, cp);
}

// sum over the anchors of ((|p - c| - R) / sigma)^2 at the circle (rho, phi, d) given by rho,
// (sin phi, cos phi) and d, each residual in
// the exact cancellation-free form 2 eps / (1 + sqrt(1 + 2 rho eps))
template <class T, int NMAX>
__device__ __forceinline__ T circle_chi2_n(const T* x, const T* y, int n, T rho, T sp, T cp, T d, T sigma) {
  T chi2 = 0;
#pragma unroll
  for (int a = 0; a < NMAX; ++a) {
    if (a < n) {
      const T eps = T(0.5) * rho * (x[a] * x[a] + y[a] * y[a]) - (T(1) + rho * d) * (x[a] * sp - y[a] * cp) +
                    T(0.5) * rho * d * d + d;
      const T res = T(2) * eps / (T(1) + m_sqrt(T(1) + T(2) * rho * eps)) / sigma;
      chi2 += res * res;
    }
  }
  return chi2;
}
template <class T, int N>
__device__ __forceinline__ T circle_chi2(const T* x, const T* y, T rho, T sp, T cp, T d, T sigma) {
  return circle_chi2_n<T, N>(x, y, N, rho, sp, cp, d, sigma);
}

__host__ __device__ __forceinline__ int64_t lst_min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Azimuth of (x, y) relative to a module's centre azimuth phic (in [0, 2 pi)), wrapped to
// (-pi, pi]. Hits are binned, and MDs ordered, by this value; the Line-Segment search windows are
// taken in it. Every use evaluates this one function, so its float32 rounding is the same everywhere.
__device__ __forceinline__ float rel_phi(float x, float y, float phic) {
  float d = atan2f(y, x) - phic;
  if (d <= -3.14159265f) d += 6.28318531f;
  if (d > 3.14159265f) d -= 6.28318531f;
  return d;
}
// An output-only per-object float: stored as IEEE binary16 (round to nearest) when the half array
// is set, else as float32.
__device__ __forceinline__ void store_out(float* f32, uint16_t* f16, int64_t i, float v) {
  if (f16) f16[i] = __half_as_ushort(__float2half_rn(v));
  else f32[i] = v;
}

// Unsigned key with the order of the float (for sorting floats as integers)
__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Warp-aggregated atomic add of `pred ? 1 : 0` per lane; returns each predicated lane's slot.
__device__ __forceinline__ int warp_agg_slot(bool pred, int* counter) {
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, pred);
  if (m == 0) return -1;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane_id() == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(act, base, leader);
  return pred ? base + __popc(m & ((1u << lane_id()) - 1u)) : -1;
}

// warp-aggregated slot reservation where lanes may target different counters (counters[key])
__device__ __forceinline__ int warp_agg_slot_keyed(bool pred, int key, int* counters) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  int slot = -1;
  if (pred) {
    const unsigned grp = __match_any_sync(m, key);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane_id() == leader) base = atomicAdd(&counters[key], __popc(grp));
    base = __shfl_sync(grp, base, leader);
    slot = base + __popc(grp & ((1u << lane_id()) - 1u));
  }
  return slot;
}

}  // namespace lst
