// Triplets and Quintuplets (paper Sec. 2.3).
//
// T3: two LS sharing an MD. The circle through the three anchor hits gives a pT estimate
// (pT = k R >= f_t3 pT_thr) and an impact parameter (|hypot(centre) - R| <= d0_t3); a straight
// line in (arc length, z) through the anchors gives chi2_rz <= chi2_t3.
// T5: two T3 sharing an MD. Inner and outer T3 curvatures must agree
// (|k_in - k_out| <= c_rel max + c_abs); Karimaki's circle fit of the five anchors and an r-z line
// fit give chi2_c <= chi2_t5_c and chi2_rz <= chi2_t5_rz.
//
// Candidates are enumerated in float32 with a conservative pre-filter; the survivors are decided
// (and their stored floats computed) in double-float arithmetic (float64-exact outside ~1e-12 of a
// threshold) from the float32 hit coordinates.
#include <type_traits>

#include "lst_internal.h"

namespace lst {
namespace {

template <class T>
struct Anchor {
  T x, y, z, r;
  bool ec;
};

template <class T>
__device__ __forceinline__ Anchor<T> anchor(const Ws& w, int d) {
  Anchor<T> a;
  const float4 p = w.md_xyzr[d];
  a.x = (T)p.x;
  a.y = (T)p.y;
  a.z = (T)p.z;
  if constexpr (sizeof(T) == 4) a.r = p.w;
  else if constexpr (std::is_same<T, ff>::value) a.r = ff_fast_two_sum(p.w, w.md_rlo[d]);   // r to ~2^-47
  else a.r = m_sqrt(a.x * a.x + a.y * a.y);
  a.ec = w.md_ec[d] != 0;
  return a;
}

// T3 selection on anchors (h1, h2, h3), in the decision precision (double-float): circle through
// the anchors with the pT and d0 cuts, and the straight-line fit in (s, z) of the three anchors in
// closed form: chi2 = (c.z)^2 / sum(c_i^2 sigma_i^2) with c = (s3 - s2, s1 - s3, s2 - s1), the
// combination of the z's that every line annuls (identical to the weighted least-squares fit's chi2).
template <class T>
__device__ __forceinline__ int t3_eval(const Cst<T>& c, const Anchor<T>& h1, const Anchor<T>& h2,
                                       const Anchor<T>& h3, Circle3<T>& circ, T& chi2) {
  circ = circle3<T>(h1.x, h1.y, h2.x, h2.y, h3.x, h3.y);
  const T ak = m_abs(circ.kappa);
  typename AccOf<T>::type acc;
  acc.cut_ge(c.f_t3 * c.pt_thr, c.k * circ.R);
  acc.cut(c.d0_t3, circ.d0);
  const T two_r = T(2) / ak;
  const T s1 = arc_len(ak, two_r, h1.r), s2 = arc_len(ak, two_r, h2.r), s3 = arc_len(ak, two_r, h3.r);
  if (!(s3 > s1)) {
    acc.reject();
    chi2 = T(1) / T(0);
  } else {
    const T b0 = m_abs((h3.z - h1.z) / (s3 - s1));
    const T sg1 = m_max(h1.ec ? c.sigma_r * b0 : c.sigma_z, c.sigma_floor);
    const T sg2 = m_max(h2.ec ? c.sigma_r * b0 : c.sigma_z, c.sigma_floor);
    const T sg3 = m_max(h3.ec ? c.sigma_r * b0 : c.sigma_z, c.sigma_floor);
    const T c1 = s3 - s2, c2 = s1 - s3, c3 = s2 - s1;
    const T num = c1 * h1.z + c2 * h2.z + c3 * h3.z;
    const T den = c1 * c1 * sg1 * sg1 + c2 * c2 * sg2 * sg2 + c3 * c3 * sg3 * sg3;
    chi2 = num * num / den;
    acc.cut(c.chi2_t3, chi2);
  }
  return acc.verdict();
}

// Quick rejection of a T3 candidate from its three anchors, exact-safe (true only when the float64
// selection is certain to reject; margins far above float32 rounding). With u = p2 - p1,
// v = p3 - p1 and cr = u x v:
//  pT: k R >= f pT_thr  <=>  4 cr^2 <= kappa_max^2 |u|^2 |v|^2 |v - u|^2 (no square root);
//  d0: the circle through 0, u, v (frame at p1) has centre c' = N / (2 cr), N = (|u|^2 v_y - |v|^2 u_y,
//    |v|^2 u_x - |u|^2 v_x), so with c = p1 + c' and R = |c'|, Q = cr (|c|^2 - R^2) = |p1|^2 cr + p1.N
//    and d0 = ||c| - R| = |Q| / (|cr| (|c| + R)); since |cr| (|c| + R) <= |p1| |cr| + |N|, a |Q| above
//    d0_t3 (|p1|_1 |cr| + |N|_1) rejects, without a division or a square root.
__device__ __forceinline__ bool t3_quick_reject(const Cst<float>& c, float kmax2, float x1, float y1, float x2,
                                                float y2, float x3, float y3) {
  const float ux = x2 - x1, uy = y2 - y1, vx = x3 - x1, vy = y3 - y1;
  const float cr = diff_prod(ux, vy, uy, vx);
  const float uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
  const float wx = vx - ux, wy = vy - uy;
  if (4.0f * cr * cr > kmax2 * (uu * vv * (wx * wx + wy * wy))) return true;
  const float Nx = uu * vy - vv * uy, Ny = vv * ux - uu * vx;
  const float Q = fmaf(x1 * x1 + y1 * y1, cr, fmaf(x1, Nx, y1 * Ny));
  const float p1 = fabsf(x1) + fabsf(y1);
  const float bound = c.d0_t3 * fmaf(p1, fabsf(cr), fabsf(Nx) + fabsf(Ny));
  return fabsf(Q) > fmaf(bound, 1.001f, 1e-6f * p1 * fabsf(cr));
}

// T3 candidates, flattened across each warp: the warp takes 32 inner LS, a warp scan of their
// outer-LS list lengths turns the (inner, outer) pairs into one index range, and each lane finds
// its pair's inner LS by a shuffle search. Pairs that pass the quick test go to a per-warp queue;
// whenever it holds 32, the full float32 pre-filter runs on them with every lane busy.
constexpr int kT3Warps = 8;
constexpr int kT3Q = 64;

// Float32 pre-filter of a T3 candidate that passed the quick test (whose pT and d0 bounds already
// hold): the r-z chi2 of the three anchors in closed form. For three points the best straight line
// leaves chi2 = (c.z)^2 / sum(c_i^2 sigma_i^2) with c = (s3 - s2, -(s3 - s1), s2 - s1), the one
// combination of the z's that every line annuls, which equals the weighted least-squares fit's
// chi2. Rejects only chi2 clearly above the cut (the float32 error is ~1e-3 relative).
__device__ __forceinline__ bool t3_pre_keep(const Cst<float>& c, const Anchor<float>& h1, const Anchor<float>& h2,
                                            const Anchor<float>& h3) {
  const float ux = h2.x - h1.x, uy = h2.y - h1.y, vx = h3.x - h1.x, vy = h3.y - h1.y;
  const float cr = diff_prod(ux, vy, uy, vx);
  const float wx = h3.x - h2.x, wy = h3.y - h2.y;
  const float rs = sqrtf((ux * ux + uy * uy) * (vx * vx + vy * vy) * (wx * wx + wy * wy));
  const float ak = 2.0f * fabsf(cr) / rs;   // |curvature| of the circle through the anchors
  const float two_r = 2.0f / ak;
  const float s1 = arc_len(ak, two_r, h1.r), s2 = arc_len(ak, two_r, h2.r), s3 = arc_len(ak, two_r, h3.r);
  if (!(s3 > s1)) return true;   // decided in double-float
  const float b0 = (h3.z - h1.z) / (s3 - s1);
  const float sg1 = fmaxf(h1.ec ? c.sigma_r * fabsf(b0) : c.sigma_z, c.sigma_floor);
  const float sg2 = fmaxf(h2.ec ? c.sigma_r * fabsf(b0) : c.sigma_z, c.sigma_floor);
  const float sg3 = fmaxf(h3.ec ? c.sigma_r * fabsf(b0) : c.sigma_z, c.sigma_floor);
  const float c1 = s3 - s2, c2 = s1 - s3, c3 = s2 - s1;
  const float num = c1 * h1.z + c2 * h2.z + c3 * h3.z;
  const float den = c1 * c1 * sg1 * sg1 + c2 * c2 * sg2 * sg2 + c3 * c3 * sg3 * sg3;
  return !(num * num > (c.chi2_t3 * (1.0f + kGuardChi2) + kGuardChi2Abs) * den);
}

__device__ __forceinline__ void t3_flush(const Ws& w, const Cst<float>& c, const int2* qe, int n) {
  const int lane = threadIdx.x & 31;
  bool keep = false;
  int2 e = make_int2(0, 0);
  if (lane < n) {
    e = qe[lane];
    keep = t3_pre_keep(c, anchor<float>(w, w.ls_in[e.x]), anchor<float>(w, w.ls_out[e.x]),
                       anchor<float>(w, w.ls_out[e.y]));
  }
  const int q = warp_agg_slot(keep, &w.status[ST_Q_T3]);
  if (q >= 0 && q < w.cap.q_t3) w.q_t3[q] = e;
}

__global__ void __launch_bounds__(32 * kT3Warps) k_t3_pre(Ws w, Cst<float> c) {
  __shared__ int2 queue[kT3Warps][kT3Q];
  int2* qe = queue[threadIdx.x >> 5];
  const int n_ls = w.ls_off[w.V];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const float kmax = c.k / (c.f_t3 * c.pt_thr);
  const float kmax2 = kmax * kmax * (1.0f + 4.0f * kGuardWindow);
  int qn = 0;
  const long long t0 = clock64();
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n_ls; base += nwarps * 32) {
    if (warp_over_budget(w, t0)) break;
    const int i = base + lane;
    int j0 = 0, size = 0;
    float x1 = 0.f, y1 = 0.f, x2 = 0.f, y2 = 0.f;
    if (i < n_ls) {
      const int d1 = w.ls_in[i], d2 = w.ls_out[i];
      j0 = min(w.lsin_off[d2], n_ls);
      size = min(w.lsin_off[d2 + 1], n_ls) - j0;
      const float4 p1 = w.md_xyzr[d1];
      x1 = p1.x; y1 = p1.y;
      const float2 p2 = w.ls_xy_out[i];
      x2 = p2.x; y2 = p2.y;
    }
    int incl = size;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - size;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int b = 0; b < total; b += 32) {
      const int cidx = b + lane;
      int lo = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int cand = lo + step;
        if (__shfl_sync(0xffffffffu, excl, cand) <= cidx) lo = cand;
      }
      const int jj = __shfl_sync(0xffffffffu, j0, lo) + (cidx - __shfl_sync(0xffffffffu, excl, lo));
      const float ax = __shfl_sync(0xffffffffu, x1, lo), ay = __shfl_sync(0xffffffffu, y1, lo);
      const float bx = __shfl_sync(0xffffffffu, x2, lo), by = __shfl_sync(0xffffffffu, y2, lo);
      bool keep = false;
      if (cidx < total) {
        const float2 p3 = w.ls_xy_out[jj];
        keep = !t3_quick_reject(c, kmax2, ax, ay, bx, by, p3.x, p3.y);
      }
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      if (keep) qe[qn + __popc(km & ((1u << lane) - 1u))] = make_int2(base + lo, jj);
      qn += __popc(km);
      if (qn >= 32) {
        __syncwarp();
        t3_flush(w, c, qe, 32);
        __syncwarp();
        qn -= 32;
        if (lane < qn) qe[lane] = qe[32 + lane];
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (qn > 0) t3_flush(w, c, qe, qn);
}

// float64-exact decision of the pre-filter's survivors, evaluated in double-float
__global__ void k_t3_decide(Ws w, Cst<ff> c) {
  const int n = min((int64_t)w.status[ST_Q_T3], w.cap.q_t3);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 q = w.q_t3[k];
    const int md0 = w.ls_in[q.x], md1 = w.ls_out[q.x], md2 = w.ls_out[q.y];
    Circle3<ff> circ;
    ff chi2;
    const int v = t3_eval<ff>(c, anchor<ff>(w, md0), anchor<ff>(w, md1), anchor<ff>(w, md2), circ, chi2);
    if (v != kAccept) continue;
    const int vm = w.md_vm[md0];
    const int slot = atomicAdd(&w.t3_cnt[vm], 1);
    const int cap = w.t3_cap[vm], base = w.t3_base[vm];
    if (slot < cap && (int64_t)base + slot < w.cap.t3_slots) {
      const int s = base + slot;
      w.t3s_a[s] = q.x;
      w.t3s_b[s] = q.y;
      atomicAdd(&w.t3md_off[md0 + 1], 1);
      w.t3s_R[s] = (float)circ.R;
      w.t3s_xc[s] = (float)circ.xc;
      w.t3s_yc[s] = (float)circ.yc;
      w.t3s_chi2[s] = (float)chi2;
      w.t3s_pte[s] = (float)m_min(c.k * circ.R, c.pt_cap);
    }
  }
}

__device__ __forceinline__ int clamp_cap2(double pred, long long bound, int ovr) {
  long long p = (long long)ceil(pred);
  if (p < ovr) p = ovr;
  if (p > bound) p = bound;
  if (p > (1 << 28)) p = 1 << 28;
  return (int)p;
}

// T3 capacity of module vm from its bound (the number of (inner LS, outer LS) pairs whose inner LS
// starts in vm, summed while the LS were compacted)
__global__ void k_t3_caps(Ws w) {
  zero_group_counts(w.t3md_off, w.md_off[w.V]);   // T3 are grouped by first MD
  clamp_group_offsets(w.lsin_off, w.md_off[w.V], w.cap.ls_dense, w.status[ST_DENSE_LS] != 0);
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const long long bound = (long long)w.t3_bound[vm];
    const int cc = clamp_cap2(w.cap_scale * w.stage_scale[2] * (32.0 + 0.5 * (double)bound), bound, w.t3_ovr[vm]);
    w.t3_cap[vm] = cc;
    w.t3_base[vm] = cc;
  }
}


// T5 capacity of module vm from its bound (the number of (inner T3, outer T3) pairs whose inner T3
// starts in vm, summed while the T3 were compacted)
__global__ void k_t5_caps(Ws w) {
  zero_group_counts(w.grp_key, w.t3_off[w.V]);   // T5 are grouped by inner T3
  clamp_group_offsets(w.t3md_off, w.md_off[w.V], w.cap.t3_dense, w.status[ST_DENSE_T3] != 0);
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const long long bound = (long long)w.t5_bound[vm];
    const int cc = clamp_cap2(w.cap_scale * w.stage_scale[3] * (16.0 + 0.5 * (double)bound), bound, w.t5_ovr[vm]);
    w.t5_cap[vm] = cc;
    w.t5_base[vm] = cc;
  }
}

__device__ __forceinline__ float kappa_of(float R) { return isinf(R) ? 0.0f : 1.0f / R; }

// T5 candidates: the curvature-compatibility window in float32 with the window guard, then
// Karimaki's fit and the r-z fit in float32 as a pre-filter (rejects only chi2 > 1.25 cut + 1: the
// float32 fit parameters enter chi2 at second order and the residual rounding at ~0.3 %).
// Flattened across each warp like the T3 candidates: the warp takes 32 inner T3, a warp scan of
// their outer-T3 list lengths turns the (inner, outer) pairs into one index range, each lane takes
// one pair through the window test, and the pairs that pass go to a per-warp queue whose fits run
// 32 at a time with every lane busy.
constexpr int kT5Warps = 8;
constexpr int kT5Q = 64;

// the float32 fits of the first n (<= 32) queued (inner, outer) T3 pairs, one per lane; the pairs
// that pass go to the decision queue. Called by the whole warp.
__device__ __forceinline__ void t5_flush(const Ws& w, const Cst<float>& c, const int2* qe, int n) {
  const int lane = threadIdx.x & 31;
  const int64_t T = w.cap.t3_dense;
  bool keep = false;
  int2 e = make_int2(0, 0);
  if (lane < n) {
    e = qe[lane];
    float x[5], y[5], z[5], r[5];
    bool ec[5];
    const uint8_t ecm_i = w.t3_ecm[e.x], ecm_j = w.t3_ecm[e.y];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 a4 = w.t3_anc[k * T + e.x];
      x[k] = a4.x; y[k] = a4.y; z[k] = a4.z; r[k] = a4.w;
      ec[k] = (ecm_i >> k) & 1;
    }
#pragma unroll
    for (int k = 1; k < 3; ++k) {
      const float4 a4 = w.t3_anc[k * T + e.y];
      x[k + 2] = a4.x; y[k + 2] = a4.y; z[k + 2] = a4.z; r[k + 2] = a4.w;
      ec[k + 2] = (ecm_j >> k) & 1;
    }
    float rho, phi, d, sp, cp;
    karimaki<float, 5>(x, y, rho, phi, d, sp, cp);
    const float chi2c = circle_chi2<float, 5>(x, y, rho, sp, cp, d, c.sigma_rphi);
    keep = !(chi2c > 1.25f * c.chi2_t5_c + 1.0f);
    if (keep) {
      float chi2rz, slope;
      if (rz_fit<float, 5>(c, fabsf(rho), r, z, ec, chi2rz, slope) && chi2rz > 1.25f * c.chi2_t5_rz + 1.0f)
        keep = false;
    }
  }
  const int q = warp_agg_slot(keep, &w.status[ST_Q_T5]);
  if (q >= 0 && q < w.cap.q_t5) w.q_t5[q] = e;
}

__global__ void __launch_bounds__(32 * kT5Warps) k_t5_pre(Ws w, Cst<float> c) {
  __shared__ int2 queue[kT5Warps][kT5Q];
  int2* qe = queue[threadIdx.x >> 5];
  const int n_t3 = w.t3_off[w.V];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  int qn = 0;
  const long long t0 = clock64();
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n_t3; base += nwarps * 32) {
    if (warp_over_budget(w, t0)) break;
    const int i = base + lane;
    int j0 = 0, size = 0;
    float kin = 0.f;
    if (i < n_t3) {
      const int m3 = w.t3_md2[i];
      j0 = w.t3md_off[m3];
      size = w.t3md_off[m3 + 1] - j0;
      kin = kappa_of(w.t3_R[i]);
    }
    int incl = size;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - size;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int b = 0; b < total; b += 32) {
      const int cidx = b + lane;
      int lo = 0;   // the lane whose inner T3 holds pair cidx
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int cand = lo + step;
        if (__shfl_sync(0xffffffffu, excl, cand) <= cidx) lo = cand;
      }
      const int jj = __shfl_sync(0xffffffffu, j0, lo) + (cidx - __shfl_sync(0xffffffffu, excl, lo));
      const float kin_i = __shfl_sync(0xffffffffu, kin, lo);
      bool keep = false;
      if (cidx < total) {
        const float kout = kappa_of(w.t3_R[jj]);
        Acc32 acc(kGuardWindow);
        acc.cut(c.c_rel * fmaxf(kin_i, kout) + c.c_abs, fabsf(kin_i - kout));
        keep = !acc.fail;
      }
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      if (keep) qe[qn + __popc(km & ((1u << lane) - 1u))] = make_int2(base + lo, jj);
      qn += __popc(km);
      if (qn >= 32) {
        __syncwarp();
        t5_flush(w, c, qe, 32);
        __syncwarp();
        qn -= 32;
        if (lane < qn) qe[lane] = qe[32 + lane];
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (qn > 0) t5_flush(w, c, qe, qn);
}

// float64-exact decision of the pre-filter's survivors, evaluated in double-float
__global__ void k_t5_decide(Ws w, Cst<ff> c) {
  const int n = min((int64_t)w.status[ST_Q_T5], w.cap.q_t5);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 q = w.q_t5[k];
    const int i = q.x, j = q.y;
    const float Ri = w.t3_R[i], Rj = w.t3_R[j];
    const ff kin = isinf(Ri) ? ff(0.0f) : ff(1.0f) / ff(Ri);
    const ff kout = isinf(Rj) ? ff(0.0f) : ff(1.0f) / ff(Rj);
    AccFF acc;
    acc.cut(c.c_rel * m_max(kin, kout) + c.c_abs, m_abs(kin - kout));
    if (acc.fail) continue;
    const int md[5] = {w.t3_md0[i], w.t3_md1[i], w.t3_md2[i], w.t3_md1[j], w.t3_md2[j]};
    ff x[5], y[5], z[5], r[5];
    bool ec[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const float4 p = w.md_xyzr[md[a]];
      x[a] = ff(p.x);
      y[a] = ff(p.y);
      z[a] = ff(p.z);
      r[a] = ff_fast_two_sum(p.w, w.md_rlo[md[a]]);   // the MD's radius as a float pair (~2^-47)
      ec[a] = w.md_ec[md[a]] != 0;
    }
    ff rho, phi, d, sp, cp;
    karimaki<ff, 5>(x, y, rho, phi, d, sp, cp);
    const ff chi2c = circle_chi2<ff, 5>(x, y, rho, sp, cp, d, c.sigma_rphi);
    acc.cut(c.chi2_t5_c, chi2c);
    ff chi2rz, slope;
    if (!rz_fit<ff, 5>(c, m_abs(rho), r, z, ec, chi2rz, slope)) {
      acc.reject();
    } else {
      acc.cut(c.chi2_t5_rz, chi2rz);
    }
    if (acc.fail) continue;
    const int vm = w.md_vm[md[0]];
    const int slot = atomicAdd(&w.t5_cnt[vm], 1);
    const int cap = w.t5_cap[vm], base = w.t5_base[vm];
    if (slot < cap && (int64_t)base + slot < w.cap.t5_slots) {
      const int s = base + slot;
      const int64_t S = w.cap.t5_slots;
      w.t5s_a[s] = i;
      w.t5s_b[s] = j;
      atomicAdd(&w.grp_key[i + 1], 1);
      w.t5s_f[0 * S + s] = (float)kin;
      w.t5s_f[1 * S + s] = (float)kout;
      w.t5s_f[2 * S + s] = (float)rho;
      w.t5s_f[3 * S + s] = (float)chi2c;
      w.t5s_f[4 * S + s] = (float)chi2rz;
      w.t5s_f[5 * S + s] = asinhf((float)slope);
      w.t5s_f[6 * S + s] = (float)phi;
      w.t5s_f[7 * S + s] = rho.hi == 0.0f ? (float)c.pt_cap : (float)m_min(c.k / m_abs(rho), c.pt_cap);
    }
  }
}

// dense T5 ordered by (inner T3, outer T3), with member MDs, fit results and an anchor cache
__global__ void k_t5_dense(Ws w) {
  const int n = (int)lst_min64(w.t5_off[w.V], w.cap.t5_dense);
  const int n_mods = w.V / w.E;
  const int64_t S = w.cap.t5_slots, D = w.cap.t5_dense;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
    const int s = w.perm[d];
    const int a = w.t5s_a[s], b = w.t5s_b[s];
    w.t5_a[d] = a;
    w.t5_b[d] = b;
    const int md[5] = {w.t3_md0[a], w.t3_md1[a], w.t3_md2[a], w.t3_md1[b], w.t3_md2[b]};
    uint8_t ecm = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      w.t5_md[k * D + d] = md[k];
      w.t5_anc[k * D + d] = w.md_xyzr[md[k]];
      w.t5_anc_rlo[k * D + d] = w.md_rlo[md[k]];
      ecm |= (uint8_t)(w.md_ec[md[k]] << k);
    }
    w.t5_ecm[d] = ecm;
    // event-local member indices (the T3 of the event start at the first T3 of its first module)
    const int vm = w.md_vm[md[0]];
    const int first_t3 = w.t3_off[vm - vm % n_mods];
    w.o_t5_a[d] = a - first_t3;
    w.o_t5_b[d] = b - first_t3;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      // kappa_in, kappa_out and chi2_rz are outputs only (binary16 when enabled); the others are read
      // by later selections and stay float32
      const int h = f == 0 ? 0 : f == 1 ? 1 : f == 4 ? 2 : -1;
      if (h >= 0 && w.t5_h) store_out(nullptr, w.t5_h + (int64_t)h * D, d, w.t5s_f[f * S + s]);
      else w.t5_f[f * D + d] = w.t5s_f[f * S + s];
    }
  }
}

int resident_blocks(const void* kernel, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

int t3_pre_resident_blocks() { return resident_blocks(reinterpret_cast<const void*>(k_t3_pre), 32 * kT3Warps); }
int t5_pre_resident_blocks() { return resident_blocks(reinterpret_cast<const void*>(k_t5_pre), 32 * kT5Warps); }

void run_t3(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  (void)g;
  k_t3_caps<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w);
  LST_LAUNCH(L);
  scan_exclusive(w.t3_base, w.t3_base, w.V, w.scan_tmp, L);
  KT_BEGIN(L, K_T3_PRE);
  // every resident block and no more: the blocks divide the inner LS statically, so a second,
  // partly filled wave would hold up the launch
  k_t3_pre<<<L.n_sm * (L.t3_blocks_per_sm > 0 ? L.t3_blocks_per_sm : 8), 32 * kT3Warps, 0, L.stream>>>(w, c.f);
  KT_END(L, K_T3_PRE);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_T3_DECIDE);
  k_t3_decide<<<grid_for(w.cap.q_t3, 128, 152 * 8), 128, 0, L.stream>>>(w, c.x);
  KT_END(L, K_T3_DECIDE);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_T3_COMPACT);
  GroupArgs ga{w.t3_cnt, w.t3_cap, w.t3_base, w.cap.t3_slots, ST_OVF_T3, ST_ARENA_T3, w.t3s_a, w.t3s_b,
               w.ls_in, w.t3md_off, w.cap.md_dense, &w.md_off[w.V], w.cap.t3_dense, ST_DENSE_T3,
               w.t3_off, w.md_off, 1, kDenseT3};
  // T3 grouped by their first MD (the inner MD of their inner LS; LS are ordered by inner MD, so the
  // (inner LS, outer LS) order is kept inside each group): the group offsets are the T3-by-first-MD
  // adjacency that the T5 stage reads
  group_slots(w, ga, L);   // (writes the dense T3: t3_dense_write)
  KT_END(L, K_T3_COMPACT);
}

void run_t5(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  (void)g;
  k_t5_caps<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w);
  LST_LAUNCH(L);
  scan_exclusive(w.t5_base, w.t5_base, w.V, w.scan_tmp, L);
  KT_BEGIN(L, K_T5_PRE);
  k_t5_pre<<<L.n_sm * (L.t5_blocks_per_sm > 0 ? L.t5_blocks_per_sm : 8), 32 * kT5Warps, 0, L.stream>>>(w, c.f);
  KT_END(L, K_T5_PRE);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_T5_DECIDE);
  k_t5_decide<<<grid_for(w.cap.q_t5, 128, 152 * 8), 128, 0, L.stream>>>(w, c.x);
  KT_END(L, K_T5_DECIDE);
  LST_LAUNCH(L);
  GroupArgs ga{w.t5_cnt, w.t5_cap, w.t5_base, w.cap.t5_slots, ST_OVF_T5, ST_ARENA_T5, w.t5s_a, w.t5s_b,
               nullptr, nullptr, w.cap.t3_dense, &w.t3_off[w.V], w.cap.t5_dense, ST_DENSE_T5,
               w.t5_off, w.t3_off, 1, kDensePerm};
  group_slots(w, ga, L);
  k_t5_dense<<<grid_for(w.cap.t5_dense, 256), 256, 0, L.stream>>>(w);
  LST_LAUNCH(L);
}

}  // namespace lst
