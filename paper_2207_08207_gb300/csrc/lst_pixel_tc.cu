// Pixel seeds, pT3 / pT5 (paper Sec. 2.4) and Track Candidates with cross-cleaning (Sec. 2.5).
//
// pT3 / pT5: a seed (pLS) is linked to a T3 / T5 whose first MD lies in a module the pixel map
// lists for the seed's (eta, phi, charge) bin. The seed's helix is not refitted: the outer anchor
// hits are tested against the circle and the r-z line the seed's parameters define (chi2_xy and
// chi2_rz cuts; per-anchor uncertainties from the hit resolution and the seed's direction and pT
// uncertainties).
// Track candidates: pT5, then pT3, then T5, then pLS (Sec. 2.5). One pT5 and one pT3 per seed (lowest
// (score, hit tuple)); T5 duplicates removed (a T5 sharing >= 7 of 10 hits with a T5 of lower
// (chi2, hit tuple) is dropped); pT3 kept only if no accepted pT5 uses its seed or lies within
// dR < dr_min; T5 only if no accepted pT5 / pT3 is within dR; pLS only if it is in no pT3 / pT5 and
// no accepted candidate is within dR. Output ordered by type, then sorted hit tuple.
#include <type_traits>

#include "lst_internal.h"

namespace lst {
namespace {

__device__ __forceinline__ int find_seg(const int32_t* off, int n, int i) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// seed helix in precision T: circle centre c = (x0, y0) + (1/rho) n, n = (sin phi, -cos phi),
// rho = q / R, R = pT / k
template <class T>
struct Seed {
  T x0, y0, z0, rho, akap, sp, cp, cot, R;
};

template <class T>
__device__ __forceinline__ Seed<T> make_seed(const lst_pls& s, const Cst<T>& c) {
  Seed<T> o;
  o.x0 = s.x0; o.y0 = s.y0; o.z0 = s.z0;
  o.R = (T)s.pt / c.k;
  o.akap = T(1) / o.R;
  o.rho = s.charge > 0 ? o.akap : -o.akap;
  if constexpr (sizeof(T) == 4) {
    sincosf(s.phi, &o.sp, &o.cp);
    o.cot = sinhf(s.eta);
  } else if constexpr (std::is_same<T, ff>::value) {
    ff_sincos(s.phi, o.sp, o.cp);
    o.cot = ff_sinh(s.eta);
  } else {
    sincos((double)s.phi, &o.sp, &o.cp);
    o.cot = sinh((double)s.eta);
  }
  return o;
}

// ---------------------------------------------------------------------------------------------
// pixel seeds: validation and pixel-map bin. The bin index is computed in float64 with explicitly
// rounded operations (floor(20 eta + 50), floor(phi_[0,2pi) * 64 / pi)), the same sequence of IEEE
// operations any implementation of the definition performs.
// ---------------------------------------------------------------------------------------------
__global__ void k_pls_prep(Ws w, Geo g, Cst<float> c, Cst<ff> cx) {
  const int P = w.n_pls();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const lst_pls s = w.pls[p];
    const bool ok = isfinite(s.pt) && isfinite(s.eta) && isfinite(s.phi) && isfinite(s.x0) &&
                    isfinite(s.y0) && isfinite(s.z0) && s.pt > 0.f && (s.charge == 1 || s.charge == -1);
    int bin = -1;
    const int e = find_seg(w.ev_pls_off, w.E, p);
    w.pls_ev[p] = e;
    if (!ok) {
      atomicOr(&w.status[ST_ERROR], ERR_BAD_PLS);
      atomicOr(&w.ev_stat[e * kEvWords + kEvErr], ERR_BAD_PLS);
    } else if (g.n_pix_bins > 0) {
      const double ie = floor(__dadd_rn(__dmul_rn((double)s.eta, 20.0), 50.0));
      if (ie >= 0.0 && ie < (double)kPixNEta) {
        double ph = (double)s.phi;
        if (ph < 0.0) ph = __dadd_rn(ph, kTwoPiD);
        double ip = floor(__dmul_rn(ph, 64.0 / kPiD));
        ip = fmin(fmax(ip, 0.0), (double)(kPixNPhi - 1));
        bin = ((int)ie * kPixNPhi + (int)ip) * 2 + (s.charge > 0 ? 1 : 0);
        if (bin >= g.n_pix_bins) bin = -1;
      }
    }
    w.pls_bin[p] = bin;
    if (bin >= 0) {   // the seed helix, once per seed: float32 for the pre-filters, double-float
                      // for the decisions
      const Seed<float> sd = make_seed<float>(s, c);
      w.pls_seed[p] = make_float4(sd.x0, sd.y0, sd.z0, sd.rho);
      w.pls_seed[w.P + p] = make_float4(sd.akap, sd.sp, sd.cp, sd.cot);
      const Seed<ff> sx = make_seed<ff>(s, cx);
      const ff v[9] = {sx.x0, sx.y0, sx.z0, sx.rho, sx.akap, sx.sp, sx.cp, sx.cot, sx.R};
      float2* o = w.pls_seed_ff + (int64_t)p * 9;
#pragma unroll
      for (int k = 0; k < 9; ++k) o[k] = make_float2(v[k].hi, v[k].lo);
    }
  }
}

// distance of (x, y) from the seed circle, |p - c| - R up to sign, as 2A / (1 + sqrt(1 + 2 rho A))
// with A = rho/2 |u|^2 - u.n, u = p - (x0, y0): exact, and free of the cancellation of |p-c| - R
template <class T>
__device__ __forceinline__ T seed_dist(const Seed<T>& s, T x, T y) {
  const T ux = x - s.x0, uy = y - s.y0;
  const T A = T(0.5) * s.rho * (ux * ux + uy * uy) - (ux * s.sp - uy * s.cp);
  return T(2) * A / (T(1) + m_sqrt(T(1) + T(2) * s.rho * A));
}

template <class T>
__device__ __forceinline__ void seed_terms(const Seed<T>& s, const Cst<T>& c, T x, T y, T z, T r,
                                           bool ec, T& xy_term, T& rz_term) {
  const T d = seed_dist(s, x, y);
  const T e1 = r * c.pls_dir_err;
  const T e2 = c.pls_pt_err * r * r * T(0.5) * s.akap;
  xy_term = d * d / (c.sigma_rphi * c.sigma_rphi + e1 * e1 + e2 * e2);
  const T sa = arc_len(s.akap, T(2) * s.R, r);
  const T zp = s.z0 + sa * s.cot;
  const T sz = ec ? c.sigma_r * m_abs(s.cot) : c.sigma_z;
  const T th = sa * (T(1) + s.cot * s.cot) * c.pls_dir_err;
  rz_term = (z - zp) * (z - zp) / (sz * sz + th * th);
}

// member anchors of T3 / T5 objects: anc[k * stride + i] = (x, y, z, r) of anchor k of object i,
// ecm[i] bit k = anchor k is on an endcap module
struct ObjAnc {
  const float4* anc;
  const float* rlo;   // low part of each anchor's radius
  const uint8_t* ecm;
  int64_t stride;
};

// bounding boxes of the first anchors of each module's T3 and of its T5 (kBoxLanes lanes per module
// and type: modules hold a few T3 / T5 each, most none), stored in the form the seed test reads:
// box[vm] = (centre x, centre y, half diagonal, largest r), box[V + vm] = (smallest z, largest z,
// smallest r, 1 for an endcap module)
constexpr int kBoxLanes = 4;

__global__ void k_obj_box(Ws w, Geo g) {
  const int sub = threadIdx.x & (kBoxLanes - 1);
  const unsigned gmask = ((1u << kBoxLanes) - 1u) << ((threadIdx.x & 31) & ~(kBoxLanes - 1));
  const int ngroups = gridDim.x * (blockDim.x / kBoxLanes);
  for (int item = (blockIdx.x * blockDim.x + threadIdx.x) / kBoxLanes; item < 2 * w.V; item += ngroups) {
    const bool t5 = item >= w.V;   // items [0, V): T3 boxes; [V, 2V): T5 boxes
    const int vm = t5 ? item - w.V : item;
    const int32_t* obj_off = t5 ? w.t5_off : w.t3_off;
    const float4* anc0 = t5 ? w.t5_anc : w.t3_anc;
    float4* box = t5 ? w.box5 : w.box3;
    const int a = obj_off[vm], b = obj_off[vm + 1];
    if (a == b) continue;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
    for (int i = a + sub; i < b; i += kBoxLanes) {
      const float4 h = anc0[i];
      lo.x = fminf(lo.x, h.x); lo.y = fminf(lo.y, h.y); lo.z = fminf(lo.z, h.z); lo.w = fminf(lo.w, h.w);
      hi.x = fmaxf(hi.x, h.x); hi.y = fmaxf(hi.y, h.y); hi.z = fmaxf(hi.z, h.z); hi.w = fmaxf(hi.w, h.w);
    }
#pragma unroll
    for (int o = kBoxLanes / 2; o >= 1; o >>= 1) {
      lo.x = fminf(lo.x, __shfl_xor_sync(gmask, lo.x, o, kBoxLanes));
      lo.y = fminf(lo.y, __shfl_xor_sync(gmask, lo.y, o, kBoxLanes));
      lo.z = fminf(lo.z, __shfl_xor_sync(gmask, lo.z, o, kBoxLanes));
      lo.w = fminf(lo.w, __shfl_xor_sync(gmask, lo.w, o, kBoxLanes));
      hi.x = fmaxf(hi.x, __shfl_xor_sync(gmask, hi.x, o, kBoxLanes));
      hi.y = fmaxf(hi.y, __shfl_xor_sync(gmask, hi.y, o, kBoxLanes));
      hi.z = fmaxf(hi.z, __shfl_xor_sync(gmask, hi.z, o, kBoxLanes));
      hi.w = fmaxf(hi.w, __shfl_xor_sync(gmask, hi.w, o, kBoxLanes));
    }
    if (sub == 0) {
      const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y);
      box[vm] = make_float4(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), sqrtf(hx * hx + hy * hy), hi.w);
      box[w.V + vm] = make_float4(lo.z, hi.z, lo.w, g.endcap[vm % g.n_mods] ? 1.f : 0.f);
    }
  }
}

// Whole-module rejection for a seed, exact-safe: true only when every object of the module has a
// first-anchor term (alone) above the pre-filter limit, so the chi-square sums are too. b0, b1: the
// module's box (k_obj_box).
//  x-y: the signed distance to the seed circle, |p - c| - R, is 1-Lipschitz, so over the anchors'
//    box it is at least its value at the box centre minus the half diagonal; the resolution term
//    grows with r and is taken at the box's largest r.
//  r-z: the predicted z at radius r, z0 + s(r) cot, is linear in the arc length s(r) = 2R asin(r/2R),
//    so over the box's r range it lies between its values at bounds of s: s(r) >= min(r, pi R) and
//    s(r) <= min(r / sqrt(1 - (r/2R)^2), pi R) (asin x <= tan(asin x); the arc length is capped at pi R
//    where the circle does not reach r), which need no arc sine. The gap between that interval and
//    the box's z range bounds |z - z_pred|; the variance is taken at the largest s bound.
// Margins (1e-3 cm, relative 1e-4, 1/16 on the squared limits, pi rounded outward by 3e-5) lie far
// above float32 rounding.
__device__ __forceinline__ bool seed_box_reject(const Seed<float>& s, const Cst<float>& c, float4 b0, float4 b1,
                                                float lim_xy, float lim_rz) {
  const float ux = b0.x - s.x0, uy = b0.y - s.y0;
  // distance at the centre: at least |A| / g with A = rho/2 |u|^2 - u.n and g = 1 + |rho A| / 2
  // (the exact 2A / (1 + sqrt(1 + 2 rho A)) without its square root and division); the test
  // lb = |A| / g - margin > 0, lb^2 > limit is multiplied through by g
  const float A = 0.5f * s.rho * (ux * ux + uy * uy) - (ux * s.sp - uy * s.cp);
  const float g = 1.0f + 0.5f * fabsf(s.rho * A);
  const float m = b0.z * 1.0001f + 1e-3f + 1e-4f * (fabsf(ux) + fabsf(uy));
  const float lbg = fabsf(A) - m * g;
  const float r_hi = b0.w, r_lo = b1.z;
  if (lbg > 0.f) {
    const float e1 = r_hi * c.pls_dir_err;
    const float e2 = c.pls_pt_err * r_hi * r_hi * 0.5f * s.akap;
    const float sig2 = c.sigma_rphi * c.sigma_rphi + e1 * e1 + e2 * e2;
    if (lbg * lbg > lim_xy * sig2 * 1.0625f * g * g) return true;
  }
  const float xh = 0.5f * s.akap * r_hi;
  const float s_cap = 3.1416f * s.R;
  const float sh = xh < 1.0f ? fminf(r_hi * rsqrtf(1.0f - xh * xh), s_cap) : s_cap;
  const float sl = fminf(r_lo, 3.1415f * s.R);
  const float za = s.z0 + sl * s.cot, zb = s.z0 + sh * s.cot;
  const float zmin = fminf(za, zb), zmax = fmaxf(za, zb);
  const float gap = fmaxf(b1.x - zmax, zmin - b1.y) - 1e-3f -
                    1e-4f * (fabsf(zmin) + fabsf(zmax) + fabsf(b1.x) + fabsf(b1.y));
  if (gap > 0.f) {
    const float sz = b1.w != 0.f ? c.sigma_r * fabsf(s.cot) : c.sigma_z;
    const float th = sh * (1.0f + s.cot * s.cot) * c.pls_dir_err;
    if (gap * gap > lim_rz * (sz * sz + th * th) * 1.0625f) return true;
  }
  return false;
}

__device__ __forceinline__ Seed<float> cached_seed(const Ws& w, int p) {
  const float4 a = w.pls_seed[p], b = w.pls_seed[w.P + p];
  Seed<float> s;
  s.x0 = a.x; s.y0 = a.y; s.z0 = a.z; s.rho = a.w;
  s.akap = b.x; s.sp = b.y; s.cp = b.z; s.cot = b.w;
  s.R = 1.0f / b.x;
  return s;
}

// xy term of one anchor against the remaining room lim - acc, exact-safe: with A = rho/2 |u|^2 - u.n
// the residual is 2A / (1 + sqrt(1 + 2 rho A)), whose size is at least |A| / (1 + |rho A| / 2), so a
// term that exceeds the room on that bound alone is rejected without a square root or a division
__device__ __forceinline__ bool seed_xy_term(const Seed<float>& s, const Cst<float>& c, float4 h, float room,
                                             float& term) {
  const float ux = h.x - s.x0, uy = h.y - s.y0;
  const float A = 0.5f * s.rho * (ux * ux + uy * uy) - (ux * s.sp - uy * s.cp);
  const float e1 = h.w * c.pls_dir_err;
  const float e2 = c.pls_pt_err * h.w * h.w * 0.5f * s.akap;
  const float sig2 = c.sigma_rphi * c.sigma_rphi + e1 * e1 + e2 * e2;
  const float g = 1.0f + 0.5f * fabsf(s.rho * A);
  if (A * A > room * sig2 * g * g) return false;
  const float dd = 2.0f * A / (1.0f + sqrtf(1.0f + 2.0f * s.rho * A));
  term = dd * dd / sig2;
  return true;
}

// full float32 pre-filter of the first n (<= 32) queued (seed, object) pairs, one per lane
template <int N>
__device__ __forceinline__ void pt_flush(const Ws& w, const Cst<float>& c, const ObjAnc& oa, const int2* qe,
                                         int n, float lim_xy, float lim_rz, int2* queue, int q_word,
                                         int64_t q_cap) {
  const int lane = threadIdx.x & 31;
  bool keep = false;
  int2 e = make_int2(0, 0);
  if (lane < n) {
    e = qe[lane];
    const Seed<float> s = cached_seed(w, e.x);
    const int obj = e.y;
    float xy = 0.f, rz = 0.f;
    keep = true;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      float t;
      if (!seed_xy_term(s, c, oa.anc[a * oa.stride + obj], lim_xy - xy, t)) { keep = false; break; }
      xy += t;
      if (xy > lim_xy) { keep = false; break; }
    }
    if (keep) {
      const uint8_t ecm = oa.ecm[obj];
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const float4 h = oa.anc[a * oa.stride + obj];
        const float sa = arc_len(s.akap, 2.0f * s.R, h.w);
        const float zp = s.z0 + sa * s.cot;
        const float sz = ((ecm >> a) & 1) ? c.sigma_r * fabsf(s.cot) : c.sigma_z;
        const float th = sa * (1.0f + s.cot * s.cot) * c.pls_dir_err;
        rz += (h.z - zp) * (h.z - zp) / (sz * sz + th * th);
        if (rz > lim_rz) { keep = false; break; }
      }
    }
  }
  const int q = warp_agg_slot(keep, &w.status[q_word]);
  if (q >= 0 && q < q_cap) queue[q] = e;
}

// Candidate pre-filter: one warp per seed. The seed's pixel-map row is scanned 32 modules at a time;
// modules that cannot hold a passing object are dropped whole (seed_box_reject); the objects of the
// rest are flattened across the warp by a shuffle search over the per-module counts. Each candidate
// gets the first anchor's x-y test; survivors go to a per-warp queue that carries over from seed to
// seed, and whenever it holds 32 the full float32 pre-filter runs on them with every lane busy.
constexpr int kPxMaxWarps = 8;
constexpr int kPxQ = 64;

template <int N>
__global__ void __launch_bounds__(32 * kPxMaxWarps, 4) k_pt_pre(Ws w, Geo g, Cst<float> c, const int32_t* obj_off,
                                                             const float4* box, ObjAnc oa, int2* queue,
                                                             int q_word, int64_t q_cap, float cut_xy,
                                                             float cut_rz) {
  __shared__ int2 qbuf[kPxMaxWarps][kPxQ];
  int2* qe = qbuf[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const float lim_xy = cut_xy * (1.0f + kGuardChi2) + kGuardChi2Abs;
  const float lim_rz = cut_rz * (1.0f + kGuardChi2) + kGuardChi2Abs;
  const int P = w.n_pls();
  int qn = 0;
  const long long t0 = clock64();
  for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += nwarps) {
    if (warp_over_budget(w, t0)) break;
    const int bin = w.pls_bin[p];
    if (bin < 0) continue;
    const int e0 = w.pls_ev[p] * g.n_mods;
    const Seed<float> s = cached_seed(w, p);
    const int tb = g.pix_off[bin], nt = g.pix_off[bin + 1] - tb;
    for (int t0 = 0; t0 < nt; t0 += 32) {
      const int k = t0 + lane;
      int start = 0, size = 0;
      if (k < nt) {
        const int mk = g.pix_tgt[tb + k];
        const int vmk = e0 + mk;
        start = obj_off[vmk];
        size = obj_off[vmk + 1] - start;
        if (size > 0 && seed_box_reject(s, c, box[vmk], box[w.V + vmk], lim_xy, lim_rz)) size = 0;
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
          const int ex = __shfl_sync(0xffffffffu, excl, cand);
          if (ex <= cidx) lo = cand;
        }
        const int st = __shfl_sync(0xffffffffu, start, lo);
        const int ex0 = __shfl_sync(0xffffffffu, excl, lo);
        const int obj = st + (cidx - ex0);
        float t;
        const bool keep = cidx < total && seed_xy_term(s, c, oa.anc[obj], lim_xy, t) && t <= lim_xy;
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) qe[qn + __popc(km & ((1u << lane) - 1u))] = make_int2(p, obj);
        qn += __popc(km);
        if (qn >= 32) {
          __syncwarp();
          pt_flush<N>(w, c, oa, qe, 32, lim_xy, lim_rz, queue, q_word, q_cap);
          __syncwarp();
          qn -= 32;
          if (lane < qn) qe[lane] = qe[32 + lane];
          __syncwarp();
        }
      }
    }
  }
  __syncwarp();
  if (qn > 0) pt_flush<N>(w, c, oa, qe, qn, lim_xy, lim_rz, queue, q_word, q_cap);
}

// decision of the pre-filter's survivors (chi2 sums of the seed's circle and r-z line over the
// object's anchors), evaluated in double-float: float64-exact outside ~1e-12 of a threshold
template <int N>
__global__ void k_pt_decide(Ws w, Cst<ff> c, ObjAnc oa, const int2* queue, int q_word, int64_t q_cap,
                            ff cut_xy, ff cut_rz, int32_t* a_pls, int32_t* a_obj, float* a_xy,
                            float* a_rz, float* a_sc, int n_word, int64_t a_cap, int32_t* per_pls) {
  const int n = min((int64_t)w.status[q_word], q_cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 q = queue[k];
    Seed<ff> s;   // the seed's double-float helix, cached per seed
    {
      const float2* v = w.pls_seed_ff + (int64_t)q.x * 9;
      s.x0 = ff(v[0].x, v[0].y); s.y0 = ff(v[1].x, v[1].y); s.z0 = ff(v[2].x, v[2].y);
      s.rho = ff(v[3].x, v[3].y); s.akap = ff(v[4].x, v[4].y); s.sp = ff(v[5].x, v[5].y);
      s.cp = ff(v[6].x, v[6].y); s.cot = ff(v[7].x, v[7].y); s.R = ff(v[8].x, v[8].y);
    }
    ff xy = ff(0.0f), rz = ff(0.0f);
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const float4 h = oa.anc[a * oa.stride + q.y];
      const ff x(h.x), y(h.y), z(h.z);
      const ff r = ff_fast_two_sum(h.w, oa.rlo[a * oa.stride + q.y]);   // the anchor's radius (~2^-47)
      ff t1, t2;
      seed_terms<ff>(s, c, x, y, z, r, ((oa.ecm[q.y] >> a) & 1) != 0, t1, t2);
      xy += t1;
      rz += t2;
    }
    const bool pass = xy <= cut_xy && rz <= cut_rz;
    const int slot = warp_agg_slot(pass, &w.status[n_word]);   // one atomic per warp on the shared count
    if (!pass || slot >= a_cap) continue;
    a_pls[slot] = q.x;
    a_obj[slot] = q.y;
    a_xy[slot] = (float)xy;
    a_rz[slot] = (float)rz;
    a_sc[slot] = (float)(xy + rz);
    atomicAdd(&per_pls[q.x], 1);
  }
}

// group appended pT objects by seed (ordered by object index within a seed)
__global__ void k_pt_group(Ws w, int n_word, int64_t a_cap, const int32_t* a_pls, const int32_t* a_obj,
                           const int32_t* off, int32_t* cur, int32_t* tmp_idx) {
  const int n = (int)min((int64_t)w.status[n_word], a_cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int p = a_pls[k];
    tmp_idx[off[p] + atomicAdd(&cur[p], 1)] = k;
  }
  (void)a_obj;
}


// ---------------------------------------------------------------------------------------------
// track candidates
// ---------------------------------------------------------------------------------------------
enum TcType : int { TC_PT5 = 0, TC_PT3 = 1, TC_T5 = 2, TC_PLS = 3 };

// hits of an object in output order: seed hits, then (lower, upper) of each MD inner -> outer;
// event-local input indices
__device__ __forceinline__ int md_hits(const Ws& w, int d, int* h) {
  h[0] = w.borig[w.md_lo[d]];
  h[1] = w.borig[w.md_up[d]];
  return 2;
}
__device__ int t5_hits(const Ws& w, int i, int* h) {
  const int64_t S = w.cap.t5_dense;
  int n = 0;
  for (int k = 0; k < 5; ++k) n += md_hits(w, w.t5_md[k * S + i], h + n);
  return n;
}
__device__ int t3_hits(const Ws& w, int i, int* h) {
  int n = md_hits(w, w.t3_md0[i], h);
  n += md_hits(w, w.t3_md1[i], h + n);
  n += md_hits(w, w.t3_md2[i], h + n);
  return n;
}
__device__ int pls_hits(const Ws& w, int p, int* h) {
  const lst_pls s = w.pls[p];
  for (int k = 0; k < 4; ++k) h[k] = s.pix_hit[k];
  return 4;
}
// type / index as stored in a candidate code: pT5 / pT3 -> dense pT index, T5 -> T5, pLS -> seed
__device__ int code_hits(const Ws& w, int type, int idx, int* h) {
  if (type == TC_PT5) {
    const int n = pls_hits(w, w.pt5_pls[idx], h);
    return n + t5_hits(w, w.pt5_obj[idx], h + n);
  }
  if (type == TC_PT3) {
    const int n = pls_hits(w, w.pt3_pls[idx], h);
    return n + t3_hits(w, w.pt3_obj[idx], h + n);
  }
  if (type == TC_T5) return t5_hits(w, idx, h);
  return pls_hits(w, idx, h);
}
__device__ __forceinline__ void sort_small(int* h, int n) {
  for (int i = 1; i < n; ++i) {
    const int v = h[i];
    int j = i - 1;
    while (j >= 0 && h[j] > v) {
      h[j + 1] = h[j];
      --j;
    }
    h[j + 1] = v;
  }
}
// lexicographic comparison of the sorted hit tuples of two candidates of the same type
__device__ bool key_less(const Ws& w, int type, int a, int b) {
  int ha[14], hb[14];
  const int na = code_hits(w, type, a, ha), nb = code_hits(w, type, b, hb);
  sort_small(ha, na);
  sort_small(hb, nb);
  const int n = min(na, nb);
  for (int k = 0; k < n; ++k)
    if (ha[k] != hb[k]) return ha[k] < hb[k];
  return na < nb;
}

// best pT5 and pT3 of each seed by (score, hit tuple): a group of G lanes per seed (gmask: the
// group's lanes), each lane the best of its share of the candidates, then a shuffle reduction
template <int Type, int G>
__device__ __forceinline__ int best_of(const Ws& w, const int32_t* off, const float* sc, int p, int sub,
                                       unsigned gmask) {
  int b = -1;
  for (int i = off[p] + sub; i < off[p + 1]; i += G)
    if (b < 0 || sc[i] < sc[b] || (sc[i] == sc[b] && key_less(w, Type, i, b))) b = i;
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) {
    const int c = __shfl_xor_sync(gmask, b, o, G);
    if (c >= 0 && (b < 0 || sc[c] < sc[b] || (sc[c] == sc[b] && key_less(w, Type, c, b)))) b = c;
  }
  return b;
}

// order each seed's objects by object index (unique within a seed): a group of kPtLanes lanes per
// seed (seeds hold a few objects: a median of 2-3; 16 lanes for pT3, whose seeds reach dozens more
// often, 8 for pT5); each element's output position is its rank, the number of the seed's keys below
// its own (by shuffles up to kPtLanes objects, else with the keys staged in shared memory for up to
// kPtStage). The same group then picks the seed's best candidate
// by (score, hit tuple) for the track-candidate stage; the pT5 pass (the second) also records
// whether the seed is in any pT3 / pT5.
constexpr int kPtOrderWarps = 4;
constexpr int kPtStage = 64;

// event-local outputs of a pT object of seed p and object obj at position o: the seed's index in its
// event, the object's index among the event's T3 / T5 (obj_off: per-module T3 / T5 offsets)
__device__ __forceinline__ void pt_local(const Ws& w, int p, int obj, int o, int n_mods, int32_t* o_pls,
                                         int32_t* o_obj, const int32_t* obj_off) {
  const int e = w.pls_ev[p];
  o_pls[o] = p - w.ev_pls_off[e];
  o_obj[o] = obj - obj_off[e * n_mods];
}
template <int Type> __host__ __device__ constexpr int pt_lanes() { return Type == TC_PT3 ? 16 : 8; }

template <int Type>
__global__ void __launch_bounds__(32 * kPtOrderWarps) k_pt_order(
    Ws w, const int32_t* off, int32_t* tmp_idx, const int32_t* a_pls, const int32_t* a_obj, const float* a_xy,
    const float* a_rz, const float* a_sc, int32_t* d_pls, int32_t* d_obj, float* d_xy, float* d_rz, float* d_sc,
    int32_t* best, int32_t* o_pls, int32_t* o_obj, const int32_t* obj_off, uint16_t* d_xy_h, uint16_t* d_rz_h) {
  constexpr int kPtLanes = pt_lanes<Type>();
  const int n_mods = w.V / w.E;
  __shared__ int keys[32 * kPtOrderWarps / kPtLanes][kPtStage];
  int* K = keys[threadIdx.x / kPtLanes];
  const int sub = threadIdx.x & (kPtLanes - 1);
  const unsigned gmask = ((1u << kPtLanes) - 1u) << ((threadIdx.x & 31) & ~(kPtLanes - 1));
  const int P = w.n_pls();
  const int ngroups = gridDim.x * (blockDim.x / kPtLanes);
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) / kPtLanes; p < P; p += ngroups) {
    const int a = off[p], n = off[p + 1] - a;
    if (n == 0) {
      if (sub == 0) {
        best[p] = -1;
        if (Type == TC_PT5) w.pls_member[p] = w.best3[p] >= 0 ? 1 : 0;
      }
      continue;
    }
    if (n <= kPtLanes) {
      int v = 0, key = 0x7fffffff;
      if (sub < n) {
        v = tmp_idx[a + sub];
        key = a_obj[v];
      }
      int rank = 0;
      for (int j = 0; j < n; ++j) rank += __shfl_sync(gmask, key, j, kPtLanes) < key;
      if (sub < n) {
        const int o = a + rank;
        d_pls[o] = a_pls[v]; d_obj[o] = key; d_sc[o] = a_sc[v];
        store_out(d_xy, d_xy_h, o, a_xy[v]);
        store_out(d_rz, d_rz_h, o, a_rz[v]);
        pt_local(w, p, key, o, n_mods, o_pls, o_obj, obj_off);
      }
    } else {
      const bool staged = n <= kPtStage;
      if (staged)
        for (int j = sub; j < n; j += kPtLanes) K[j] = a_obj[tmp_idx[a + j]];
      __syncwarp(gmask);
      for (int i = sub; i < n; i += kPtLanes) {
        const int v = tmp_idx[a + i];
        const int key = a_obj[v];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += (staged ? K[j] : a_obj[tmp_idx[a + j]]) < key;
        const int o = a + rank;
        d_pls[o] = a_pls[v]; d_obj[o] = key; d_sc[o] = a_sc[v];
        store_out(d_xy, d_xy_h, o, a_xy[v]);
        store_out(d_rz, d_rz_h, o, a_rz[v]);
        pt_local(w, p, key, o, n_mods, o_pls, o_obj, obj_off);
      }
    }
    __syncwarp(gmask);   // the ordered rows are read back by the other lanes below
    const int b = best_of<Type, kPtLanes>(w, off, d_sc, p, sub, gmask);
    if (sub == 0) {
      best[p] = b;
      if (Type == TC_PT5) w.pls_member[p] = (b >= 0 || w.best3[p] >= 0) ? 1 : 0;
    }
  }
}

// hit -> T5 adjacency (binned hit indices)
// hit -> T5 lists (counting pass, then fill pass); the counting pass also caches each T5's ten
// hits in one row
__global__ void k_h5_count(Ws w, int fill) {
  const int n = w.t5_off[w.V];
  const int64_t S = w.cap.t5_dense;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int k = 0; k < 5; ++k) {
      const int d = w.t5_md[k * S + i];
      const int hs[2] = {w.md_lo[d], w.md_up[d]};
      for (int t = 0; t < 2; ++t) {
        if (!fill) {
          atomicAdd(&w.h5_cnt[hs[t]], 1);
          w.t5_hit[(int64_t)i * 10 + 2 * k + t] = hs[t];
        } else {
          w.h5_idx[w.h5_off[hs[t]] + atomicAdd(&w.h5_cur[hs[t]], 1)] = i;
        }
      }
    }
  }
}

// T5 duplicate removal: T5 a is dropped when another passing T5 shares at least `overlap` of its
// ten hits and ranks lower (chi2_c as float32, then hit tuple). A T5 sharing `overlap` hits with a
// contains at least one of a's first 11 - overlap hits (a misses at most 10 - overlap of them), so
// only those hits' T5 lists are searched (about a dozen T5 in all, typically). kCleanLanes lanes per
// T5: the candidates of the searched lists are spread over them, and any lane's hit drops it.
constexpr int kCleanLanes = 8;

__global__ void k_t5_clean(Ws w, int overlap) {
  const int n = w.t5_off[w.V];
  const int64_t S = w.cap.t5_dense;
  const int n_probe = min(10, max(1, 11 - overlap));
  const int sub = threadIdx.x & (kCleanLanes - 1);
  const unsigned gmask = ((1u << kCleanLanes) - 1u) << ((threadIdx.x & 31) & ~(kCleanLanes - 1));
  const int ngroups = gridDim.x * (blockDim.x / kCleanLanes);
  for (int a = (blockIdx.x * blockDim.x + threadIdx.x) / kCleanLanes; a < n; a += ngroups) {
    // a T5's 10 hits are 40 bytes from an 8-byte aligned base: five independent 8-byte loads
    int ha[10];
    {
      const int2* pa = reinterpret_cast<const int2*>(w.t5_hit + (int64_t)a * 10);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int2 v = pa[k];
        ha[2 * k] = v.x;
        ha[2 * k + 1] = v.y;
      }
    }
    const float ca = w.t5_f[3 * S + a];
    // the probed lists, concatenated: list t covers [beg[t], beg[t] + len[t])
    int beg[10], end_[10];
    int total = 0;
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      beg[t] = t < n_probe ? w.h5_off[ha[t]] : 0;
      const int len = t < n_probe ? w.h5_off[ha[t] + 1] - beg[t] : 0;
      total += len;
      end_[t] = total;
    }
    bool drop = false;
    for (int k = sub; k < total && !drop; k += kCleanLanes) {
      // the list holding entry k (the lists end at end_[0] <= end_[1] <= ...): its start in the
      // concatenation and in h5_idx, carried along the scan (no run-time index into the arrays)
      int start = 0, bt = beg[0];
#pragma unroll
      for (int u = 0; u < 9; ++u)
        if (k >= end_[u]) {
          start = end_[u];
          bt = beg[u + 1];
        }
      const int b = w.h5_idx[bt + (k - start)];
      if (b == a) continue;
      // b's hits loaded together (no chain of dependent loads), then all 100 comparisons
      int hb[10];
      {
        const int2* pb = reinterpret_cast<const int2*>(w.t5_hit + (int64_t)b * 10);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int2 v = pb[k];
          hb[2 * k] = v.x;
          hb[2 * k + 1] = v.y;
        }
      }
      int shared = 0;
#pragma unroll
      for (int kb = 0; kb < 10; ++kb)
#pragma unroll
        for (int u = 0; u < 10; ++u) shared += ha[u] == hb[kb];
      if (shared < overlap) continue;
      const float cb = w.t5_f[3 * S + b];
      if (cb < ca || (cb == ca && key_less(w, TC_T5, b, a))) drop = true;
    }
    drop = __any_sync(gmask, drop);
    if (sub == 0) w.t5_kept[a] = drop ? 0 : 1;
  }
}

// eta-phi grid of 0.02 x (2 pi / 314) cells, wider than dr_min, so any pair closer than dr_min lies
// in the same or adjacent cells
constexpr int kCellsEta = 320;
constexpr int kCellsPhi = 314;
constexpr float kCellEtaMin = -3.2f;
constexpr float kCellEtaW = 0.02f;

__device__ __forceinline__ int cell_eta(float eta) {
  int i = (int)floorf((eta - kCellEtaMin) / kCellEtaW);
  return min(max(i, 0), kCellsEta - 1);
}
__device__ __forceinline__ int cell_phi(float phi) {
  float p = fmodf(phi, 6.2831853f);
  if (p < 0.f) p += 6.2831853f;
  int i = (int)floorf(p * (kCellsPhi / 6.2831853f));
  return min(max(i, 0), kCellsPhi - 1);
}

// dR < dr_min decided in float64 on the stored float32 eta / phi, with explicitly rounded
// operations (the same IEEE sequence as any evaluation of the definition)
__device__ __forceinline__ bool dr_close(double dr2, float ea, float pa, float eb, float pb) {
  const double de = __dsub_rn((double)ea, (double)eb);
  double dp = __dsub_rn((double)pa, (double)pb);
  if (dp > kPiD) dp = __dsub_rn(dp, kTwoPiD);
  if (dp <= -kPiD) dp = __dadd_rn(dp, kTwoPiD);
  const double d2 = __dadd_rn(__dmul_rn(de, de), __dmul_rn(dp, dp));
  return d2 < dr2;
}

__device__ __forceinline__ void item_of(const Ws& w, int code, float& eta, float& phi, int& type, int& idx) {
  type = code >> 29;
  idx = code & ((1 << 29) - 1);
  if (type == TC_T5) {
    const int64_t S = w.cap.t5_dense;
    eta = w.t5_f[5 * S + idx];
    phi = w.t5_f[6 * S + idx];
  } else {
    eta = w.pls[idx].eta;
    phi = w.pls[idx].phi;
  }
}

// pass 0: count, pass 1: fill; items: accepted pT5 seeds (type 0), pT3 candidates (1), kept T5 (2)
__global__ void k_grid_items(Ws w, Geo g, int fill) {
  const int n_t5 = w.t5_off[w.V];
  const int P = w.n_pls();
  const int total = P + n_t5;
  const int NC = kCellsEta * kCellsPhi;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    int code, e;
    if (k < P) {
      const int p = k;
      if (w.best5[p] >= 0) code = (TC_PT5 << 29) | p;
      else if (w.best3[p] >= 0) code = (TC_PT3 << 29) | p;
      else continue;
      e = w.pls_ev[p];
    } else {
      const int i = k - P;
      if (!w.t5_kept[i]) continue;
      code = (TC_T5 << 29) | i;
      e = w.md_vm[w.t5_md[i]] / g.n_mods;
    }
    float eta, phi;
    int type, idx;
    item_of(w, code, eta, phi, type, idx);
    const int cell = e * NC + cell_eta(eta) * kCellsPhi + cell_phi(phi);
    if (!fill) atomicAdd(&w.cell_cnt[cell], 1);
    else w.cell_item[w.cell_off[cell] + atomicAdd(&w.cell_cur[cell], 1)] = code;
  }
}

// is (eta, phi) of event e within dr_min of an item accepted so far? mask: which item types count
__device__ bool near_accepted(const Ws& w, double dr2, int e, float eta, float phi, int mask) {
  const int NC = kCellsEta * kCellsPhi;
  const int ce = cell_eta(eta), cp = cell_phi(phi);
  for (int de = -1; de <= 1; ++de) {
    const int ie = ce + de;
    if (ie < 0 || ie >= kCellsEta) continue;
    for (int dp = -1; dp <= 1; ++dp) {
      const int ip = (cp + dp + kCellsPhi) % kCellsPhi;
      const int cell = e * NC + ie * kCellsPhi + ip;
      for (int k = w.cell_off[cell]; k < w.cell_off[cell + 1]; ++k) {
        float eb, pb;
        int type, idx;
        item_of(w, w.cell_item[k], eb, pb, type, idx);
        if (!((mask >> type) & 1)) continue;
        if (type == TC_PT3 && !w.acc3[idx]) continue;
        if (type == TC_T5 && !w.acc5t[idx]) continue;
        if (dr_close(dr2, eta, phi, eb, pb)) return true;
      }
    }
  }
  return false;
}

__global__ void k_clean_pt3(Ws w, double dr2) {
  const int P = w.n_pls();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    uint8_t acc = 0;
    if (w.best5[p] < 0 && w.best3[p] >= 0) {
      const int e = w.pls_ev[p];
      acc = near_accepted(w, dr2, e, w.pls[p].eta, w.pls[p].phi, 1 << TC_PT5) ? 0 : 1;
    }
    w.acc3[p] = acc;
  }
}

__global__ void k_clean_t5(Ws w, Geo g, double dr2) {
  const int n = w.t5_off[w.V];
  const int64_t S = w.cap.t5_dense;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint8_t acc = 0;
    if (w.t5_kept[i]) {
      const int e = w.md_vm[w.t5_md[i]] / g.n_mods;
      acc = near_accepted(w, dr2, e, w.t5_f[5 * S + i], w.t5_f[6 * S + i], (1 << TC_PT5) | (1 << TC_PT3)) ? 0 : 1;
    }
    w.acc5t[i] = acc;
  }
}

__global__ void k_clean_pls(Ws w, double dr2) {
  const int P = w.n_pls();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    uint8_t acc = 0;
    if (!w.pls_member[p]) {
      const int e = w.pls_ev[p];
      acc = near_accepted(w, dr2, e, w.pls[p].eta, w.pls[p].phi,
                          (1 << TC_PT5) | (1 << TC_PT3) | (1 << TC_T5)) ? 0 : 1;
    }
    w.accl[p] = acc;
  }
}

// Per-event assembly: one block per event collects the accepted candidates, sorts them by
// (type, sorted hit tuple) and writes the output rows. The sort is a bitonic sort of 64-bit keys
// (type, smallest hit) in shared memory, followed by an exact ordering of equal-key runs.
constexpr int kTcSortMax = 8192;

// order-preserving 64-bit prefix of (type, sorted hit tuple): the type, then the first two hits
// saturated at 2^30 - 1 (hit ids are non-negative); equal prefixes are ordered on the full tuple
__device__ __forceinline__ unsigned long long tc_sort_key(int type, int h0, int h1) {
  const unsigned long long m = (1ull << 30) - 1;
  const unsigned long long a = (unsigned long long)min((unsigned)h0, (unsigned)m);
  const unsigned long long b = (unsigned long long)min((unsigned)h1, (unsigned)m);
  return ((unsigned long long)(unsigned)type << 60) | (a << 30) | b;
}

__device__ __forceinline__ int hit_key_cmp(const int* a, const int* b) {
  for (int k = 0; k < 14; ++k)
    if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
  return 0;
}

// accepted candidates of each event and type (block per event)
__global__ void k_tc_count(Ws w, Geo g) {
  __shared__ int ty[4];
  const int e = blockIdx.x;
  if (threadIdx.x < 4) ty[threadIdx.x] = 0;
  __syncthreads();
  const int p0 = w.ev_pls_off[e], p1 = w.ev_pls_off[e + 1];
  const int t0 = w.t5_off[e * g.n_mods], t1 = w.t5_off[(e + 1) * g.n_mods];
  int c[4] = {0, 0, 0, 0};
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    c[TC_PT5] += w.best5[p] >= 0;
    c[TC_PT3] += w.acc3[p];
    c[TC_PLS] += w.accl[p];
  }
  for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x) c[TC_T5] += w.acc5t[i];
  for (int t = 0; t < 4; ++t)
    if (c[t]) atomicAdd(&ty[t], c[t]);
  __syncthreads();
  if (threadIdx.x < 4) w.ev_stat[e * kEvWords + 7 + threadIdx.x] = ty[threadIdx.x];
  if (threadIdx.x == 0) w.tc_cnt[e] = ty[0] + ty[1] + ty[2] + ty[3];
}

// Assembly of the track candidates of each (event, type), ordered by their sorted hit tuple, in four
// launches: collect the accepted candidates, build their keys (all candidates in parallel), sort
// the keys (bitonic sort of 64-bit prefix keys in shared memory, then an exact ordering of
// equal-prefix runs), write the rows (in parallel). Rows of type t start after the event's rows of
// the types before it.
__device__ __forceinline__ int tc_region(const Ws& w, const Geo& g, int e, int type) {
  int before = 0;
  for (int t = 0; t < type; ++t) before += w.ev_stat[e * kEvWords + 7 + t];
  return w.ev_pls_off[e] + w.t5_off[e * g.n_mods] + before;
}

// (1) a block per (event, type) collects the accepted candidates' codes (type << 29 | index)
__global__ void k_tc_collect(Ws w, Geo g) {
  __shared__ int n_sh;
  const int e = blockIdx.x, type = blockIdx.y;
  if (e >= w.E) return;
  const int p0 = w.ev_pls_off[e], p1 = w.ev_pls_off[e + 1];
  const int t0 = w.t5_off[e * g.n_mods], t1 = w.t5_off[(e + 1) * g.n_mods];
  int* code = w.tc_code + tc_region(w, g, e, type);
  if (threadIdx.x == 0) n_sh = 0;
  __syncthreads();
  if (type == TC_T5) {
    for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x)
      if (w.acc5t[i]) code[atomicAdd(&n_sh, 1)] = (TC_T5 << 29) | i;
  } else {
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const bool take = type == TC_PT5 ? w.best5[p] >= 0 : (type == TC_PT3 ? w.acc3[p] != 0 : w.accl[p] != 0);
      if (take) code[atomicAdd(&n_sh, 1)] = (type << 29) | p;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) w.tc_n[e * 4 + type] = n_sh;
}

// (2) the sorted hit tuple (padded with INT_MAX) and 64-bit prefix key of every collected candidate;
// blockIdx.y = event * 4 + type, the x blocks share its candidates
__global__ void k_tc_keys(Ws w, Geo g) {
  const int e = blockIdx.y >> 2, type = blockIdx.y & 3;
  if (e >= w.E) return;
  const int n = w.tc_n[blockIdx.y];
  const int region = tc_region(w, g, e, type);
  const int* code = w.tc_code + region;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int idx = code[k] & ((1 << 29) - 1);
    int h[14];
    const int obj = (type == TC_PT5) ? w.best5[idx] : (type == TC_PT3 ? w.best3[idx] : idx);
    const int nh = code_hits(w, type, obj, h);
    sort_small(h, nh);
    int* hk = w.tc_hit_key + (int64_t)(region + k) * 14;
    for (int t = 0; t < 14; ++t) hk[t] = t < nh ? h[t] : 0x7fffffff;
    w.tc_key[region + k] = tc_sort_key(type, h[0], nh > 1 ? h[1] : 0x7fffffff);
  }
}

// (3) a block per (event, type) sorts the keys (bitonic in shared memory; equal prefixes ordered on
// the full tuples) and records each row's source: tc_perm[region + rank] = collected index
__global__ void __launch_bounds__(1024) k_tc_sort(Ws w, Geo g) {
  extern __shared__ unsigned char smem_raw[];
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(smem_raw);
  int* sidx = reinterpret_cast<int*>(skey + kTcSortMax);
  const int e = blockIdx.x, type = blockIdx.y;
  if (e >= w.E) return;
  const int n = w.tc_n[e * 4 + type];
  if (n == 0) return;
  const int region = tc_region(w, g, e, type);
  const unsigned long long* key = w.tc_key + region;
  const int* hk = w.tc_hit_key + (int64_t)region * 14;
  int* perm = w.tc_perm + region;
  if (n > kTcSortMax) {   // ranks counted directly, equal tuples ordered by collected index as below
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      int rank = 0;
      for (int j = 0; j < n; ++j) {
        const int cmp = hit_key_cmp(hk + (int64_t)j * 14, hk + (int64_t)k * 14);
        rank += cmp < 0 || (cmp == 0 && j < k);
      }
      perm[rank] = k;
    }
    return;
  }
  int m = 1;
  while (m < n) m <<= 1;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    skey[k] = k < n ? key[k] : ~0ull;
    sidx[k] = k < n ? k : 0x7fffffff;
  }
  __syncthreads();
  // a stage of stride <= 32 exchanges elements inside one warp's 64-element blocks (pair t touches
  // [64 (t / 32), 64 (t / 32) + 64)), so between two such stages a warp barrier suffices; a wider
  // stage, before or after, needs the block
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < m / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long a = skey[lo], b = skey[hi];
        const bool gt = (a > b) || (a == b && sidx[lo] > sidx[hi]);
        if (gt == up) {
          skey[lo] = b; skey[hi] = a;
          const int ti = sidx[lo]; sidx[lo] = sidx[hi]; sidx[hi] = ti;
        }
      }
      const int next = stride > 1 ? stride >> 1 : size;   // the next stage's stride
      if (stride <= 32 && next <= 32) __syncwarp();
      else __syncthreads();
    }
  }
  __syncthreads();
  // exact order inside runs of equal prefix keys (rare, short: insertion sort on full tuples by the
  // thread at the start of each run)
  for (int r0 = threadIdx.x; r0 < n; r0 += blockDim.x) {
    if ((r0 == 0 || skey[r0 - 1] != skey[r0]) && r0 + 1 < n && skey[r0 + 1] == skey[r0]) {
      int r1 = r0 + 1;
      while (r1 < n && skey[r1] == skey[r0]) ++r1;
      for (int i = r0 + 1; i < r1; ++i) {
        const int v = sidx[i];
        int j = i - 1;
        while (j >= r0 && hit_key_cmp(hk + (int64_t)sidx[j] * 14, hk + (int64_t)v * 14) > 0) {
          sidx[j + 1] = sidx[j];
          --j;
        }
        sidx[j + 1] = v;
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) perm[k] = sidx[k];
}

// (4) the rows in order: blockIdx.y = event * 4 + type, the x blocks share its rows
__global__ void k_tc_write(Ws w, Geo g) {
  const int e = blockIdx.y >> 2, type = blockIdx.y & 3;
  if (e >= w.E) return;
  const int n = w.tc_n[blockIdx.y];
  const int region = tc_region(w, g, e, type);
  const int p0 = w.ev_pls_off[e];
  const int t0 = w.t5_off[e * g.n_mods];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int src = w.tc_perm[region + r];
    const int idx = w.tc_code[region + src] & ((1 << 29) - 1);
    const int row = region + r;
    int h[14];
    int obj, nh;
    float pt, eta, phi;
    if (type == TC_PT5 || type == TC_PT3) {
      const int dense = type == TC_PT5 ? w.best5[idx] : w.best3[idx];
      nh = code_hits(w, type, dense, h);
      obj = dense - (type == TC_PT5 ? w.pt5_off[p0] : w.pt3_off[p0]);
      pt = w.pls[idx].pt; eta = w.pls[idx].eta; phi = w.pls[idx].phi;
    } else if (type == TC_T5) {
      nh = code_hits(w, type, idx, h);
      obj = idx - t0;
      const int64_t S = w.cap.t5_dense;
      pt = w.t5_f[7 * S + idx]; eta = w.t5_f[5 * S + idx]; phi = w.t5_f[6 * S + idx];
    } else {
      nh = code_hits(w, type, idx, h);
      obj = idx - p0;
      pt = w.pls[idx].pt; eta = w.pls[idx].eta; phi = w.pls[idx].phi;
    }
    w.tc_type[row] = type;
    w.tc_obj[row] = obj;
    for (int t = 0; t < 14; ++t) w.tc_hits[(int64_t)row * 14 + t] = t < nh ? h[t] : -1;
    w.tc_pt[row] = pt;
    w.tc_eta[row] = eta;
    w.tc_phi[row] = phi;
  }
}

// track candidates of all events packed densely (event e's rows start at tcd_off[e]), so that the
// whole batch's candidates reach the host in one transfer per array
__global__ void k_tc_dense(Ws w, Geo g) {
  // blockIdx.y: event; blocks along x share its rows
  const int e = blockIdx.y;
  if (e >= w.E) return;
  const int n = w.tc_cnt[e];
  const int src0 = w.ev_pls_off[e] + w.t5_off[e * g.n_mods];
  const int dst0 = w.tcd_off[e];
  const int stride = gridDim.x * blockDim.x;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int a = src0 + k, b = dst0 + k;
    w.tcd_type[b] = w.tc_type[a];
    w.tcd_obj[b] = w.tc_obj[a];
    w.tcd_pt[b] = w.tc_pt[a];
    w.tcd_eta[b] = w.tc_eta[a];
    w.tcd_phi[b] = w.tc_phi[a];
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 14 * n; k += stride)
    w.tcd_hits[(int64_t)dst0 * 14 + k] = w.tc_hits[(int64_t)src0 * 14 + k];
}

// ---------------------------------------------------------------------------------------------
// Track extensions (Sec. 2.5.1). A pT5, pT3 or T5 track candidate (MDs m_1..m_K inner to outer) is
// extended by the T3 that continues it outward: a T3 starting at m_K adds its two other MDs, one
// starting at m_(K-1) whose second MD is m_K adds its third. A candidate T3 must agree in curvature
// with the track candidate (the T5 compatibility: |k_T3 - k_TC| <= c_rel max(k) + c_abs, k_TC the
// seed's k / pT or the T5 fit's |kappa|) and the extended track's n anchors must lie on the T5's
// r-z line in arc length with the T5 cut per degree of freedom, chi2_rz <= chi2_t5_rz (n - 2) / 3.
// Karimaki's circle through the n anchors gives the arc lengths and a circle chi2 that ranks the
// candidates (it is not cut on). Decided in double-float, like the T5 selection; of several passing
// T3 the one with the lowest (chi2_c + chi2_rz as float32, sorted hit tuple) is taken. The rows'
// candidates are queued by anchor count (A), fitted one per thread (B), and chosen per row (C, with
// the rare rows whose candidates did not all fit the queues finished by D).
// ---------------------------------------------------------------------------------------------
struct ExtCuts {
  ff rz[8];   // r-z chi2 bounds for n anchors (n = 4..7)
};

// the fit of the n anchors of md[0, n) (4 <= n <= kExtMaxAnchors): Karimaki's circle and its chi2,
// and the r-z line in arc length with its cut; one copy of the code for every anchor count
constexpr int kExtMaxAnchors = 7;

__device__ __forceinline__ bool ext_fit(const Ws& w, const Cst<ff>& c, const int* md, int n, ff cut_rz, ff& chi2c,
                                        ff& chi2rz) {
  ff x[kExtMaxAnchors], y[kExtMaxAnchors], z[kExtMaxAnchors], r[kExtMaxAnchors];
  bool ec[kExtMaxAnchors];
#pragma unroll
  for (int a = 0; a < kExtMaxAnchors; ++a) {
    if (a < n) {
      const float4 p = w.md_xyzr[md[a]];
      x[a] = ff(p.x);
      y[a] = ff(p.y);
      z[a] = ff(p.z);
      r[a] = ff_fast_two_sum(p.w, w.md_rlo[md[a]]);
      ec[a] = w.md_ec[md[a]] != 0;
    }
  }
  ff rho, phi, d, sp, cp;
  karimaki_n<ff, kExtMaxAnchors>(x, y, n, rho, phi, d, sp, cp);
  chi2c = circle_chi2_n<ff, kExtMaxAnchors>(x, y, n, rho, sp, cp, d, c.sigma_rphi);
  ff slope;
  if (!rz_fit_n<ff, kExtMaxAnchors>(c, m_abs(rho), r, z, ec, n, chi2rz, slope)) return false;
  AccFF acc;
  acc.cut(cut_rz, chi2rz);
  return !acc.fail;
}

__device__ __forceinline__ void t3_sorted_hits(const Ws& w, int t3, int* h) {
  int n = 0;
  const int md[3] = {w.t3_md0[t3], w.t3_md1[t3], w.t3_md2[t3]};
  for (int k = 0; k < 3; ++k) n += md_hits(w, md[k], h + n);
  sort_small(h, 6);
}

// the MDs of a dense track-candidate row (inner to outer) and its curvature; K = 0 for pLS rows
__device__ __forceinline__ int ext_row(const Ws& w, const Geo& g, const Cst<ff>& c, int e, int row, int* md,
                                       ff& ktc) {
  const int type = w.tcd_type[row], obj = w.tcd_obj[row];
  const int p0 = w.ev_pls_off[e];
  const int64_t S5 = w.cap.t5_dense;
  if (type == TC_PT5) {
    const int gi = obj + w.pt5_off[p0];
    const int t5 = w.pt5_obj[gi];
    for (int a = 0; a < 5; ++a) md[a] = w.t5_md[a * S5 + t5];
    ktc = c.k / ff(w.pls[w.pt5_pls[gi]].pt);
    return 5;
  }
  if (type == TC_PT3) {
    const int gi = obj + w.pt3_off[p0];
    const int t3 = w.pt3_obj[gi];
    md[0] = w.t3_md0[t3]; md[1] = w.t3_md1[t3]; md[2] = w.t3_md2[t3];
    ktc = c.k / ff(w.pls[w.pt3_pls[gi]].pt);
    return 3;
  }
  if (type == TC_T5) {
    const int t5 = obj + w.t5_off[e * g.n_mods];
    for (int a = 0; a < 5; ++a) md[a] = w.t5_md[a * S5 + t5];
    ktc = m_abs(ff(w.t5_f[2 * S5 + t5]));
    return 5;
  }
  return 0;
}

// the candidate T3 of a row, in a fixed order: those starting at m_K (overlap 1), then those
// starting at m_(K-1) whose second MD is m_K (overlap 2), each in dense T3 order. Calls f(t3,
// overlap) for each that agrees with the row's curvature.
template <class F>
__device__ __forceinline__ void ext_candidates(const Ws& w, const Cst<ff>& c, const int* md, int K, ff ktc, F f) {
  const int n_t3 = w.t3_off[w.V];
  for (int overlap = 1; overlap <= 2 && K > 0; ++overlap) {
    const int first = md[K - overlap];
    const int j0 = min(w.t3md_off[first], n_t3), j1 = min(w.t3md_off[first + 1], n_t3);
    for (int d = j0; d < j1; ++d) {
      if (overlap == 2 && w.t3_md1[d] != md[K - 1]) continue;
      const float R3 = w.t3_R[d];
      const ff kt3 = isinf(R3) ? ff(0.0f) : ff(1.0f) / ff(R3);
      AccFF acc;
      acc.cut(c.c_rel * m_max(kt3, ktc) + c.c_abs, m_abs(kt3 - ktc));
      if (!acc.fail) f(d, overlap);
    }
  }
}

// the fit of one candidate with n = K + 3 - overlap anchors; result (score, chi2_c, chi2_rz, passed)
__device__ __forceinline__ float4 ext_eval(const Ws& w, const Cst<ff>& c, const ExtCuts& xc, const int* md, int K,
                                           int t3, int overlap) {
  int all[kExtMaxAnchors];
#pragma unroll
  for (int a = 0; a < 5; ++a)
    if (a < K) all[a] = md[a];
  const int add1 = w.t3_md1[t3], add2 = w.t3_md2[t3];
  // the added MDs follow the row's K (3 or 5), with the indices known at compile time
  if (K == 3) {
    if (overlap == 1) { all[3] = add1; all[4] = add2; } else { all[3] = add2; }
  } else {
    if (overlap == 1) { all[5] = add1; all[6] = add2; } else { all[5] = add2; }
  }
  const int n = K + 3 - overlap;
  ff cut = xc.rz[4];   // the bound for n anchors, selected without a run-time index into the parameter
#pragma unroll
  for (int k = 5; k <= kExtMaxAnchors; ++k)
    if (n == k) cut = xc.rz[k];
  ff chi2c, chi2rz;
  const bool ok = ext_fit(w, c, all, n, cut, chi2c, chi2rz);
  return make_float4((float)(chi2c + chi2rz), (float)chi2c, (float)chi2rz, ok ? 1.f : 0.f);
}

// a queued candidate: dense T3 index (< 2^30) and overlap (1 or 2) in one word
__device__ __forceinline__ int ext_pack(int t3, int overlap) { return (int)((unsigned)t3 | ((unsigned)overlap << 30)); }
__device__ __forceinline__ int ext_t3(int v) { return (int)((unsigned)v & ((1u << 30) - 1u)); }
__device__ __forceinline__ int ext_overlap(int v) { return (int)((unsigned)v >> 30); }

// (A) each row's candidates that agree in curvature go to the queue region of their anchor count;
// the row keeps up to kExtRefs references and the total. A row's candidates fall in two regions
// (overlap 1: K + 2 anchors, overlap 2: K + 1). The rows of a warp first count theirs, reserve their
// queue space with one atomic per warp and region (the regions' four counters would otherwise take
// one atomic per candidate), then list them again in the same order and write them.
__global__ void k_ext_cand(Ws w, Geo g, Cst<ff> c) {
  const int nrow = w.tcd_off[w.E];
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int row0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); row0 < nrow; row0 += stride) {
    const int row = row0 + lane;
    int md[5];
    ff ktc;
    int K = 0;
    if (row < nrow) K = ext_row(w, g, c, find_seg(w.tcd_off, w.E, row), row, md, ktc);
    // pass 1: referenced candidates per overlap (the first kExtRefs in listing order) and the total
    int n = 0, n1 = 0, n2 = 0;
    ext_candidates(w, c, md, K, ktc, [&](int, int overlap) {
      if (n < kExtRefs) {
        if (overlap == 1) ++n1; else ++n2;
      }
      ++n;
    });
    // one reservation per warp and region: the region of overlap o is (K + 3 - o) - 4, so K - 2 for
    // overlap 1 and K - 3 for overlap 2
    int pos1 = 0, pos2 = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int mine = (K > 0 && K - 2 == r ? n1 : 0) + (K > 0 && K - 3 == r ? n2 : 0);
      int incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      int base = 0;
      if (lane == 31 && total > 0) base = atomicAdd(&w.ext_qn[r], total);
      base = __shfl_sync(0xffffffffu, base, 31) + incl - mine;
      if (K > 0 && K - 2 == r) pos1 = base;   // overlap 1 takes [base, base + n1)
      if (K > 0 && K - 3 == r) pos2 = base;   // overlap 2 takes [base, base + n2)
    }
    // pass 2: the same candidates in the same order, written to the reserved positions
    int k = 0;
    ext_candidates(w, c, md, K, ktc, [&](int d, int overlap) {
      if (k < kExtRefs) {   // candidates beyond the row's references are evaluated by the slow pass
        const int reg = K + 3 - overlap - 4;
        const int pos = overlap == 1 ? pos1++ : pos2++;
        if (pos < w.ext_qcap) {
          w.ext_q[reg * w.ext_qcap + pos] = make_int2(row, ext_pack(d, overlap));
          w.ext_ref[(int64_t)row * kExtRefs + k] = (reg << 28) | pos;
        } else {
          w.ext_ref[(int64_t)row * kExtRefs + k] = -1;   // not queued: evaluated by the slow pass
        }
      }
      ++k;
    });
    if (row < nrow) w.ext_cnt[row] = n;
  }
}

// (B) the fits, one thread per queued candidate; blockIdx.y selects the anchor count (4 + y), so a
// warp's threads take the same branches through the one fit code and the four counts run side by side
__global__ void __launch_bounds__(128, 4) k_ext_fit(Ws w, Geo g, Cst<ff> c, ExtCuts xc) {
  const int reg = blockIdx.y;
  const int n = (int)min((int64_t)w.ext_qn[reg], w.ext_qcap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 q = w.ext_q[reg * w.ext_qcap + k];
    const int row = q.x, d = ext_t3(q.y), overlap = ext_overlap(q.y);
    const int e = find_seg(w.tcd_off, w.E, row);
    int md[5];
    ff ktc;
    const int K = ext_row(w, g, c, e, row, md, ktc);
    w.ext_res[reg * w.ext_qcap + k] = ext_eval(w, c, xc, md, K, d, overlap);
  }
}

// the best passing candidate of a row so far: by (score as float32, sorted hit tuple of the T3)
struct ExtBest {
  int t3 = -1, n_add = 0;
  float sc = 0.f, chi2c = 0.f, chi2rz = 0.f;
};

__device__ __forceinline__ void ext_consider(const Ws& w, ExtBest& b, int d, int overlap, float4 r) {
  if (r.w == 0.f) return;
  bool better = b.t3 < 0 || r.x < b.sc;
  if (!better && r.x == b.sc) {   // equal scores (rare): the sorted hit tuples decide
    int key[6], bkey[6];
    t3_sorted_hits(w, d, key);
    t3_sorted_hits(w, b.t3, bkey);
    for (int t = 0; t < 6; ++t)
      if (key[t] != bkey[t]) { better = key[t] < bkey[t]; break; }
  }
  if (better) {
    b.t3 = d; b.n_add = 3 - overlap; b.sc = r.x; b.chi2c = r.y; b.chi2rz = r.z;
  }
}

// the row's outputs (T3 index within its event, added MDs, their hits, the chi2 of the fit); the
// extended rows are counted per event, aggregated over a thread's consecutive rows of one event
__device__ __forceinline__ void ext_write(const Ws& w, const Geo& g, int e, int row, const ExtBest& b,
                                          int& e_acc, int& n_acc) {
  int h[4] = {-1, -1, -1, -1};
  if (b.t3 >= 0) {
    const int add[2] = {w.t3_md1[b.t3], w.t3_md2[b.t3]};
    int m = 0;
    for (int a = 2 - b.n_add; a < 2; ++a) m += md_hits(w, add[a], h + m);
    if (e != e_acc) {
      if (n_acc) atomicAdd(&w.ev_stat[e_acc * kEvWords + kEvExt], n_acc);
      e_acc = e;
      n_acc = 0;
    }
    ++n_acc;
  }
  w.tcd_ext_t3[row] = b.t3 >= 0 ? b.t3 - w.t3_off[e * g.n_mods] : -1;
  w.tcd_ext_n[row] = b.n_add;
  for (int t = 0; t < 4; ++t) w.tcd_ext_hits[(int64_t)row * 4 + t] = h[t];
  w.tcd_ext_c[row] = b.t3 >= 0 ? b.chi2c : 0.f;
  w.tcd_ext_rz[row] = b.t3 >= 0 ? b.chi2rz : 0.f;
}

// the queued candidates of a row; false when some candidate was not queued (the row is then slow)
__device__ __forceinline__ bool ext_queued(const Ws& w, int row, ExtBest& b) {
  const int ncand = w.ext_cnt[row];
  bool all = ncand <= kExtRefs;
  for (int k = 0; k < min(ncand, kExtRefs); ++k) {
    const int ref = w.ext_ref[(int64_t)row * kExtRefs + k];
    if (ref < 0) { all = false; continue; }
    const int reg = ref >> 28, pos = ref & ((1 << 28) - 1);
    const int2 q = w.ext_q[reg * w.ext_qcap + pos];
    ext_consider(w, b, ext_t3(q.y), ext_overlap(q.y), w.ext_res[reg * w.ext_qcap + pos]);
  }
  return all;
}

// (C) per row, the best passing queued candidate. Rows with candidates beyond their references or
// the queues are handed to (D).
__global__ void k_ext_select(Ws w, Geo g) {
  const int nrow = w.tcd_off[w.E];
  int n_acc = 0, e_acc = -1;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nrow; row += gridDim.x * blockDim.x) {
    ExtBest b;
    if (!ext_queued(w, row, b)) {
      const int k = atomicAdd(&w.ext_qn[4], 1);
      if (k < w.tc_capacity) w.ext_slow[k] = row;
      continue;
    }
    ext_write(w, g, find_seg(w.tcd_off, w.E, row), row, b, e_acc, n_acc);
  }
  if (n_acc) atomicAdd(&w.ev_stat[e_acc * kEvWords + kEvExt], n_acc);
}

// (D) the rare slow rows: their queued candidates, and the others fitted here
__global__ void k_ext_slow(Ws w, Geo g, Cst<ff> c, ExtCuts xc) {
  const int n = (int)min((int64_t)w.ext_qn[4], w.tc_capacity);
  int n_acc = 0, e_acc = -1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int row = w.ext_slow[i];
    const int e = find_seg(w.tcd_off, w.E, row);
    ExtBest b;
    ext_queued(w, row, b);
    int md[5];
    ff ktc;
    const int K = ext_row(w, g, c, e, row, md, ktc);
    int k = 0;
    ext_candidates(w, c, md, K, ktc, [&](int d, int overlap) {
      const int ref = k < kExtRefs ? w.ext_ref[(int64_t)row * kExtRefs + k] : -1;
      ++k;
      if (ref >= 0) return;   // already considered
      ext_consider(w, b, d, overlap, ext_eval(w, c, xc, md, K, d, overlap));
    });
    ext_write(w, g, e, row, b, e_acc, n_acc);
  }
  if (n_acc) atomicAdd(&w.ev_stat[e_acc * kEvWords + kEvExt], n_acc);
}

}  // namespace


void run_pixel(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  k_pls_prep<<<grid_for(w.P, 256), 256, 0, L.stream>>>(w, g, c.f, c.x);
  LST_LAUNCH(L);
  const int threads = 32 * L.warps_px;
  // at most the resident blocks: the warps divide the seeds statically, so a second wave of blocks
  // would only start as the first one drains
  auto pt_blocks = [&](int bps) { return grid_for((int64_t)w.P * 32, threads, L.n_sm * (bps > 0 ? bps : 16)); };
  ObjAnc om3{w.t3_anc, w.t3_anc_rlo, w.t3_ecm, w.cap.t3_dense};
  ObjAnc om5{w.t5_anc, w.t5_anc_rlo, w.t5_ecm, w.cap.t5_dense};
  if (g.n_pix_bins > 0) {
    k_obj_box<<<grid_for((int64_t)w.V * 2 * kBoxLanes, 256), 256, 0, L.stream>>>(w, g);
    *L.launches += 1;
    KT_BEGIN(L, K_PT3_PRE);
  k_pt_pre<3><<<pt_blocks(L.pt3_blocks_per_sm), threads, 0, L.stream>>>(w, g, c.f, w.t3_off, w.box3, om3, w.q_p3, ST_Q_PT3, w.cap.q_p3,
                                                   c.f.chi2_pt3_xy, c.f.chi2_pt3_rz);
  KT_END(L, K_PT3_PRE);
    LST_LAUNCH(L);
    KT_BEGIN(L, K_PT5_PRE);
  k_pt_pre<5><<<pt_blocks(L.pt5_blocks_per_sm), threads, 0, L.stream>>>(w, g, c.f, w.t5_off, w.box5, om5, w.q_p5, ST_Q_PT5, w.cap.q_p5,
                                                   c.f.chi2_pt5_xy, c.f.chi2_pt5_rz);
  KT_END(L, K_PT5_PRE);
    LST_LAUNCH(L);
  }
  KT_BEGIN(L, K_PT3_DECIDE);
  k_pt_decide<3><<<grid_for(w.cap.q_p3, 128, 152 * 8), 128, 0, L.stream>>>(
      w, c.x, om3, w.q_p3, ST_Q_PT3, w.cap.q_p3, c.x.chi2_pt3_xy, c.x.chi2_pt3_rz, w.p3a_pls, w.p3a_obj,
      w.p3a_xy, w.p3a_rz, w.p3a_sc, ST_N_PT3, w.cap.p3_slots, w.p3_cnt);
  KT_END(L, K_PT3_DECIDE);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_PT5_DECIDE);
  k_pt_decide<5><<<grid_for(w.cap.q_p5, 128, 152 * 8), 128, 0, L.stream>>>(
      w, c.x, om5, w.q_p5, ST_Q_PT5, w.cap.q_p5, c.x.chi2_pt5_xy, c.x.chi2_pt5_rz, w.p5a_pls, w.p5a_obj,
      w.p5a_xy, w.p5a_rz, w.p5a_sc, ST_N_PT5, w.cap.p5_slots, w.p5_cnt);
  KT_END(L, K_PT5_DECIDE);
  LST_LAUNCH(L);
  scan_exclusive(w.p3_cnt, w.pt3_off, w.P, w.scan_tmp, L);
  scan_exclusive(w.p5_cnt, w.pt5_off, w.P, w.scan_tmp, L);
  k_pt_group<<<grid_for(w.cap.p3_slots, 256), 256, 0, L.stream>>>(w, ST_N_PT3, w.cap.p3_slots, w.p3a_pls,
                                                                   w.p3a_obj, w.pt3_off, w.p3_cur, w.grp_tmp);
  k_pt_order<TC_PT3><<<grid_for((int64_t)w.P * pt_lanes<TC_PT3>(), 32 * kPtOrderWarps), 32 * kPtOrderWarps, 0, L.stream>>>(
      w, w.pt3_off, w.grp_tmp, w.p3a_pls, w.p3a_obj, w.p3a_xy, w.p3a_rz, w.p3a_sc, w.pt3_pls, w.pt3_obj,
      w.pt3_xy, w.pt3_rz, w.pt3_sc, w.best3, w.o_pt3_pls, w.o_pt3_obj, w.t3_off, w.pt3_xy_h, w.pt3_rz_h);
  k_pt_group<<<grid_for(w.cap.p5_slots, 256), 256, 0, L.stream>>>(w, ST_N_PT5, w.cap.p5_slots, w.p5a_pls,
                                                                   w.p5a_obj, w.pt5_off, w.p5_cur, w.grp_tmp);
  k_pt_order<TC_PT5><<<grid_for((int64_t)w.P * pt_lanes<TC_PT5>(), 32 * kPtOrderWarps), 32 * kPtOrderWarps, 0, L.stream>>>(
      w, w.pt5_off, w.grp_tmp, w.p5a_pls, w.p5a_obj, w.p5a_xy, w.p5a_rz, w.p5a_sc, w.pt5_pls, w.pt5_obj,
      w.pt5_xy, w.pt5_rz, w.pt5_sc, w.best5, w.o_pt5_pls, w.o_pt5_obj, w.t5_off, w.pt5_xy_h, w.pt5_rz_h);
  *L.launches += 4;
}

void run_tc(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  const double dr2 = c.d.dr_min * c.d.dr_min;
  k_h5_count<<<grid_for(w.cap.t5_dense, 256), 256, 0, L.stream>>>(w, 0);
  *L.launches += 1;
  scan_exclusive(w.h5_cnt, w.h5_off, w.cap.H, w.scan_tmp, L);
  k_h5_count<<<grid_for(w.cap.t5_dense, 256), 256, 0, L.stream>>>(w, 1);
  KT_BEGIN(L, K_TC_CLEAN);
  k_t5_clean<<<grid_for((int64_t)w.cap.t5_dense * kCleanLanes, 256, 152 * 32), 256, 0, L.stream>>>(
      w, c.d.t5_overlap_hits);
  KT_END(L, K_TC_CLEAN);
  k_grid_items<<<grid_for(w.P + w.cap.t5_dense, 256), 256, 0, L.stream>>>(w, g, 0);
  *L.launches += 3;
  scan_exclusive(w.cell_cnt, w.cell_off, (int64_t)w.E * w.n_cells, w.scan_tmp, L);
  k_grid_items<<<grid_for(w.P + w.cap.t5_dense, 256), 256, 0, L.stream>>>(w, g, 1);
  k_clean_pt3<<<grid_for(w.P, 128), 128, 0, L.stream>>>(w, dr2);
  k_clean_t5<<<grid_for(w.cap.t5_dense, 128), 128, 0, L.stream>>>(w, g, dr2);
  k_clean_pls<<<grid_for(w.P, 128), 128, 0, L.stream>>>(w, dr2);
  const size_t smem = kTcSortMax * (sizeof(unsigned long long) + sizeof(int));
  KT_BEGIN(L, K_TC_ASSEMBLE);
  k_tc_count<<<w.E, 256, 0, L.stream>>>(w, g);
  LST_LAUNCH(L);
  k_tc_collect<<<dim3(w.E, 4), 256, 0, L.stream>>>(w, g);
  k_tc_keys<<<dim3(8, 4 * w.E), 256, 0, L.stream>>>(w, g);
  k_tc_sort<<<dim3(w.E, 4), 1024, smem, L.stream>>>(w, g);
  k_tc_write<<<dim3(8, 4 * w.E), 256, 0, L.stream>>>(w, g);
  *L.launches += 3;
  KT_END(L, K_TC_ASSEMBLE);
  scan_exclusive(w.tc_cnt, w.tcd_off, w.E, w.scan_tmp, L);
  k_tc_dense<<<dim3(16, w.E), 256, 0, L.stream>>>(w, g);
  LST_LAUNCH(L);
  *L.launches += 5;
  // track extensions of the dense rows; the per-anchor-count cut bounds in float64, as pairs
  ExtCuts xc;
  for (int na = 0; na < 8; ++na) xc.rz[na] = ff(c.d.chi2_t5_rz * (na - 2) / 3.0);
  KT_BEGIN(L, K_TC_EXT);
  const int rows_grid = grid_for(w.tc_capacity, 128, 152 * 8);
  const int fit_grid = grid_for(w.ext_qcap, 128, 152 * 4);
  k_ext_cand<<<rows_grid, 128, 0, L.stream>>>(w, g, c.x);
  k_ext_fit<<<dim3(fit_grid, 4), 128, 0, L.stream>>>(w, g, c.x, xc);
  k_ext_select<<<rows_grid, 128, 0, L.stream>>>(w, g);
  k_ext_slow<<<grid_for(w.tc_capacity, 64, 152 * 8), 64, 0, L.stream>>>(w, g, c.x, xc);
  KT_END(L, K_TC_EXT);
  *L.launches += 4;
}

int pt_pre_resident_blocks(int n, int warps) {
  const void* k = n == 3 ? reinterpret_cast<const void*>(k_pt_pre<3>) : reinterpret_cast<const void*>(k_pt_pre<5>);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 32 * warps, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

// the grid's cells per event
int tc_cells_per_event() { return kCellsEta * kCellsPhi; }

void tc_configure() {
  const size_t smem = kTcSortMax * (sizeof(unsigned long long) + sizeof(int));
  cudaFuncSetAttribute(k_tc_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace lst
