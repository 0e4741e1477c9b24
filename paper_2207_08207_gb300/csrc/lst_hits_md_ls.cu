// Hit binning, Mini-Doublets and Line Segments (paper Sec. 2.2 and Sec. 4.2).
//
// Every per-module array is indexed by the virtual module vm = event * n_mods + module, so one
// launch processes a whole batch of events; objects of different events never meet because a
// module's connections stay inside its own event.
#include <mutex>

#include "lst_internal.h"

namespace lst {
namespace {

__device__ __forceinline__ int find_seg(const int32_t* off, int n, int i) {
  int lo = 0, hi = n;   // largest e in [0, n) with off[e] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------------
// hit binning: counting sort by virtual sensor (2 * vm + side), stable in the input order
// ---------------------------------------------------------------------------------------------
__global__ void k_bin_count(Ws w, int n_sens) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ++*w.scan_run;   // a new chain run: new scan epochs
  const int H = w.n_hits();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H; i += gridDim.x * blockDim.x) {
    const int e = find_seg(w.ev_hit_off, w.E, i);
    const int s = w.sensor[i];
    const float x = w.x[i], y = w.y[i], z = w.z[i];
    int err = 0;
    if (s < 0 || s >= n_sens) err |= ERR_BAD_SENSOR;
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) err |= ERR_BAD_COORD;
    if (err) {
      atomicOr(&w.status[ST_ERROR], err);
      atomicOr(&w.ev_stat[e * kEvWords + kEvErr], err);
      w.hit_vs[i] = -1;
      continue;
    }
    const int vs = e * n_sens + s;
    w.hit_vs[i] = vs;
    atomicAdd(&w.sens_cnt[vs], 1);
  }
}

__global__ void k_bin_scatter(Ws w) {
  const int H = w.n_hits();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H; i += gridDim.x * blockDim.x) {
    const int vs = w.hit_vs[i];
    if (vs < 0) continue;
    const int pos = w.sens_off[vs] + atomicAdd(&w.sens_cur[vs], 1);
    w.bidx[pos] = i;
  }
}

// order each sensor's hits by (azimuth relative to the module centre, input index), then gather the
// binned coordinates. The MDs of a module, ordered by lower hit, are then in azimuth order of their
// anchors, which the Line-Segment search uses to take windows of them. The order is a pure function
// of the input (the keys are unique). Groups of 8 lanes take one sensor each (4 per warp); a hit's
// position is its rank among the sensor's keys. Sensors with more than 64 hits are taken by the
// whole warp (ranks up to 256 hits, else one lane's insertion sort).
constexpr int kBinG = 8;      // lanes per sensor
constexpr int kBinPer = 8;    // hits per lane in the grouped path

__device__ __forceinline__ void bin_gather(Ws& w, int pos, int src, int h0) {
  w.bidx[pos] = src;
  w.bx[pos] = w.x[src];
  w.by[pos] = w.y[src];
  w.bz[pos] = w.z[src];
  w.borig[pos] = src - h0;
}

// sort key of input hit src on a module of centre azimuth pc: (relative azimuth, input index)
__device__ __forceinline__ unsigned long long bin_key(const Ws& w, int src, float pc) {
  return ((unsigned long long)float_key(rel_phi(w.x[src], w.y[src], pc)) << 32) | (unsigned)src;
}

// the grouped path for sensors of at most kBinG * T hits: lane `sub` of the sensor's group holds
// hits sub, sub + kBinG, ... and ranks them by the group's keys
template <int T>
__device__ __forceinline__ void bin_rank_gather(Ws& w, const Geo& g, int a, int n, int sub, int vs, bool valid,
                                                int n_sens) {
  const int h0 = valid ? w.ev_hit_off[vs / n_sens] : 0;
  const float pc = valid ? g.phic[(vs % n_sens) >> 1] : 0.f;
  unsigned long long v[T];
  int rk[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int idx = sub + kBinG * t;
    v[t] = idx < n ? bin_key(w, w.bidx[a + idx], pc) : ~0ull;
    rk[t] = 0;
  }
#pragma unroll
  for (int t2 = 0; t2 < T; ++t2) {
#pragma unroll
    for (int s2 = 0; s2 < kBinG; ++s2) {
      const unsigned long long vj = __shfl_sync(0xffffffffu, v[t2], s2, kBinG);
#pragma unroll
      for (int t = 0; t < T; ++t) rk[t] += vj < v[t];
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int idx = sub + kBinG * t;
    if (idx < n) bin_gather(w, a + rk[t], (int)(unsigned)(v[t] & 0xffffffffu), h0);
  }
}

__global__ void k_bin_sort_gather(Ws w, Geo g, int n_sens) {
  const int lane = threadIdx.x & 31;
  const int tile = lane / kBinG, sub = lane % kBinG;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4; base < w.S; base += nwarps * 4) {
    const int vs = base + tile;
    const bool valid = vs < w.S;
    const int a = valid ? w.sens_off[vs] : 0;
    const int n = valid ? w.sens_off[vs + 1] - a : 0;
    int nmax = n;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    if (nmax == 0) continue;
    if (nmax <= kBinG * kBinPer) {
      // T = hits per lane, uniform over the warp: the rank loops are unrolled for each T, so that a
      // warp of small sensors (most hold a few hits) runs only the comparisons it needs
      switch ((nmax + kBinG - 1) / kBinG) {
        case 1: bin_rank_gather<1>(w, g, a, n, sub, vs, valid, n_sens); break;
        case 2: bin_rank_gather<2>(w, g, a, n, sub, vs, valid, n_sens); break;
        case 3: bin_rank_gather<3>(w, g, a, n, sub, vs, valid, n_sens); break;
        case 4: bin_rank_gather<4>(w, g, a, n, sub, vs, valid, n_sens); break;
        case 5: bin_rank_gather<5>(w, g, a, n, sub, vs, valid, n_sens); break;
        case 6: bin_rank_gather<6>(w, g, a, n, sub, vs, valid, n_sens); break;
        case 7: bin_rank_gather<7>(w, g, a, n, sub, vs, valid, n_sens); break;
        default: bin_rank_gather<8>(w, g, a, n, sub, vs, valid, n_sens); break;
      }
      continue;
    }
    // a sensor with more than 64 hits in this warp: the whole warp takes the four sensors in turn
    for (int q = 0; q < 4; ++q) {
      const int vq = base + q;
      if (vq >= w.S) break;
      const int aq = w.sens_off[vq], nq = w.sens_off[vq + 1] - aq;
      if (nq == 0) continue;
      const int h0 = w.ev_hit_off[vq / n_sens];
      const float pc = g.phic[(vq % n_sens) >> 1];
      if (nq <= 256) {
        unsigned long long vv[8];
        int rr[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          vv[t] = lane + 32 * t < nq ? bin_key(w, w.bidx[aq + lane + 32 * t], pc) : ~0ull;
          rr[t] = 0;
        }
        for (int j0 = 0; j0 < nq; j0 += 32) {
          const unsigned long long own = j0 + lane < nq ? bin_key(w, w.bidx[aq + j0 + lane], pc) : ~0ull;
          const int m = min(32, nq - j0);
          for (int j = 0; j < m; ++j) {
            const unsigned long long vj = __shfl_sync(0xffffffffu, own, j);
#pragma unroll
            for (int t = 0; t < 8; ++t) rr[t] += vj < vv[t];
          }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (lane + 32 * t < nq) bin_gather(w, aq + rr[t], (int)(unsigned)(vv[t] & 0xffffffffu), h0);
      } else {
        if (lane == 0) {
          for (int i = aq + 1; i < aq + nq; ++i) {
            const int val = w.bidx[i];
            const unsigned long long kv = bin_key(w, val, pc);
            int j = i - 1;
            while (j >= aq && bin_key(w, w.bidx[j], pc) > kv) {
              w.bidx[j + 1] = w.bidx[j];
              --j;
            }
            w.bidx[j + 1] = val;
          }
        }
        __syncwarp();
        for (int i = aq + lane; i < aq + nq; i += 32) bin_gather(w, i, w.bidx[i], h0);
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------------------------
// per-module capacities, overflow accounting, ordered compaction
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int clamp_cap(double pred, long long bound, int ovr) {
  long long p = (long long)ceil(pred);
  if (p < ovr) p = ovr;
  if (p > bound) p = bound;
  if (p > (1 << 28)) p = 1 << 28;
  return (int)p;
}

__global__ void k_md_caps(Ws w) {
  zero_group_counts(w.grp_key, w.n_hits());   // MDs are grouped by lower hit
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const long long nlo = w.sens_off[2 * vm + 1] - w.sens_off[2 * vm];
    const long long nup = w.sens_off[2 * vm + 2] - w.sens_off[2 * vm + 1];
    const double pred = w.cap_scale * w.stage_scale[0] * (3.0 * (double)max(nlo, nup) + 4.0);
    const int c = clamp_cap(pred, nlo * nup, w.md_ovr[vm]);
    w.md_cap[vm] = c;
    w.md_base[vm] = c;
    w.md_rmin[vm] = 0x7f800000;   // +inf: the dense pass takes the minimum anchor radius
    w.md_rmax[vm] = 0;
  }
}

// Quick rejection of a (lower, upper) hit pair by the Mini-Doublet's z window (barrel) or radial
// window (endcap), exact-safe: true only when the float64 selection is certain to fail, with
// margins far above float32 rounding. Barrel: the window lo = delta min(t1, g t1) - tol_z,
// hi = delta max(t2, g t2) + tol_z (t1,2 = (z_l -+ z_lum) / r_l, 1 <= g <= g_max = 1 / cos(asin(
// sin_max))) contains its g = g_max counterpart, multiplied through by r_l. Endcap: dr = r_u - r_l
// against [dr_min, dr_max] -+ tol_r with dr_max,min = r_l delta / (|z_l| -+ z_lum), multiplied out.
__device__ __forceinline__ bool md_quick_reject(const Cst<float>& c, bool endcap, float delta, float gmax, float xl,
                                               float yl, float zl, float xu, float yu, float zu) {
  const float rl = sqrtf(xl * xl + yl * yl);
  if (!endcap) {
    const float dz = zu - zl;
    const float e1 = zl - c.z_lum, e2 = zl + c.z_lum;
    const float lo = delta * (e1 < 0.f ? gmax * e1 : e1) - c.tol_z * rl;
    const float hi = delta * (e2 > 0.f ? gmax * e2 : e2) + c.tol_z * rl;
    const float m = 1e-4f * (delta * gmax * (fabsf(zl) + c.z_lum) + (c.tol_z + fabsf(dz)) * rl) + 1e-6f;
    return dz * rl < lo - m || dz * rl > hi + m;
  }
  const float az = fabsf(zl);
  if (!(az > c.z_lum * 1.001f)) return false;
  const float ru = sqrtf(xu * xu + yu * yu);
  const float dr = ru - rl;
  const float ld = rl * delta;
  const float m = 2e-4f * (ld + (fabsf(dr) + c.tol_r) * (az + c.z_lum)) + 1e-6f * (ru + rl) * (az + c.z_lum);
  return (dr - c.tol_r) * (az - c.z_lum) > ld + m || (dr + c.tol_r) * (az + c.z_lum) < ld - m;
}

// full float32 evaluation of the first n (<= 32) queued (module, lower hit, upper hit) triples
__device__ __forceinline__ void md_flush(const Ws& w, const Geo& g, const Cst<float>& c, const int4* qe, int n) {
  const int lane = threadIdx.x & 31;
  int v = kReject, vm = 0, l = 0, u = 0;
  float dpc = 0.f, pte = 0.f;
  if (lane < n) {
    const int4 e = qe[lane];
    vm = e.x; l = e.y; u = e.z;
    const int m = vm % g.n_mods;
    v = md_eval<float>(c, g.endcap[m] != 0, g.spacing[m], w.bx[l], w.by[l], w.bz[l], w.bx[u], w.by[u], w.bz[u],
                       kGuardWindow, dpc, pte);
  }
  const int slot = warp_agg_slot_keyed(v == kAccept, vm, w.md_cnt);
  if (slot >= 0) {
    const int cap = w.md_cap[vm], base = w.md_base[vm];
    if (slot < cap && (int64_t)base + slot < w.cap.md_slots) {
      w.ms_lo[base + slot] = l;
      w.ms_up[base + slot] = u;
      w.ms_dpc[base + slot] = dpc;
      w.ms_pte[base + slot] = pte;
      atomicAdd(&w.grp_key[l + 1], 1);
    }
  }
  const int q = warp_agg_slot(v == kUnsure, &w.status[ST_Q_MD]);
  if (q >= 0 && q < w.cap.q_md) w.q_md[q] = make_int4(vm, l, u, 0);
}

// MD candidates: every (lower hit, upper hit) pair of each module. A warp takes G modules at a time
// (G = 1..32, chosen at launch so that the resident warps stay busy), one per lane, spread over the
// whole range (module vm = sweep * G W + lane * W + warp for W warps, which spreads the busy
// inner-layer modules over the warps); a warp scan of their pair counts turns their pairs into one
// index range, and each lane finds its pair's module by a shuffle search, so a warp's lanes stay
// busy however few hits a module holds. Pairs that pass the quick window test
// go to a per-warp queue that carries over and is evaluated fully 32 pairs at a time.
constexpr int kMdWarps = 8;
constexpr int kMdQ = 64;

__global__ void __launch_bounds__(32 * kMdWarps) k_md(Ws w, Geo g, Cst<float> c, int G) {
  __shared__ int4 qbuf[kMdWarps][kMdQ];
  int4* qe = qbuf[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const float gmax = (1.0f + 1e-5f) / sqrtf((1.0f - c.sin_max) * (1.0f + c.sin_max));
  int qn = 0;
  const long long t0 = clock64();
  for (int64_t sweep = 0; sweep * G * nwarps < w.V; ++sweep) {
    if (warp_over_budget(w, t0)) break;
    const int64_t vm64 = sweep * G * nwarps + (int64_t)lane * nwarps + gw;
    const int vm = (int)vm64;
    int lo0 = 0, up0 = 0, nup = 0, np = 0;
    bool ec = false;
    float delta = 0.f;
    if (lane < G && vm64 < w.V) {
      lo0 = w.sens_off[2 * vm];
      up0 = w.sens_off[2 * vm + 1];
      nup = w.sens_off[2 * vm + 2] - up0;
      np = (up0 - lo0) * nup;
      if (np > 0) {
        const int m = vm % g.n_mods;
        ec = g.endcap[m] != 0;
        delta = g.spacing[m];
      }
    }
    int incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - np;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int p0 = 0; p0 < total; p0 += 32) {
      const int p = p0 + lane;
      int j = 0;   // the lane whose module holds pair p: the last lane with excl <= p
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int cand = j + step;
        if (__shfl_sync(0xffffffffu, excl, cand) <= p) j = cand;
      }
      const int pj = p - __shfl_sync(0xffffffffu, excl, j);
      const int nupj = __shfl_sync(0xffffffffu, nup, j);
      const int lo0j = __shfl_sync(0xffffffffu, lo0, j), up0j = __shfl_sync(0xffffffffu, up0, j);
      const bool ecj = __shfl_sync(0xffffffffu, (int)ec, j) != 0;
      const float deltaj = __shfl_sync(0xffffffffu, delta, j);
      const int vmj = __shfl_sync(0xffffffffu, vm, j);
      bool keep = false;
      int l = 0, u = 0;
      if (p < total) {
        // pj / nupj from a float estimate corrected by one step either way (exact: pj < 2^24, and
        // the estimate is within one of the quotient)
        int il = __float2int_rz(__fdividef((float)pj, (float)nupj));
        if (il * nupj > pj) --il;
        else if ((il + 1) * nupj <= pj) ++il;
        l = lo0j + il;
        u = up0j + (pj - il * nupj);
        keep = !md_quick_reject(c, ecj, deltaj, gmax, w.bx[l], w.by[l], w.bz[l], w.bx[u], w.by[u], w.bz[u]);
      }
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      if (keep) qe[qn + __popc(km & ((1u << lane) - 1u))] = make_int4(vmj, l, u, 0);
      qn += __popc(km);
      if (qn >= 32) {
        __syncwarp();
        md_flush(w, g, c, qe, 32);
        __syncwarp();
        qn -= 32;
        if (lane < qn) qe[lane] = qe[32 + lane];
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (qn > 0) md_flush(w, g, c, qe, qn);
}

__global__ void k_md_recheck(Ws w, Geo g, Cst<double> c) {
  const int n = min((int64_t)w.status[ST_Q_MD], w.cap.q_md);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 q = w.q_md[i];
    const int vm = q.x, l = q.y, u = q.z;
    const int m = vm % g.n_mods;
    double dpc, pte;
    const int v = md_eval<double>(c, g.endcap[m] != 0, (double)g.spacing[m], (double)w.bx[l],
                                  (double)w.by[l], (double)w.bz[l], (double)w.bx[u], (double)w.by[u],
                                  (double)w.bz[u], 0.0, dpc, pte);
    atomicAdd(&w.status[ST_REC_MD], 1);
    if (v != kAccept) continue;
    const int slot = atomicAdd(&w.md_cnt[vm], 1);
    const int cap = w.md_cap[vm], base = w.md_base[vm];
    if (slot < cap && (int64_t)base + slot < w.cap.md_slots) {
      w.ms_lo[base + slot] = l;
      w.ms_up[base + slot] = u;
      w.ms_dpc[base + slot] = (float)dpc;
      w.ms_pte[base + slot] = (float)pte;
      atomicAdd(&w.grp_key[l + 1], 1);
    }
  }
}

// dense MDs ordered by (lower hit, upper hit), with the anchor (lower hit) data downstream stages read
__global__ void k_md_dense(Ws w, Geo g, Cst<float> c) {
  const int n = (int)lst_min64(w.md_off[w.V], w.cap.md_dense);
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
    const int s = w.perm[d];
    const int lo = w.ms_lo[s], up = w.ms_up[s];
    const int vm = w.hit_vs[w.bidx[lo]] >> 1;
    w.md_lo[d] = lo;
    w.md_up[d] = up;
    w.md_vm[d] = vm;
    w.o_md_lo[d] = w.borig[lo];   // event-local outputs: input hit indices, module
    w.o_md_up[d] = w.borig[up];
    w.o_md_mod[d] = vm % g.n_mods;
    store_out(w.md_dpc, w.md_dpc_h, d, w.ms_dpc[s]);
    store_out(w.md_pte, w.md_pte_h, d, w.ms_pte[s]);
    const float x = w.bx[lo], y = w.by[lo];
    // x^2 + y^2 as an unevaluated float pair (products exact by FMA), its float32 square root, and
    // the low part of the radius: r = r_hi + (q - r_hi^2) / (2 r_hi) to float-float accuracy
    const float xx = x * x, exx = fmaf(x, x, -xx);
    const float yy = y * y, eyy = fmaf(y, y, -yy);
    const float q = xx + yy;
    const float qb = q - xx;                                  // TwoSum: q + qs == xx + yy exactly
    const float qs = (xx - (q - qb)) + (yy - qb);
    const float qe = qs + exx + eyy;
    const float r = sqrtf(q);
    const float rlo = (fmaf(-r, r, q) + qe) / (2.0f * r);
    w.md_rlo[d] = r > 0.f ? rlo : 0.f;
    const float sthr = c.two_rthr * asinf(fminf(r / c.two_rthr, 1.0f));
    const float alpha = asinf(fminf(r * c.k2p, c.sin_max));
    w.md_xyzr[d] = make_float4(x, y, w.bz[lo], r);
    w.md_sa[d] = make_float2(sthr, alpha);
    w.md_ec[d] = g.endcap[vm % g.n_mods];
    w.md_rphi[d] = rel_phi(x, y, g.phic[vm % g.n_mods]);
    // radius range of the module's anchors (r >= 0: float bits order like the values), one atomic
    // per module and warp (a module's MDs are contiguous)
    const unsigned grp = __match_any_sync(__activemask(), vm);
    const int rmin = __reduce_min_sync(grp, __float_as_int(r)), rmax = __reduce_max_sync(grp, __float_as_int(r));
    if ((threadIdx.x & 31) == __ffs(grp) - 1) {
      atomicMin(&w.md_rmin[vm], rmin);
      atomicMax(&w.md_rmax[vm], rmax);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Line Segments
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ int md_count(const Ws& w, int vm) { return w.md_off[vm + 1] - w.md_off[vm]; }

// LS capacity of each module (exact bound: its MDs x the MDs of its connected modules), its number
// of work items (chunks of its outer MDs: ceil(outer MDs / ls_chunk), at most kLsMaxChunks), their
// cost bucket floor(log2(pairs per chunk)) for the persistent kernel's work list, and the inputs of
// the LS azimuth windows that depend on the module's MDs alone (alpha_thr of the largest anchor
// radius, 1 / the smallest), computed once here instead of by every item that connects to it
__global__ void k_ls_caps(Ws w, Geo g, Cst<float> c) {
  zero_group_counts(w.lsin_off, w.md_off[w.V]);   // LS are grouped by inner MD
  __shared__ int hist[32];
  if (threadIdx.x < 32) hist[threadIdx.x] = 0;
  __syncthreads();
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const int m = vm % g.n_mods, e0 = vm - m;
    const long long na = md_count(w, vm);
    long long nb = 0;
    float2 win = make_float2(0.f, 0.f);
    if (na > 0) {
      for (int k = g.conn_off[m]; k < g.conn_off[m + 1]; ++k) nb += md_count(w, e0 + g.conn_tgt[k]);
      win.x = asinf(fminf(__int_as_float(w.md_rmax[vm]) * c.k2p, c.sin_max));
      win.y = 1.0f / __int_as_float(w.md_rmin[vm]);
    }
    w.md_win[vm] = win;
    const long long bound = na * nb;
    const double pred = w.cap_scale * w.stage_scale[1] * (32.0 + 0.5 * (double)bound);
    const int cc = clamp_cap(pred, bound, w.ls_ovr[vm]);
    w.ls_cap[vm] = cc;
    w.ls_base[vm] = cc;
    int b = -1, nch = 0;
    if (bound > 0) {
      nch = (int)lst_min64((nb + w.ls_chunk - 1) / w.ls_chunk, kLsMaxChunks);
      const long long per = na * ((nb + nch - 1) / nch);
      b = 63 - __clzll((unsigned long long)per);
      if (b > 31) b = 31;
      atomicAdd(&hist[b], nch);
    }
    w.work_bucket[vm] = b;
    w.work_nch[vm] = nch;
  }
  __syncthreads();
  if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(&w.work_cnt[threadIdx.x], hist[threadIdx.x]);
}

// the work list: items by cost bucket, most expensive first. Every block derives the bucket offsets
// from the 32 bucket counts itself; block 0 also stores them (the LS kernel reads the total).
__global__ void k_ls_work_fill(Ws w) {
  __shared__ int off[33];
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 31; b >= 0; --b) {
      off[b] = acc;
      acc += w.work_cnt[b];
    }
    off[32] = acc;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x <= 32) w.work_off[threadIdx.x] = off[threadIdx.x];
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm - (int)(threadIdx.x & 31) < w.V;
       vm += gridDim.x * blockDim.x) {
    const int lane = threadIdx.x & 31;
    const int b = vm < w.V ? w.work_bucket[vm] : -1;
    const int nch = b >= 0 ? w.work_nch[vm] : 0;
    // one atomic per bucket and warp: lanes with the same bucket share it; a lane's items follow
    // those of the lower lanes of its bucket
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(grp) - 1;
    int pre = 0;
    for (int j = 0; j < 32; ++j) {
      const int v = __shfl_sync(0xffffffffu, nch, j);
      if (j < lane && ((grp >> j) & 1u)) pre += v;
    }
    const int sum = __reduce_add_sync(grp, nch);
    int base = 0;
    if (b >= 0 && lane == leader) base = atomicAdd(&w.work_cur[b], sum);
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b >= 0)
      for (int k = 0; k < nch; ++k) {
        const int at = off[b] + base + pre + k;
        w.work[at] = vm;
        w.work_c[at] = k;
      }
  }
}

// One warp per work item at a time: a module, or, in small batches, one of up to kLsMaxChunks equal
// chunks of a heavy module's candidate outer MDs (so that one module does not hold the whole launch).
// The module's own MDs (A) are staged 32 at a time in shared memory; each lane holds one MD of the
// connected modules (B) in registers and sweeps the staged A. The MDs of every module are ordered by
// anchor azimuth about the module centre (the binning orders hits so), so for each staged chunk of A
// only a contiguous window of each connected module's MDs can pass the azimuth cut: the window
// [min phi_A - W, max phi_A + W] (in B's own azimuth frame), W an upper bound of the cut's
// bound over the chunk's and the target's radius ranges (alpha_thr(r2max) - alpha_thr(r1min) +
// (n_sigma sigma_rphi + d0_max)(1 / r1min + 1 / r2min), plus a margin far above the float32 error of
// the azimuths), is found by two binary searches per target and only those B are swept. A pair
// outside the window fails the exact azimuth cut, so the skipped pairs are ones every evaluation
// rejects. Inside it a conservative division-free test (below) rejects most pairs, and the survivors
// go to a per-warp queue that carries over from item to item; whenever it holds 32 pairs, every lane
// takes one of them through the full evaluation, so the expensive path runs with a full warp.
// Persistent mode: the grid holds every resident warp and the warps take the cost-ordered work list
// in a boustrophedon order (heaviest modules first, one pass forward and the next backward, which
// evens out the sums); otherwise warps stride over all modules in index order.
constexpr int kLsAW = 32;   // inner MDs staged per chunk
constexpr int kLsQ = 64;    // survivor queue per warp (at most 31 carried + 32 new)
constexpr int kLsGrab = 8;   // most items a warp takes from the device queue per atomic

// Per-warp shared memory of k_ls: T target slots (the loaded map's largest degree rounded up to 32).
struct LsSmem {
  float4* a_xyzr;   // [kLsAW] staged inner anchors (x, y, z, r)
  float4* tinfo;    // [T] per connected module: (its centre azimuth relative to A's, alpha_thr of its
                    //     largest anchor radius, 1 / its smallest anchor radius, endcap flag)
  float2* a_sal;    // [kLsAW] (arc length at threshold, alpha)
  int2* tbc;        // [T] (first dense MD, MD count) of each connected module
  int* wpre;        // [T + 1] prefix of the window sizes of the current inner chunk
  int* wbeg;        // [T] first dense MD of each window
  int* a_id;        // [kLsAW]
  int *q_vm, *q_a, *q_b;   // [kLsQ] survivor queue
};

__host__ __device__ inline size_t ls_smem_per_warp(int T) {
  const size_t b = (size_t)kLsAW * 16 + (size_t)T * 16 + (size_t)kLsAW * 8 + (size_t)T * 8 + (size_t)(T + 1) * 4 +
                   (size_t)T * 4 + (size_t)kLsAW * 4 + 3 * (size_t)kLsQ * 4;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ LsSmem ls_smem(unsigned char* base, int T) {
  LsSmem S;
  unsigned char* p = base;
  S.a_xyzr = reinterpret_cast<float4*>(p); p += kLsAW * 16;
  S.tinfo = reinterpret_cast<float4*>(p); p += T * 16;
  S.a_sal = reinterpret_cast<float2*>(p); p += kLsAW * 8;
  S.tbc = reinterpret_cast<int2*>(p); p += T * 8;
  S.wpre = reinterpret_cast<int*>(p); p += (T + 1) * 4;
  S.wbeg = reinterpret_cast<int*>(p); p += T * 4;
  S.a_id = reinterpret_cast<int*>(p); p += kLsAW * 4;
  S.q_vm = reinterpret_cast<int*>(p); p += kLsQ * 4;
  S.q_a = reinterpret_cast<int*>(p); p += kLsQ * 4;
  S.q_b = reinterpret_cast<int*>(p);
  return S;
}

// The window [lo, hi] of a connected module's MDs, sorted by relative azimuth rp[0, n): jl = the
// number of rp below lo, jh = the number not above hi. Up to 8 MDs are counted with independent
// loads (one memory round trip instead of a chain of dependent ones); more are bisected, both bounds
// in the same loop so that their loads overlap.
__device__ __forceinline__ void ls_window(const float* rp, int n, float lo, float hi, int& jl, int& jh) {
  if (n <= 8) {
    int a = 0, b = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < n) {
        const float v = rp[k];
        a += v < lo ? 1 : 0;
        b += v <= hi ? 1 : 0;
      }
    jl = a;
    jh = b;
    return;
  }
  int l1 = 0, h1 = n, l2 = 0, h2 = n;
  while (l1 < h1 || l2 < h2) {
    if (l1 < h1) {
      const int mid = (l1 + h1) >> 1;
      if (rp[mid] < lo) l1 = mid + 1; else h1 = mid;
    }
    if (l2 < h2) {
      const int mid = (l2 + h2) >> 1;
      if (rp[mid] <= hi) l2 = mid + 1; else h2 = mid;
    }
  }
  jl = l1;
  jh = l2;
}

// Quick rejection of an (a, b) pair, exact-safe: it returns true only when the float64 evaluation
// is certain to reject, with margins far above the float32 rounding of the anchors and of this
// arithmetic.
//  azimuth: |dphi| >= |sin dphi| = |p1 x p2| / (r1 r2), against r1 r2 times an upper bound of the
//    window, (alpha2 - alpha1) + (n_sigma sigma_rphi + d0_max)(1/r1 + 1/r2), multiplied out;
//  r-z: with D = r2 - r1, z0r = (z1 r2 - z2 r1) / D and z0s the same with the arc lengths s, the
//    window L = z_lum + n_sigma sqrt(q1^2 + .. + q4^2) has D^2 L <= D^2 z_lum + n_sigma (|D| (r2 sz1
//    + r1 sz2) + |z1 - z2| (r2 sr1 + r1 sr2)), since |q3| D^2 = r2 |z1 - z2| sr1 and |q4| D^2 =
//    r1 |z1 - z2| sr2; both z0r and z0s beyond that bound on the same side rejects. Applied only when
//    |D| >= 1 and |s2 - s1| >= |D| (always so for r below 2 R_thr), where float32 z0 is accurate.
__device__ __forceinline__ bool ls_quick_reject(const Cst<float>& c, float4 a, float2 as, float sz1, float sr1,
                                                float x2, float y2, float z2, float r2, float s2, float al2,
                                                float sz2, float sr2) {
  const float r1 = a.w;
  const float cr = fmaf(a.x, y2, -a.y * x2);
  const float win = fmaf(r1 * r2, (al2 - as.y) + 1e-5f, (c.n_sigma * c.sigma_rphi + c.d0_max) * (r1 + r2));
  if (fabsf(cr) > fmaf(win, 1.0003f, 1e-6f)) return true;
  const float D = r2 - r1, Ds = s2 - as.x;
  const float aD = fabsf(D);
  if (!(aD >= 1.0f && fabsf(Ds) >= aD)) return false;
  const float dz = fabsf(a.z - z2);
  const float ld2 = fmaf(D * D, c.z_lum,
                         c.n_sigma * fmaf(aD, fmaf(r2, sz1, r1 * sz2), dz * fmaf(r2, sr1, r1 * sr2)));
  const float E = (fabsf(a.z) + fabsf(z2)) * (as.x + s2);        // bounds |z1 r2| + |z2 r1| (s >= r)
  const float M = fmaf(ld2, 1.0f + 1.0f / 1024.0f, E * aD * (1.0f / 262144.0f));
  const float P = fmaf(a.z, r2, -z2 * r1) * D;                   // z0r D^2
  const float Ps = fmaf(a.z, s2, -z2 * as.x) * Ds * (D * D);     // z0s Ds^2 D^2
  const float Ms = M * (Ds * Ds);
  return (P > M && Ps > Ms) || (P < -M && Ps < -Ms);
}


// full float32 evaluation of the first n (<= 32) queued pairs, one per lane; called by the whole warp
__device__ __forceinline__ void ls_flush(const Ws& w, const Cst<float>& c, const LsSmem& S, int n) {
  const int lane = lane_id();
  int v = kReject, vm = 0, a = 0, b = 0;
  float z0 = 0.f, dphi = 0.f;
  if (lane < n) {
    vm = S.q_vm[lane];
    a = S.q_a[lane];
    b = S.q_b[lane];
    const float4 pa = w.md_xyzr[a], pb = w.md_xyzr[b];
    v = ls_eval<float>(c, pa.x, pa.y, pa.z, pa.w, w.md_sa[a].x, w.md_ec[a] != 0, pb.x, pb.y, pb.z, pb.w,
                       w.md_sa[b].x, w.md_ec[b] != 0, kGuardWindow, z0, dphi);
  }
  const int slot = warp_agg_slot_keyed(v == kAccept, vm, w.ls_cnt);
  bool stored = false;
  if (slot >= 0) {
    const int cap = w.ls_cap[vm], base = w.ls_base[vm];
    if (slot < cap && (int64_t)base + slot < w.cap.ls_slots) {
      w.lss_in[base + slot] = a;
      w.lss_out[base + slot] = b;
      w.lss_dphi[base + slot] = dphi;
      stored = true;
    }
  }
  warp_count_keyed(stored, a + 1, w.lsin_off);   // the group sizes of the compaction
  const int q = warp_agg_slot(v == kUnsure, &w.status[ST_Q_LS]);
  if (q >= 0 && q < w.cap.q_ls) w.q_ls[q] = make_int4(vm, a, b, 0);
}

__global__ void __launch_bounds__(256, 4) k_ls(Ws w, Geo g, Cst<float> c, int persistent) {
  extern __shared__ __align__(16) unsigned char ls_smem_raw[];
  const int T = g.ls_tcap;
  const LsSmem S = ls_smem(ls_smem_raw + (threadIdx.x >> 5) * ls_smem_per_warp(T), T);
  const int lane = lane_id();
  const int n_warps = gridDim.x * (blockDim.x >> 5);
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int n_items = persistent ? w.work_off[32] : w.V;
  const float kwin = c.n_sigma * c.sigma_rphi + c.d0_max;
  const float kPiF = 3.14159265f;
  int qn = 0;   // pairs waiting in this warp's queue
  unsigned long long n_pairs = 0;   // windowed pairs this warp evaluated (added once, at the end)
  const long long t0 = clock64();
  int sweep = 0;
  // device queue: a warp takes `grab` consecutive items per atomic on the queue head (one atomic per
  // item would serialise on that one address when there are many items); with few items per warp
  // it takes them one at a time, so that no warp holds items the others could run
  const int grab = max(1, min(kLsGrab, n_items / max(1, n_warps * 16)));
  int q_next = 0, q_end = 0;
  for (;;) {
    if (warp_over_budget(w, t0)) break;
    int item;
    if (persistent == 2) {   // device queue: the next cost-ordered item
      if (q_next >= q_end) {
        int h = 0;
        if (lane == 0) h = atomicAdd(w.ls_head, grab);
        q_next = __shfl_sync(0xffffffffu, h, 0);
        q_end = min(q_next + grab, n_items);
      }
      item = q_next++;
      if (item >= n_items) break;
    } else {                 // static deal in boustrophedon order
      if ((int64_t)sweep * n_warps >= n_items) break;
      item = sweep * n_warps + ((sweep & 1) ? n_warps - 1 - gw : gw);
      ++sweep;
      if (item >= n_items) continue;
    }
    const int vm = persistent ? w.work[item] : item;
    const int chunk = persistent ? w.work_c[item] : 0;
    const int nch = persistent ? w.work_nch[vm] : 1;
    const int na = md_count(w, vm);
    if (na == 0) continue;
    const int m = vm % g.n_mods, e0 = vm - m;
    const int t0c = g.conn_off[m];
    const int nt = min(g.conn_off[m + 1] - t0c, T);
    // the connected modules: their MD ranges and the window inputs that depend on them alone
    for (int t = lane; t < nt; t += 32) {
      const int k = t0c + t;
      const int tm = g.conn_tgt[k];
      const float dpc = g.conn_dpc[k];
      const int vb = e0 + tm;
      const int b0 = w.md_off[vb], b1 = w.md_off[vb + 1];
      const float2 tw = w.md_win[vb];
      S.tbc[t] = make_int2(b0, b1 - b0);
      S.tinfo[t] = make_float4(dpc, tw.x, tw.y, g.endcap[tm] ? 1.f : 0.f);
    }
    const bool aec = g.endcap[m] != 0;
    const float sz1 = aec ? 0.f : c.sigma_z, sr1 = aec ? c.sigma_r : 0.f;
    const int a_begin = w.md_off[vm];
    for (int a0 = 0; a0 < na; a0 += kLsAW) {
      const int nA = min(kLsAW, na - a0);
      __syncwarp();
      float r1 = 3.0e38f, al1 = 3.0e38f;
      if (lane < nA) {
        const int d = a_begin + a0 + lane;
        const float4 pa = w.md_xyzr[d];
        const float2 sa = w.md_sa[d];
        S.a_xyzr[lane] = pa;
        S.a_sal[lane] = sa;
        S.a_id[lane] = d;
        r1 = pa.w;
        al1 = sa.y;
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        r1 = fminf(r1, __shfl_xor_sync(0xffffffffu, r1, o));
        al1 = fminf(al1, __shfl_xor_sync(0xffffffffu, al1, o));
      }
      // the chunk's azimuth range (the module's MDs are in azimuth order)
      const float ph_lo = w.md_rphi[a_begin + a0], ph_hi = w.md_rphi[a_begin + a0 + nA - 1];
      const float ir1 = 1.0f / r1;
      // each target's window, and their prefix by a warp scan, 32 targets at a time
      int run = 0;
      for (int t = lane; t - lane < nt; t += 32) {
        int cw = 0;
        if (t < nt) {
          const int2 bc = S.tbc[t];
          int jl = 0, jh = 0;
          if (bc.y > 0) {
            const float4 ti = S.tinfo[t];
            const float W = (ti.y - al1) + kwin * (ir1 + ti.z) + 2e-4f;
            const float lo = ti.x + ph_lo - W, hi = ti.x + ph_hi + W;
            if (lo < -kPiF || hi > kPiF) {   // the window wraps: take the whole module
              jh = bc.y;
            } else if (lo <= hi) {
              ls_window(w.md_rphi + bc.x, bc.y, lo, hi, jl, jh);
            }
          }
          S.wbeg[t] = bc.x + jl;
          cw = jh - jl;
        }
        int incl = cw;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (t < nt) S.wpre[t + 1] = run + incl;
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) S.wpre[0] = 0;
      __syncwarp();
      const int totB = run;
      // this item's share of the windowed outer MDs: chunk `chunk` of nch equal chunks
      const int csz = (totB + nch - 1) / max(nch, 1);
      const int jbeg = chunk * csz, jend = min(totB, jbeg + csz);
      if (jend > jbeg) n_pairs += (unsigned long long)(jend - jbeg) * (unsigned long long)nA;
      for (int j0 = jbeg; j0 < jend; j0 += 32) {
        const int j = j0 + lane;
        const bool has_b = j < jend;
        float x2 = 0.f, y2 = 0.f, z2 = 0.f, r2 = 1.f, s2 = 1.f, al2 = 0.f, sz2 = 0.f, sr2 = 0.f;
        int bid = 0;
        if (has_b) {
          int lo = 0, hi = nt;   // target k with wpre[k] <= j < wpre[k + 1]
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (S.wpre[mid] <= j) lo = mid; else hi = mid;
          }
          bid = S.wbeg[lo] + (j - S.wpre[lo]);
          const float4 pb = w.md_xyzr[bid];
          const float2 sb = w.md_sa[bid];
          x2 = pb.x; y2 = pb.y; z2 = pb.z; r2 = pb.w;
          s2 = sb.x; al2 = sb.y;
          const bool bec = S.tinfo[lo].w != 0.f;
          sz2 = bec ? 0.f : c.sigma_z;
          sr2 = bec ? c.sigma_r : 0.f;
        }
        for (int ia = 0; ia < nA; ++ia) {
          const bool keep = has_b && !ls_quick_reject(c, S.a_xyzr[ia], S.a_sal[ia], sz1, sr1, x2, y2, z2, r2,
                                                      s2, al2, sz2, sr2);
          const unsigned km = __ballot_sync(0xffffffffu, keep);
          if (km == 0) continue;
          if (keep) {
            const int pos = qn + __popc(km & ((1u << lane) - 1u));
            S.q_vm[pos] = vm;
            S.q_a[pos] = S.a_id[ia];
            S.q_b[pos] = bid;
          }
          qn += __popc(km);
          if (qn >= 32) {
            __syncwarp();
            ls_flush(w, c, S, 32);
            __syncwarp();
            qn -= 32;
            if (lane < qn) {   // move the rest (at most 31) to the front
              const int t_vm = S.q_vm[32 + lane], t_a = S.q_a[32 + lane], t_b = S.q_b[32 + lane];
              S.q_vm[lane] = t_vm;
              S.q_a[lane] = t_a;
              S.q_b[lane] = t_b;
            }
            __syncwarp();
          }
        }
      }
    }
    __syncwarp();
  }
  __syncwarp();
  if (qn > 0) ls_flush(w, c, S, qn);
  if (lane == 0 && n_pairs) atomicAdd(reinterpret_cast<unsigned long long*>(&w.status[ST_LS_PAIRS]), n_pairs);
}

// dynamic shared memory of k_ls for a block of `block` threads and T target slots per warp
inline size_t ls_smem_bytes(int block, int T) { return ls_smem_per_warp(T) * (size_t)(block / 32); }

}  // namespace

// The kernel's dynamic shared memory limit is a property of the function, shared by every context of
// the process: it is only ever raised, to what the largest block (256 threads) of the largest map
// loaded so far needs, so that no context lowers it below what another one launches with.
int ls_resident_blocks(int block, int T) {
  static std::mutex mu;
  static size_t limit = 0;
  const size_t bytes = ls_smem_bytes(block, T);
  {
    std::lock_guard<std::mutex> lock(mu);
    const size_t want = ls_smem_bytes(256, T);
    if (want > limit) {
      if (cudaFuncSetAttribute(k_ls, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      limit = want;
    }
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ls, block, bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

namespace {

__device__ __forceinline__ void md_anchor64(const Ws& w, const Cst<double>& c, int d, double& x,
                                            double& y, double& z, double& r, double& s) {
  const float4 p = w.md_xyzr[d];
  x = p.x; y = p.y; z = p.z;
  r = sqrt(x * x + y * y);
  s = c.two_rthr * asin(fmin(r / c.two_rthr, 1.0));
}

__global__ void k_ls_recheck(Ws w, Cst<double> c) {
  const int n = min((int64_t)w.status[ST_Q_LS], w.cap.q_ls);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 q = w.q_ls[i];
    const int vm = q.x, a = q.y, b = q.z;
    double x1, y1, z1, r1, s1, x2, y2, z2, r2, s2, z0, dphi;
    md_anchor64(w, c, a, x1, y1, z1, r1, s1);
    md_anchor64(w, c, b, x2, y2, z2, r2, s2);
    const int v = ls_eval<double>(c, x1, y1, z1, r1, s1, w.md_ec[a] != 0, x2, y2, z2, r2, s2,
                                  w.md_ec[b] != 0, 0.0, z0, dphi);
    atomicAdd(&w.status[ST_REC_LS], 1);
    if (v != kAccept) continue;
    const int slot = atomicAdd(&w.ls_cnt[vm], 1);
    const int cap = w.ls_cap[vm], base = w.ls_base[vm];
    if (slot < cap && (int64_t)base + slot < w.cap.ls_slots) {
      w.lss_in[base + slot] = a;
      w.lss_out[base + slot] = b;
      w.lss_dphi[base + slot] = (float)dphi;
      atomicAdd(&w.lsin_off[a + 1], 1);
    }
  }
}

// single-event binning on plain arrays (the standalone lst_bin_hits entry point)
__global__ void k_braw_count(const int32_t* sensor, int n, int n_sens, int32_t* cnt, int32_t* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = sensor[i];
    if (s < 0 || s >= n_sens) { atomicOr(err, ERR_BAD_SENSOR); continue; }
    atomicAdd(&cnt[s], 1);
  }
}

__global__ void k_braw_scatter(const int32_t* sensor, int n, int n_sens, const int32_t* off, int32_t* cur,
                               int32_t* order) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = sensor[i];
    if (s < 0 || s >= n_sens) continue;
    order[off[s] + atomicAdd(&cur[s], 1)] = i;
  }
}

__global__ void k_braw_sort(const int32_t* off, int n_sens, int32_t* order) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sens; s += gridDim.x * blockDim.x) {
    const int a = off[s], b = off[s + 1];
    for (int i = a + 1; i < b; ++i) {
      const int v = order[i];
      int j = i - 1;
      while (j >= a && order[j] > v) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = v;
    }
  }
}

}  // namespace

void run_bin_raw(const int32_t* sensor, int n, int n_sens, int32_t* order, int32_t* offsets, int32_t* cnt,
                 int32_t* cur, int32_t* err, int32_t* scan_tmp, const Launch& L) {
  k_braw_count<<<grid_for(n, 256), 256, 0, L.stream>>>(sensor, n, n_sens, cnt, err);
  LST_LAUNCH(L);
  scan_exclusive(cnt, offsets, n_sens, scan_tmp, L);
  k_braw_scatter<<<grid_for(n, 256), 256, 0, L.stream>>>(sensor, n, n_sens, offsets, cur, order);
  LST_LAUNCH(L);
  k_braw_sort<<<grid_for(n_sens, 128), 128, 0, L.stream>>>(offsets, n_sens, order);
  LST_LAUNCH(L);
}

void run_binning(const Ws& w, const Geo& g, const Launch& L) {
  const int n_sens = 2 * g.n_mods;
  k_bin_count<<<grid_for(w.H, 256), 256, 0, L.stream>>>(w, n_sens);
  LST_LAUNCH(L);
  scan_exclusive(w.sens_cnt, w.sens_off, w.S, w.scan_tmp, L);
  k_bin_scatter<<<grid_for(w.H, 256), 256, 0, L.stream>>>(w);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_BIN);
  k_bin_sort_gather<<<grid_for((int64_t)w.S * 8, 256, 152 * 32), 256, 0, L.stream>>>(w, g, n_sens);
  KT_END(L, K_BIN);
  LST_LAUNCH(L);
}

void run_md(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  k_md_caps<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w);
  LST_LAUNCH(L);
  scan_exclusive(w.md_base, w.md_base, w.V, w.scan_tmp, L);
  KT_BEGIN(L, K_MD);
  {
    const int64_t resident_warps = (int64_t)L.n_sm * 8 * kMdWarps;
    int G = 1;   // modules per warp and sweep: about two sweeps over the resident warps
    while (G < 32 && (int64_t)G * 2 * resident_warps * 2 <= w.V) G *= 2;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((w.V / G + kMdWarps - 1) / kMdWarps, L.n_sm * 8));
    k_md<<<blocks, 32 * kMdWarps, 0, L.stream>>>(w, g, c.f, G);
  }
  KT_END(L, K_MD);
  LST_LAUNCH(L);
  k_md_recheck<<<grid_for(w.cap.q_md, 128, 152 * 4), 128, 0, L.stream>>>(w, g, c.d);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_MD_COMPACT);
  GroupArgs ga{w.md_cnt, w.md_cap, w.md_base, w.cap.md_slots, ST_OVF_MD, ST_ARENA_MD, w.ms_lo, w.ms_up,
               nullptr, nullptr, w.cap.H, &w.ev_hit_off[w.E], w.cap.md_dense, ST_DENSE_MD,
               w.md_off, w.sens_off, 2, kDensePerm};
  group_slots(w, ga, L);
  k_md_dense<<<grid_for(w.cap.md_dense, 256), 256, 0, L.stream>>>(w, g, c.f);
  KT_END(L, K_MD_COMPACT);
  LST_LAUNCH(L);
}

void run_ls(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  k_ls_caps<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w, g, c.f);
  LST_LAUNCH(L);
  scan_exclusive(w.ls_base, w.ls_base, w.V, w.scan_tmp, L);
  if (L.persistent) {
    k_ls_work_fill<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w);
    *L.launches += 1;
  }
  KT_BEGIN(L, K_LS);
  {
    const size_t smem = ls_smem_bytes(L.block_ls, g.ls_tcap);
    const int warps = L.block_ls / 32;
    if (L.persistent) {
      // every resident warp, no more: the boustrophedon assignment is static
      const int bps = L.ls_blocks_per_sm > 0 ? L.ls_blocks_per_sm : 1;
      k_ls<<<L.n_sm * bps, L.block_ls, smem, L.stream>>>(w, g, c.f, L.persistent);
    } else {
      k_ls<<<grid_for((w.V + warps - 1) / warps, 1, 152 * 16), L.block_ls, smem, L.stream>>>(w, g, c.f, 0);
    }
  }
  KT_END(L, K_LS);
  LST_LAUNCH(L);
  k_ls_recheck<<<grid_for(w.cap.q_ls, 128, 152 * 4), 128, 0, L.stream>>>(w, c.d);
  LST_LAUNCH(L);
  // LS ordered by inner MD: the per-MD group offsets are the "LS by inner MD" adjacency
  KT_BEGIN(L, K_LS_COMPACT);
  GroupArgs ga{w.ls_cnt, w.ls_cap, w.ls_base, w.cap.ls_slots, ST_OVF_LS, ST_ARENA_LS, w.lss_in, w.lss_out,
               nullptr, w.lsin_off, w.cap.md_dense, &w.md_off[w.V], w.cap.ls_dense, ST_DENSE_LS,
               w.ls_off, w.md_off, 1, kDenseLs};
  group_slots(w, ga, L);
  KT_END(L, K_LS_COMPACT);
}

}  // namespace lst
