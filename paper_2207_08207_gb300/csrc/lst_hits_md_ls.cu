// Hit binning, Mini-Doublets and Line Segments (paper Sec. 2.2 and Sec. 4.2).
//
// Every per-module array is indexed by the virtual module vm = event * n_mods + module, so one
// launch processes a whole batch of events; objects of different events never meet because a
// module's connections stay inside its own event.
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

// order each sensor's hits by input index (makes the binning identical to a stable sort), then
// gather the binned coordinates
__global__ void k_bin_sort_gather(Ws w, int n_sens) {
  for (int vs = blockIdx.x * blockDim.x + threadIdx.x; vs < w.S; vs += gridDim.x * blockDim.x) {
    const int a = w.sens_off[vs], b = w.sens_off[vs + 1];
    for (int i = a + 1; i < b; ++i) {
      const int v = w.bidx[i];
      int j = i - 1;
      while (j >= a && w.bidx[j] > v) {
        w.bidx[j + 1] = w.bidx[j];
        --j;
      }
      w.bidx[j + 1] = v;
    }
    const int e = vs / n_sens;
    const int h0 = w.ev_hit_off[e];
    for (int i = a; i < b; ++i) {
      const int src = w.bidx[i];
      w.bx[i] = w.x[src];
      w.by[i] = w.y[src];
      w.bz[i] = w.z[src];
      w.borig[i] = src - h0;
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
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const long long nlo = w.sens_off[2 * vm + 1] - w.sens_off[2 * vm];
    const long long nup = w.sens_off[2 * vm + 2] - w.sens_off[2 * vm + 1];
    const double pred = w.cap_scale * (3.0 * (double)max(nlo, nup) + 4.0);
    const int c = clamp_cap(pred, nlo * nup, w.md_ovr[vm]);
    w.md_cap[vm] = c;
    w.md_base[vm] = c;
  }
}

// effective count = min(count, capacity, room left in the arena); excess is recorded
__global__ void k_effective(Ws w, const int32_t* cnt, const int32_t* cap, const int32_t* base,
                            int64_t slots, int32_t* eff_out, int ovf_word, int arena_word, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = cnt[i], k = cap[i], b = base[i];
    int eff = min(c, k);
    if (c > k) atomicAdd(&w.status[ovf_word], c - k);
    if ((int64_t)b + eff > slots) {
      eff = (int)(slots - b > 0 ? slots - b : 0);
      atomicMax(&w.status[arena_word], base[n]);
    }
    eff_out[i] = eff;
  }
}

__global__ void k_md(Ws w, Geo g, Cst<float> c) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int vm = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vm < w.V; vm += nwarps) {
    const int m = vm % g.n_mods;
    const int lo0 = w.sens_off[2 * vm], up0 = w.sens_off[2 * vm + 1];
    const int nlo = up0 - lo0, nup = w.sens_off[2 * vm + 2] - up0;
    const int np = nlo * nup;
    if (np == 0) continue;
    const bool ec = g.endcap[m] != 0;
    const float delta = g.spacing[m];
    const int cap = w.md_cap[vm], base = w.md_base[vm];
    for (int p0 = 0; p0 < np; p0 += 32) {
      const int p = p0 + lane;
      int v = kReject, l = 0, u = 0;
      float dpc = 0.f, pte = 0.f;
      if (p < np) {
        l = lo0 + p / nup;
        u = up0 + p % nup;
        v = md_eval<float>(c, ec, delta, w.bx[l], w.by[l], w.bz[l], w.bx[u], w.by[u], w.bz[u],
                           kGuardWindow, dpc, pte);
      }
      const int slot = warp_agg_slot(v == kAccept, &w.md_cnt[vm]);
      if (slot >= 0 && slot < cap && (int64_t)base + slot < w.cap.md_slots) {
        w.ms_lo[base + slot] = l;
        w.ms_up[base + slot] = u;
        w.ms_dpc[base + slot] = dpc;
        w.ms_pte[base + slot] = pte;
      }
      const int q = warp_agg_slot(v == kUnsure, &w.status[ST_Q_MD]);
      if (q >= 0 && q < w.cap.q_md) w.q_md[q] = make_int4(vm, l, u, 0);
    }
  }
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
    }
  }
}

// dense MDs ordered by (lower hit, upper hit), with the anchor (lower hit) data downstream stages read
__global__ void k_md_dense(Ws w, Geo g, Cst<float> c) {
  const int n = (int)lst_min64(w.md_off[w.V], w.cap.md_dense);
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
    const int s = w.perm[d];
    const int lo = w.ms_lo[s];
    const int vm = w.hit_vs[w.bidx[lo]] >> 1;
    w.md_lo[d] = lo;
    w.md_up[d] = w.ms_up[s];
    w.md_vm[d] = vm;
    w.md_dpc[d] = w.ms_dpc[s];
    w.md_pte[d] = w.ms_pte[s];
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
    w.md_x[d] = x;
    w.md_y[d] = y;
    w.md_z[d] = w.bz[lo];
    w.md_r[d] = r;
    w.md_rlo[d] = r > 0.f ? rlo : 0.f;
    w.md_sthr[d] = c.two_rthr * asinf(fminf(r / c.two_rthr, 1.0f));
    w.md_alpha[d] = asinf(fminf(r * c.k2p, c.sin_max));
    w.md_ec[d] = g.endcap[vm % g.n_mods];
  }
}

// ---------------------------------------------------------------------------------------------
// Line Segments
// ---------------------------------------------------------------------------------------------
constexpr int kLsA = 32;           // inner MDs staged per chunk
constexpr int kLsB = 384;          // outer MDs staged per chunk
constexpr int kMaxTargets = 256;   // module-map degree limit (checked when loading the geometry)

__device__ __forceinline__ int md_count(const Ws& w, int vm) { return w.md_off[vm + 1] - w.md_off[vm]; }

// LS capacity of each module (exact bound: its MDs x the MDs of its connected modules) and its
// cost bucket floor(log2(bound)) for the persistent kernel's work list
__global__ void k_ls_caps(Ws w, Geo g) {
  __shared__ int hist[32];
  if (threadIdx.x < 32) hist[threadIdx.x] = 0;
  __syncthreads();
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const int m = vm % g.n_mods, e0 = vm - m;
    const long long na = md_count(w, vm);
    long long nb = 0;
    if (na > 0)
      for (int k = g.conn_off[m]; k < g.conn_off[m + 1]; ++k) nb += md_count(w, e0 + g.conn_tgt[k]);
    const long long bound = na * nb;
    const double pred = w.cap_scale * (32.0 + 0.5 * (double)bound);
    const int cc = clamp_cap(pred, bound, w.ls_ovr[vm]);
    w.ls_cap[vm] = cc;
    w.ls_base[vm] = cc;
    int b = -1;
    if (bound > 0) {
      b = 63 - __clzll((unsigned long long)bound);
      if (b > 31) b = 31;
      atomicAdd(&hist[b], 1);
    }
    w.work_bucket[vm] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(&w.work_cnt[threadIdx.x], hist[threadIdx.x]);
}

// offsets of the cost buckets, most expensive first
__global__ void k_ls_work_scan(Ws w) {
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 31; b >= 0; --b) {
      w.work_off[b] = acc;
      acc += w.work_cnt[b];
    }
    w.work_off[32] = acc;
  }
}

__global__ void k_ls_work_fill(Ws w) {
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const int b = w.work_bucket[vm];
    if (b >= 0) w.work[w.work_off[b] + atomicAdd(&w.work_cur[b], 1)] = vm;
  }
}

// One block per module at a time: stage the module's MDs (A) and all MDs of its connected modules
// (B) in shared memory, then evaluate every (a, b) pair across the block. Persistent mode: the grid
// is sized to the GPU and blocks pull modules from the cost-ordered work list; otherwise a
// grid-stride loop over all modules.
__global__ void __launch_bounds__(256) k_ls(Ws w, Geo g, Cst<float> c, int persistent) {
  __shared__ float ax[kLsA], ay[kLsA], az[kLsA], ar[kLsA], as_[kLsA], aal[kLsA];
  __shared__ int aid[kLsA];
  __shared__ uint8_t aec[kLsA];
  __shared__ float bx[kLsB], by[kLsB], bz[kLsB], br[kLsB], bs[kLsB], bal[kLsB];
  __shared__ int bid[kLsB];
  __shared__ uint8_t bec[kLsB];
  __shared__ int tpre[kMaxTargets + 1];
  __shared__ int tbase[kMaxTargets];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const int n_items = persistent ? w.work_off[32] : w.V;
  for (int it = blockIdx.x;; it += gridDim.x) {
    int vm;
    if (persistent) {
      if (tid == 0) s_item = atomicAdd(w.work_ctr, 1);
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= n_items) break;
      vm = w.work[item];
    } else {
      if (it >= n_items) break;
      vm = it;
    }
    const int na = md_count(w, vm);
    if (na == 0) continue;
    const int m = vm % g.n_mods, e0 = vm - m;
    const int t0 = g.conn_off[m];
    const int nt = min(g.conn_off[m + 1] - t0, kMaxTargets);
    for (int t = tid; t < nt; t += blockDim.x) {
      const int vb = e0 + g.conn_tgt[t0 + t];
      tbase[t] = w.md_off[vb];
      tpre[t + 1] = md_count(w, vb);
    }
    __syncthreads();
    if (tid == 0) {
      tpre[0] = 0;
      for (int t = 0; t < nt; ++t) tpre[t + 1] += tpre[t];
    }
    __syncthreads();
    const int totB = tpre[nt];
    const int cap = w.ls_cap[vm], base = w.ls_base[vm];
    const int a_begin = w.md_off[vm];
    for (int a0 = 0; totB > 0 && a0 < na; a0 += kLsA) {
      const int nA = min(kLsA, na - a0);
      if (tid < nA) {
        const int d = a_begin + a0 + tid;
        ax[tid] = w.md_x[d]; ay[tid] = w.md_y[d]; az[tid] = w.md_z[d];
        ar[tid] = w.md_r[d]; as_[tid] = w.md_sthr[d]; aec[tid] = w.md_ec[d]; aid[tid] = d;
        aal[tid] = w.md_alpha[d];
      }
      for (int b0 = 0; b0 < totB; b0 += kLsB) {
        const int nB = min(kLsB, totB - b0);
        for (int j = tid; j < nB; j += blockDim.x) {
          const int gj = b0 + j;
          int lo = 0, hi = nt;   // target k with tpre[k] <= gj < tpre[k+1]
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tpre[mid] <= gj) lo = mid; else hi = mid;
          }
          const int d = tbase[lo] + (gj - tpre[lo]);
          bx[j] = w.md_x[d]; by[j] = w.md_y[d]; bz[j] = w.md_z[d];
          br[j] = w.md_r[d]; bs[j] = w.md_sthr[d]; bec[j] = w.md_ec[d]; bid[j] = d;
          bal[j] = w.md_alpha[d];
        }
        __syncthreads();
        const int np = nA * nB;
        for (int p0 = 0; p0 < np; p0 += blockDim.x) {
          const int p = p0 + tid;
          int v = kReject, ia = 0, ib = 0;
          float z0 = 0.f, dphi = 0.f;
          if (p < np) {
            ia = p / nB;
            ib = p - ia * nB;
            // azimuth quick reject: |dphi| >= |sin dphi| = |p1 x p2| / (r1 r2), against an upper
            // bound of the window (alpha difference + resolution and d0 terms with 1/r1 + 1/r2)
            const float cr = ax[ia] * by[ib] - ay[ia] * bx[ib];
            const float r1 = ar[ia], r2 = br[ib];
            const float inv = 1.0f / r1 + 1.0f / r2;
            const float bup = (bal[ib] - aal[ia]) + c.n_sigma * c.sigma_rphi * inv + c.d0_max * inv + 1e-5f;
            if (fabsf(cr) > r1 * r2 * bup * 1.0001f + 1e-6f) v = kReject;
            else
              v = ls_eval<float>(c, ax[ia], ay[ia], az[ia], r1, as_[ia], aec[ia] != 0, bx[ib], by[ib], bz[ib], r2,
                                 bs[ib], bec[ib] != 0, kGuardWindow, z0, dphi);
          }
          const int slot = warp_agg_slot(v == kAccept, &w.ls_cnt[vm]);
          if (slot >= 0 && slot < cap && (int64_t)base + slot < w.cap.ls_slots) {
            w.lss_in[base + slot] = aid[ia];
            w.lss_out[base + slot] = bid[ib];
            w.lss_z0[base + slot] = z0;
            w.lss_dphi[base + slot] = dphi;
          }
          const int q = warp_agg_slot(v == kUnsure, &w.status[ST_Q_LS]);
          if (q >= 0 && q < w.cap.q_ls) w.q_ls[q] = make_int4(vm, aid[ia], bid[ib], 0);
        }
        __syncthreads();
      }
    }
    __syncthreads();   // tpre / tbase are rewritten for the next module
  }
}

__device__ __forceinline__ void md_anchor64(const Ws& w, const Cst<double>& c, int d, double& x,
                                            double& y, double& z, double& r, double& s) {
  x = w.md_x[d]; y = w.md_y[d]; z = w.md_z[d];
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
      w.lss_z0[base + slot] = (float)z0;
      w.lss_dphi[base + slot] = (float)dphi;
    }
  }
}

// dense LS ordered by (inner MD, outer MD); z0 is recomputed in float64 (its float32 form
// amplifies radius rounding up to ~20x for endcap pairs)
__global__ void k_ls_dense(Ws w) {
  const int n = (int)lst_min64(w.ls_off[w.V], w.cap.ls_dense);
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
    const int s = w.perm[d];
    const int a = w.lss_in[s], b = w.lss_out[s];
    w.ls_in[d] = a;
    w.ls_out[d] = b;
    // z0 = (z1 r2 - z2 r1) / (r2 - r1) with the radii in float-float: the float32 rounding of the
    // radii would be amplified up to ~20x for endcap pairs
    const float z1 = w.md_z[a], z2 = w.md_z[b];
    const float r1 = w.md_r[a], r1l = w.md_rlo[a], r2 = w.md_r[b], r2l = w.md_rlo[b];
    const float num = diff_prod(z1, r2, z2, r1) + (z1 * r2l - z2 * r1l);
    const float den = (r2 - r1) + (r2l - r1l);
    w.ls_z0[d] = num / den;
    w.ls_dphi[d] = w.lss_dphi[s];
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

void launch_effective(const Ws& w, const int32_t* cnt, const int32_t* cap, const int32_t* base,
                      int64_t slots, int32_t* eff, int ovf_word, int arena_word, int n, const Launch& L) {
  k_effective<<<grid_for(n, 256), 256, 0, L.stream>>>(w, cnt, cap, base, slots, eff, ovf_word, arena_word, n);
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
  k_bin_sort_gather<<<grid_for(w.S, 128), 128, 0, L.stream>>>(w, n_sens);
  KT_END(L, K_BIN);
  LST_LAUNCH(L);
}

void run_md(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  k_md_caps<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w);
  LST_LAUNCH(L);
  scan_exclusive(w.md_base, w.md_base, w.V, w.scan_tmp, L);
  KT_BEGIN(L, K_MD);
  k_md<<<grid_for((int64_t)w.V * 32, 256), 256, 0, L.stream>>>(w, g, c.f);
  KT_END(L, K_MD);
  LST_LAUNCH(L);
  k_md_recheck<<<grid_for(w.cap.q_md, 128, 152 * 4), 128, 0, L.stream>>>(w, g, c.d);
  LST_LAUNCH(L);
  KT_BEGIN(L, K_MD_COMPACT);
  GroupArgs ga{w.md_cnt, w.md_cap, w.md_base, w.cap.md_slots, ST_OVF_MD, ST_ARENA_MD, w.ms_lo, w.ms_up,
               w.mdlo_cnt, w.mdlo_cur, w.mdlo_off, w.cap.H, w.cap.md_dense, ST_DENSE_MD,
               w.md_off, w.sens_off, 2};
  group_slots(w, ga, L);
  k_md_dense<<<grid_for(w.cap.md_dense, 256), 256, 0, L.stream>>>(w, g, c.f);
  KT_END(L, K_MD_COMPACT);
  LST_LAUNCH(L);
}

void run_ls(const Ws& w, const Geo& g, const Consts& c, const Launch& L) {
  k_ls_caps<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w, g);
  LST_LAUNCH(L);
  scan_exclusive(w.ls_base, w.ls_base, w.V, w.scan_tmp, L);
  if (L.persistent) {
    k_ls_work_scan<<<1, 32, 0, L.stream>>>(w);
    k_ls_work_fill<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w);
    *L.launches += 2;
  }
  KT_BEGIN(L, K_LS);
  if (L.persistent) k_ls<<<L.n_sm * (2048 / L.block_ls), L.block_ls, 0, L.stream>>>(w, g, c.f, 1);
  else k_ls<<<grid_for(w.V, 1, 152 * 16), L.block_ls, 0, L.stream>>>(w, g, c.f, 0);
  KT_END(L, K_LS);
  LST_LAUNCH(L);
  k_ls_recheck<<<grid_for(w.cap.q_ls, 128, 152 * 4), 128, 0, L.stream>>>(w, c.d);
  LST_LAUNCH(L);
  // LS ordered by inner MD: the per-MD group offsets are the "LS by inner MD" adjacency
  KT_BEGIN(L, K_LS_COMPACT);
  GroupArgs ga{w.ls_cnt, w.ls_cap, w.ls_base, w.cap.ls_slots, ST_OVF_LS, ST_ARENA_LS, w.lss_in, w.lss_out,
               w.lsin_cnt, w.lsin_cur, w.lsin_off, w.cap.md_dense, w.cap.ls_dense, ST_DENSE_LS,
               w.ls_off, w.md_off, 1};
  group_slots(w, ga, L);
  k_ls_dense<<<grid_for(w.cap.ls_dense, 256), 256, 0, L.stream>>>(w);
  KT_END(L, K_LS_COMPACT);
  LST_LAUNCH(L);
}

}  // namespace lst
