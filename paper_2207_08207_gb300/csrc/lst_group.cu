// Ordered compaction of per-module capacity slots into dense arrays.
//
// Each stage writes its objects into per-module slots (order inside a module set by atomics). The
// dense arrays are ordered by (first member, second member). The first members of a module's
// objects lie in that module's own range of first-member indices (the previous stage's dense
// objects, or the module's binned hits for MDs), and those ranges increase with the module, so this
// order is also the module order, and the objects sharing a first member form one contiguous group.
// Groups may also be coarser, by a monotone map of the first member (T3 by the inner MD of their
// inner LS): the order inside a group is then by (first, second) member.
// The compaction therefore works per object, with no per-module sort:
//   1. count the objects of every first member (atomics on a key-indexed array, done by the kernels
//      that store the objects);
//   2. exclusive scan: the start of every group, which are also the per-key group offsets that the
//      next stage uses as its adjacency ("objects whose first member is below k");
//   3. place each object at its group's cursor (order inside a group arbitrary);
//   4. rank each object inside its group by the second member (groups are small: a few objects,
//      ranked against each other in shared memory).
// The key-indexed arrays are zeroed and scanned up to the actual key count, read on the device, so
// that the launches stay shaped by capacities (one CUDA graph serves every batch).
// The per-module dense offsets are the group offsets of each module's first key.
#include <cassert>

#include "lst_internal.h"

namespace lst {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGrpWarps = 8;   // warps per block of the slot-visiting kernels

// Visit every valid slot of up to 32 modules with all lanes of the warp, two slots per lane at a
// time so that the work of both (their loads and atomics) is in flight together. eff and b are the
// lane's module's valid-slot count and slot base (0 on lanes without a module); f(valid_a, s_a,
// valid_b, s_b) is called by all lanes together, and every valid slot comes once with valid = true.
template <class F>
__device__ __forceinline__ void visit_slots2(int lane, int eff, int b, F&& f) {
  int incl = eff;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  for (int i0 = 0; i0 < total; i0 += 64) {
    const int ia = i0 + lane, ib = i0 + 32 + lane;
    int ja = 0, jb = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int va = __shfl_sync(kFull, incl, ja + step - 1);
      const int vb = __shfl_sync(kFull, incl, jb + step - 1);
      if (va <= ia) ja += step;
      if (vb <= ib) jb += step;
    }
    const int sa = __shfl_sync(kFull, b, ja) + ia - (__shfl_sync(kFull, incl, ja) - __shfl_sync(kFull, eff, ja));
    const int sb = __shfl_sync(kFull, b, jb) + ib - (__shfl_sync(kFull, incl, jb) - __shfl_sync(kFull, eff, jb));
    f(ia < total, sa, ib < total, sb);
  }
}

// the group of an object with first member k1: k1 itself, or key_map[k1]; inside [0, nk) (they all
// are, unless an earlier stage overflowed)
__device__ __forceinline__ int group_of(const GroupArgs& a, int k1, int nk) {
  const int g = a.key_map ? a.key_map[k1] : k1;
  return max(min(g, nk - 1), 0);
}

// per-module valid slots = min(count, capacity, arena room), the excess recorded
__global__ void k_grp_eff(Ws w, GroupArgs a) {
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const int c = a.cnt[vm], k = a.cap[vm], b = a.base[vm];
    int eff = min(c, k);
    if (c > k) atomicAdd(&w.status[a.ovf_word], c - k);
    if ((int64_t)b + eff > a.slots) {
      eff = (int)(a.slots - b > 0 ? a.slots - b : 0);
      atomicMax(&w.status[a.arena_word], a.base[w.V]);
    }
    w.eff[vm] = eff + 1;   // a module weighs its valid objects plus one (its visit)
  }
}

// Work is split into tasks of about `chunk` units of weight (a module weighs its valid objects plus
// one, so that long runs of empty modules are split too): task t holds the modules whose weighted
// start (the scan of the weights, eff_off) lies in [t * chunk, (t + 1) * chunk). grp_task[t] is its
// first module: the first vm with eff_off[vm] >= t * chunk.
__global__ void k_grp_tasks(Ws w, int chunk) {
  const int total = w.eff[w.V];
  const int n_tasks = (total + chunk - 1) / chunk;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= n_tasks; t += gridDim.x * blockDim.x) {
    const int64_t target = (int64_t)t * chunk;
    int lo = 0, hi = w.V;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (w.eff[mid] < target) lo = mid + 1; else hi = mid;
    }
    w.grp_task[t] = lo;
  }
}

// all lanes of a warp visit the valid slots of task t's modules, 32 modules at a time
template <class F>
__device__ __forceinline__ void visit_task(const Ws& w, const GroupArgs& a, int t, int lane, F&& f) {
  const int m_end = w.grp_task[t + 1];
  for (int m0 = w.grp_task[t]; m0 < m_end; m0 += 32) {
    const int vm = m0 + lane;
    int eff = 0, b = 0;
    if (vm < m_end) {
      eff = w.eff[vm + 1] - w.eff[vm] - 1;
      b = a.base[vm];
    }
    visit_slots2(lane, eff, b, f);
  }
}

// warp_agg_slot_keyed for two (pred, key) sets at once, both atomics issued before either result is
// used
__device__ __forceinline__ void warp_agg_slot_keyed2(bool pa, int ka, bool pb, int kb, int* counters, int& sa,
                                                     int& sb) {
  const int lane = threadIdx.x & 31;
  const unsigned ma = __ballot_sync(kFull, pa), mb = __ballot_sync(kFull, pb);
  unsigned ga = 0, gb = 0;
  if (pa) ga = __match_any_sync(ma, ka);
  if (pb) gb = __match_any_sync(mb, kb);
  const int la = pa ? __ffs(ga) - 1 : 0, lb = pb ? __ffs(gb) - 1 : 0;
  int base_a = 0, base_b = 0;
  if (pa && lane == la) base_a = atomicAdd(&counters[ka], __popc(ga));
  if (pb && lane == lb) base_b = atomicAdd(&counters[kb], __popc(gb));
  base_a = __shfl_sync(kFull, base_a, la);
  base_b = __shfl_sync(kFull, base_b, lb);
  const unsigned below = (1u << lane) - 1u;
  sa = pa ? base_a + __popc(ga & below) : -1;
  sb = pb ? base_b + __popc(gb & below) : -1;
}

// Pass 3: after the exclusive scan E[k + 1] is the start of group k; each object takes the next
// position of its group. Afterwards E[k] is the start of group k for every k (E[0] stays 0).
__global__ void __launch_bounds__(32 * kGrpWarps, 8) k_grp_place(Ws w, GroupArgs a, int32_t* E, int chunk) {
  const int lane = threadIdx.x & 31;
  const int nk = *a.n_keys_dev;
  const int n_tasks = (w.eff[w.V] + chunk - 1) / chunk;   // (of the weights)
  for (int t = blockIdx.x * kGrpWarps + (threadIdx.x >> 5); t < n_tasks; t += gridDim.x * kGrpWarps)
    visit_task(w, a, t, lane, [&](bool va, int sa, bool vb, int sb) {
      const int k1a = va ? a.key1[sa] : 0, k1b = vb ? a.key1[sb] : 0;
      const int k2a = va ? a.key2[sa] : 0, k2b = vb ? a.key2[sb] : 0;
      int pa, pb;
      warp_agg_slot_keyed2(va, va ? group_of(a, k1a, nk) + 1 : 0, vb, vb ? group_of(a, k1b, nk) + 1 : 0, E, pa,
                           pb);
      if (va && pa >= 0 && pa < a.dense_cap) {
        w.grp_pos[pa] = sa;
        w.grp_key12[pa] = make_int2(k1a, k2a);
      }
      if (vb && pb >= 0 && pb < a.dense_cap) {
        w.grp_pos[pb] = sb;
        w.grp_key12[pb] = make_int2(k1b, k2b);
      }
    });
}

// Pass 4: the rank of each placed object inside its group by (second member, slot), which gives its
// dense position; the permutation (or, for LS and T3, the dense objects themselves) is written there, with
// the per-module dense offsets and the dense-overflow word. A block ranks a
// tile of kRankTile positions with the (slot, second member) of the tile and kRankHalo positions on
// each side in shared memory; groups reaching further (none at the sizes seen) read memory.
constexpr int kRankTile = 256, kRankHalo = 64;

template <int OUT>
__global__ void __launch_bounds__(kRankTile) k_grp_rank(Ws w, GroupArgs a, const int32_t* E) {
  __shared__ int sh_s[kRankTile + 2 * kRankHalo];
  __shared__ int sh_k1[kRankTile + 2 * kRankHalo];   // (only with a key map: else equal in a group)
  __shared__ int sh_k2[kRankTile + 2 * kRankHalo];
  const bool mapped = a.key_map != nullptr;
  const int nk = *a.n_keys_dev;
  const int total = E[nk];
  const int n = (int)lst_min64(total, a.dense_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > a.dense_cap) atomicMax(&w.status[a.dense_word], total);
  for (int t0 = blockIdx.x * kRankTile; t0 < n; t0 += gridDim.x * kRankTile) {
    for (int i = threadIdx.x; i < kRankTile + 2 * kRankHalo; i += kRankTile) {
      const int q = t0 - kRankHalo + i;
      if (q >= 0 && q < n) {
        sh_s[i] = w.grp_pos[q];
        const int2 kq = w.grp_key12[q];
        sh_k1[i] = kq.x;
        sh_k2[i] = kq.y;
      }
    }
    __syncthreads();
    const int p = t0 + threadIdx.x;
    const bool valid = p < n;
    int s = 0, k1 = 0, k2 = 0, d = 0;
    if (valid) {
      s = sh_s[kRankHalo + threadIdx.x];
      k1 = sh_k1[kRankHalo + threadIdx.x];
      k2 = sh_k2[kRankHalo + threadIdx.x];
      const int g = group_of(a, k1, nk);
      const int g_beg = E[g], g_end = (int)lst_min64(E[g + 1], n);
      int r = 0;   // members before this one: by (first, second) member, then slot
      if (g_beg >= t0 - kRankHalo && g_end <= t0 + kRankTile + kRankHalo) {
        const int i0 = g_beg - (t0 - kRankHalo), i1 = g_end - (t0 - kRankHalo);
        if (mapped) {
          for (int i = i0; i < i1; ++i) {
            const int q1 = sh_k1[i], q2 = sh_k2[i], sq = sh_s[i];
            r += q1 < k1 || (q1 == k1 && (q2 < k2 || (q2 == k2 && sq < s)));
          }
        } else {
          for (int i = i0; i < i1; ++i) {
            const int q2 = sh_k2[i], sq = sh_s[i];
            r += q2 < k2 || (q2 == k2 && sq < s);
          }
        }
      } else {
        for (int q = g_beg; q < g_end; ++q) {
          const int sq = w.grp_pos[q];
          const int2 kq = w.grp_key12[q];
          r += kq.x < k1 || (kq.x == k1 && (kq.y < k2 || (kq.y == k2 && sq < s)));
        }
      }
      d = g_beg + r;
    }
    if (OUT == kDenseLs) ls_dense_write(w, valid, d, s, k1, k2, E, n);
    else if (OUT == kDenseT3) t3_dense_write(w, valid, d, s, k1, k2, E, n);
    else if (valid) w.perm[d] = s;
    __syncthreads();
  }
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm <= w.V; vm += gridDim.x * blockDim.x)
    a.mod_off[vm] = (int)lst_min64(E[a.mod_first[(int64_t)vm * a.mod_first_stride]], a.dense_cap);
}

}  // namespace

void group_slots(const Ws& w, const GroupArgs& a, const Launch& L) {
  assert(a.dense_out == kDensePerm || a.dense_out == kDenseLs || a.dense_out == kDenseT3);
  int32_t* E = a.grp_off ? a.grp_off : w.grp_key;
  // objects per warp task: about two tasks per resident warp at the stage's dense capacity
  const int64_t resident_warps = (int64_t)L.n_sm * 64;
  int chunk = 64;
  while (chunk < 1024 && (int64_t)chunk * 2 * resident_warps * 2 <= a.dense_cap + w.V) chunk *= 2;
  const int blocks = L.n_sm * (64 / kGrpWarps);
  k_grp_eff<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w, a);
  LST_LAUNCH(L);
  if (!scan_tasks(w.eff, w.V, w.grp_task, chunk, L)) {
    scan_exclusive(w.eff, w.eff, w.V, w.scan_tmp, L);
    k_grp_tasks<<<grid_for((a.slots + w.V) / chunk + 2, 256), 256, 0, L.stream>>>(w, chunk);
    LST_LAUNCH(L);
  }
  scan_exclusive_dev(E, E, a.n_keys + 1, a.n_keys_dev, 1, w.scan_tmp, L);
  k_grp_place<<<blocks, 32 * kGrpWarps, 0, L.stream>>>(w, a, E, chunk);
  LST_LAUNCH(L);
  if (a.dense_out == kDenseLs) k_grp_rank<kDenseLs><<<L.n_sm * 8, kRankTile, 0, L.stream>>>(w, a, E);
  else if (a.dense_out == kDenseT3) k_grp_rank<kDenseT3><<<L.n_sm * 8, kRankTile, 0, L.stream>>>(w, a, E);
  else k_grp_rank<kDensePerm><<<L.n_sm * 8, kRankTile, 0, L.stream>>>(w, a, E);
  LST_LAUNCH(L);
  // (after a dense overflow, the next stage's capacity kernel clamps the group offsets it reads)
}

}  // namespace lst
