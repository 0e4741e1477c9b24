// Ordered compaction of per-module capacity slots into dense arrays.
//
// Each stage writes its objects into per-module slots (order inside a module set by atomics). The
// dense arrays are ordered by (first member, second member). The first members of a module's
// objects lie in that module's own range of first-member indices (the previous stage's dense
// objects, or the module's binned hits for MDs), and those ranges increase with the module, so the
// global order is the module order with each module's objects sorted on their own: the per-module
// dense offsets are an exclusive scan of the per-module counts, and each module sorts its few
// objects locally (a warp for most modules, a block for the largest) by a counting sort on the first
// member followed by ranks inside each first-member group. The per-key group offsets (objects whose first member is below a key) follow from the
// sorted keys by binary search.
#include "lst_internal.h"

namespace lst {
namespace {

constexpr int kSmallWarps = 8;        // warps per block of the small-module kernel
constexpr int kBigThreads = 256;      // threads per block of the large-module kernel
constexpr int kBigCap = 8192;         // objects a large module sorts in shared memory

// valid slots per module = min(count, capacity, arena room); the excess is recorded
__global__ void k_mod_eff(Ws w, const int32_t* cnt, const int32_t* cap, const int32_t* base, int64_t slots,
                          int ovf_word, int arena_word) {
  for (int vm = blockIdx.x * blockDim.x + threadIdx.x; vm < w.V; vm += gridDim.x * blockDim.x) {
    const int c = cnt[vm], k = cap[vm], b = base[vm];
    int eff = min(c, k);
    if (c > k) atomicAdd(&w.status[ovf_word], c - k);
    if ((int64_t)b + eff > slots) {
      eff = (int)(slots - b > 0 ? slots - b : 0);
      atomicMax(&w.status[arena_word], base[w.V]);
    }
    w.eff[vm] = eff;
  }
}

__device__ __forceinline__ unsigned long long pair_key(int k1, int k2) {
  return ((unsigned long long)(unsigned)k1 << 32) | (unsigned)k2;
}

struct SortArgs {
  const int32_t *base, *key1, *key2, *mod_first;
  int stride;
  int32_t* grp_off;
  int64_t n_keys, dense_cap;
  int32_t* mod_off;
  int dense_word, big_word;
};

// Modules of moderate size: a warp per module. Up to 32 objects each lane holds one and ranks it
// against the others by shuffles. Up to kMidCap objects whose first members span at most kMidCap
// keys, a counting sort in shared memory: histogram of the first members, its scan (which is the
// group offsets), placement, then each object's rank inside its first-member group by its second
// member (groups hold a few objects). Larger modules are listed for k_mod_sort_big.
constexpr int kMidCap = 512;

__global__ void __launch_bounds__(32 * kSmallWarps) k_mod_sort_small(Ws w, SortArgs a) {
  __shared__ int sh_k2[kSmallWarps][kMidCap];    // second member of each object
  __shared__ int sh_pos[kSmallWarps][kMidCap];   // objects placed by first member
  __shared__ int sh_g[kSmallWarps][kMidCap];     // group counts, then group starts (R + 1 <= kMidCap)
  const int wi = threadIdx.x >> 5;
  int* K2 = sh_k2[wi];
  int* POS = sh_pos[wi];
  int* G = sh_g[wi];
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kSmallWarps;
  const int64_t cap = a.dense_cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int total = w.eff[w.V];
    if (total > cap) atomicMax(&w.status[a.dense_word], total);
    a.mod_off[w.V] = (int)lst_min64(total, cap);
  }
  const bool offsets = a.grp_off != nullptr;
  for (int vm = blockIdx.x * kSmallWarps + wi; vm < w.V; vm += nwarps) {
    const int dest = w.eff[vm], n = w.eff[vm + 1] - dest;
    if (lane == 0) a.mod_off[vm] = (int)lst_min64(dest, cap);
    const int k0 = a.mod_first[(int64_t)vm * a.stride], k1 = a.mod_first[(int64_t)(vm + 1) * a.stride];
    const int R = k1 - k0;
    if (n > 32 && (n > kMidCap || R >= kMidCap)) {
      if (lane == 0) w.grp_big[atomicAdd(&w.grp_big_cnt[a.big_word], 1)] = vm;
      continue;
    }
    if (n == 0 && !(offsets && R > 0)) continue;
    const int b = a.base[vm];
    if (n <= 32) {
      int kv1 = 0x7fffffff;
      unsigned long long key = ~0ull;
      if (lane < n) {
        kv1 = a.key1[b + lane];
        key = pair_key(kv1, a.key2[b + lane]);
      }
      int rank = 0;
      for (int j = 0; j < n; ++j) {
        const unsigned long long kj = __shfl_sync(0xffffffffu, key, j);
        rank += kj < key || (kj == key && j < lane);
      }
      if (lane < n) {
        if (dest + rank < cap) w.perm[dest + rank] = b + lane;
        POS[rank] = kv1;
      }
      __syncwarp();
      if (offsets)
        for (int k = k0 + lane; k < k1; k += 32) {   // dest + #(first members below k)
          int lo = 0, hi = n;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (POS[mid] < k) lo = mid + 1; else hi = mid;
          }
          a.grp_off[k] = (int)lst_min64(dest + lo, cap);
        }
      __syncwarp();
      continue;
    }
    for (int k = lane; k <= R; k += 32) G[k] = 0;
    __syncwarp();
    const int gmax = R > 0 ? R - 1 : 0;   // (first members outside the range only after an overflow)
    for (int i = lane; i < n; i += 32) {
      K2[i] = a.key2[b + i];
      atomicAdd(&G[min(max(a.key1[b + i] - k0, 0), gmax)], 1);
    }
    __syncwarp();
    int run = 0;   // exclusive scan of G[0..R] in chunks of 32
    for (int k0c = 0; k0c <= R; k0c += 32) {
      const int k = k0c + lane;
      const int v = k <= R ? G[k] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (k <= R) G[k] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    if (offsets)
      for (int k = lane; k < R; k += 32) a.grp_off[k0 + k] = (int)lst_min64(dest + G[k], cap);
    // placement by first member (order inside a group arbitrary), via the group starts
    for (int i = lane; i < n; i += 32) POS[atomicAdd(&G[min(max(a.key1[b + i] - k0, 0), gmax)], 1)] = i;
    __syncwarp();
    // G[g] is now the end of group g: rank inside the group by the second member
    for (int p = lane; p < n; p += 32) {
      const int i = POS[p];
      const int g = min(max(a.key1[b + i] - k0, 0), gmax);
      const int g_end = G[g], g_beg = g > 0 ? G[g - 1] : 0;
      const int k2 = K2[i];
      int r = g_beg;
      for (int qq = g_beg; qq < g_end; ++qq) {
        const int j = POS[qq];
        const int kj = K2[j];
        r += kj < k2 || (kj == k2 && j < i);
      }
      if (dest + r < cap) w.perm[dest + r] = b + i;
    }
    __syncwarp();
  }
}

// Larger modules: a block per module, the same counting sort with the block (up to kBigCap objects
// and first-member ranges below kBigCap); beyond that, ranks counted directly from global memory.
__global__ void __launch_bounds__(kBigThreads) k_mod_sort_big(Ws w, SortArgs a) {
  extern __shared__ __align__(16) unsigned char big_smem[];
  int* K2 = reinterpret_cast<int*>(big_smem);   // [kBigCap] second members
  int* POS = K2 + kBigCap;                     // [kBigCap] objects placed by first member
  int* G = POS + kBigCap;                      // [kBigCap] group counts, then starts, then ends
  __shared__ int part[kBigThreads];
  const int n_big = w.grp_big_cnt[a.big_word];
  const int64_t cap = a.dense_cap;
  const int t = threadIdx.x;
  for (int it = blockIdx.x; it < n_big; it += gridDim.x) {
    const int vm = w.grp_big[it];
    const int dest = w.eff[vm], n = w.eff[vm + 1] - dest;
    const int b = a.base[vm];
    const int k0 = a.mod_first[(int64_t)vm * a.stride], k1 = a.mod_first[(int64_t)(vm + 1) * a.stride];
    const int R = k1 - k0;
    if (n <= kBigCap && R < kBigCap) {
      const int gmax = R > 0 ? R - 1 : 0;
      for (int k = t; k <= R; k += blockDim.x) G[k] = 0;
      __syncthreads();
      for (int i = t; i < n; i += blockDim.x) {
        K2[i] = a.key2[b + i];
        atomicAdd(&G[min(max(a.key1[b + i] - k0, 0), gmax)], 1);
      }
      __syncthreads();
      // exclusive scan of G[0..R]: each thread a contiguous run, then a scan of the run totals
      const int per = (R + 1 + blockDim.x - 1) / blockDim.x;
      const int r0 = t * per, r1 = min(r0 + per, R + 1);
      int sum = 0;
      for (int k = r0; k < r1; ++k) sum += G[k];
      part[t] = sum;
      __syncthreads();
      if (t < 32) {
        int run = 0;
        for (int c0 = 0; c0 < kBigThreads; c0 += 32) {
          const int v = part[c0 + t];
          int incl = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (t >= o) incl += y;
          }
          part[c0 + t] = run + incl - v;
          run += __shfl_sync(0xffffffffu, incl, 31);
        }
      }
      __syncthreads();
      int acc = part[t];
      for (int k = r0; k < r1; ++k) {
        const int v = G[k];
        G[k] = acc;
        acc += v;
      }
      __syncthreads();
      if (a.grp_off)
        for (int k = t; k < R; k += blockDim.x) a.grp_off[k0 + k] = (int)lst_min64(dest + G[k], cap);
      __syncthreads();
      for (int i = t; i < n; i += blockDim.x) POS[atomicAdd(&G[min(max(a.key1[b + i] - k0, 0), gmax)], 1)] = i;
      __syncthreads();
      for (int p = t; p < n; p += blockDim.x) {   // G[g] is now the end of group g
        const int i = POS[p];
        const int g = min(max(a.key1[b + i] - k0, 0), gmax);
        const int g_end = G[g], g_beg = g > 0 ? G[g - 1] : 0;
        const int k2 = K2[i];
        int r = g_beg;
        for (int q = g_beg; q < g_end; ++q) {
          const int j = POS[q];
          const int kj = K2[j];
          r += kj < k2 || (kj == k2 && j < i);
        }
        if (dest + r < cap) w.perm[dest + r] = b + i;
      }
      __syncthreads();
    } else {
      for (int i = t; i < n; i += blockDim.x) {
        const unsigned long long ki = pair_key(a.key1[b + i], a.key2[b + i]);
        int rank = 0;
        for (int j = 0; j < n; ++j) {
          const unsigned long long kj = pair_key(a.key1[b + j], a.key2[b + j]);
          rank += kj < ki || (kj == ki && j < i);
        }
        if (dest + rank < cap) w.perm[dest + rank] = b + i;
      }
      for (int k = k0 + t; a.grp_off && k < k1; k += blockDim.x) {
        int below = 0;
        for (int j = 0; j < n; ++j) below += a.key1[b + j] < k;
        a.grp_off[k] = (int)lst_min64(dest + below, cap);
      }
    }
  }
}

// group offsets of the keys past the last module's range: the (clamped) total
__global__ void k_grp_tail(Ws w, SortArgs a) {
  const int k_end = a.mod_first[(int64_t)w.V * a.stride];
  const int total = (int)lst_min64(w.eff[w.V], a.dense_cap);
  for (int64_t k = k_end + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= a.n_keys;
       k += (int64_t)gridDim.x * blockDim.x)
    a.grp_off[k] = total;
}

// out[i] = min(grp_off[first[i * stride]], cap), i in [0, n] (the clamp keeps later stages inside
// the dense arrays when they overflowed; the run is then retried with larger ones)
__global__ void k_off_compose(int32_t* out, int n, const int32_t* first, int stride, const int32_t* grp_off,
                              int64_t cap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    out[i] = (int)lst_min64(grp_off[first[(int64_t)i * stride]], cap);
}

}  // namespace

void group_configure() {
  cudaFuncSetAttribute(k_mod_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kBigCap * (int)sizeof(int));
}

void group_slots(const Ws& w, const GroupArgs& a, const Launch& L) {
  k_mod_eff<<<grid_for(w.V, 256), 256, 0, L.stream>>>(w, a.cnt, a.cap, a.base, a.slots, a.ovf_word, a.arena_word);
  LST_LAUNCH(L);
  scan_exclusive(w.eff, w.eff, w.V, w.scan_tmp, L);
  SortArgs s{a.base, a.key1, a.key2, a.mod_first, a.mod_first_stride, a.grp_off, a.n_keys, a.dense_cap,
             a.mod_off, a.dense_word, a.big_word};
  k_mod_sort_small<<<grid_for((int64_t)w.V * 32, 32 * kSmallWarps, 152 * 32), 32 * kSmallWarps, 0, L.stream>>>(w, s);
  LST_LAUNCH(L);
  k_mod_sort_big<<<L.n_sm * 2, kBigThreads, 3 * kBigCap * sizeof(int), L.stream>>>(w, s);
  LST_LAUNCH(L);
  if (a.grp_off) {
    k_grp_tail<<<grid_for(a.n_keys + 1, 256), 256, 0, L.stream>>>(w, s);
    LST_LAUNCH(L);
  }
}

void compose_offsets(int32_t* out, int n, const int32_t* first, int stride, const int32_t* grp_off, int64_t cap,
                     const Launch& L) {
  k_off_compose<<<grid_for(n + 1, 256), 256, 0, L.stream>>>(out, n, first, stride, grp_off, cap);
  LST_LAUNCH(L);
}

}  // namespace lst
