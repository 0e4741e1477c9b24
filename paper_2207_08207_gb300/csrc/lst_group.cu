// Ordered compaction of per-module capacity slots into dense arrays.
//
// Each stage writes its objects into per-module slots (order inside a module set by atomics). The
// dense arrays are ordered by (first member, second member): a counting sort by the first member
// (a dense index of the previous stage, or a binned hit index for MDs) followed by an insertion sort
// of each first-member group by the second member. Groups are small (a few objects per MD / LS / T3),
// so the whole step is O(objects). Because the first members are themselves ordered by module, the
// result is also grouped by module, and the per-module offsets are the group offsets of each
// module's first key.
#include "lst_internal.h"

namespace lst {
namespace {

// warp per virtual module: valid slots = min(count, capacity, arena room); count keys
__global__ void k_grp_count(Ws w, const int32_t* cnt, const int32_t* cap, const int32_t* base, int64_t slots,
                            int ovf_word, int arena_word, const int32_t* key1, int32_t* grp_cnt) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int vm = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vm < w.V; vm += nwarps) {
    const int c = cnt[vm], k = cap[vm], b = base[vm];
    int eff = min(c, k);
    if ((int64_t)b + eff > slots) eff = (int)(slots - b > 0 ? slots - b : 0);
    if (lane == 0) {
      if (c > k) atomicAdd(&w.status[ovf_word], c - k);
      if ((int64_t)b + min(c, k) > slots) atomicMax(&w.status[arena_word], base[w.V]);
      w.eff[vm] = eff;
    }
    for (int j = lane; j < eff; j += 32) atomicAdd(&grp_cnt[key1[b + j]], 1);
  }
}

__global__ void k_grp_scatter(Ws w, const int32_t* base, const int32_t* key1, const int32_t* grp_off,
                              int32_t* grp_cur, int64_t dense_cap) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int vm = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vm < w.V; vm += nwarps) {
    const int eff = w.eff[vm], b = base[vm];
    for (int j = lane; j < eff; j += 32) {
      const int s = b + j;
      const int k = key1[s];
      const int pos = grp_off[k] + atomicAdd(&grp_cur[k], 1);
      if (pos < dense_cap) w.perm[pos] = s;
    }
  }
}

__global__ void k_grp_sort(Ws w, const int32_t* grp_off, int64_t n_keys, const int32_t* key2, int64_t dense_cap,
                           int dense_word) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int total = grp_off[n_keys];
    if (total > dense_cap) atomicMax(&w.status[dense_word], total);
  }
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_keys; k += (int64_t)gridDim.x * blockDim.x) {
    const int a = grp_off[k];
    const int b = (int)lst_min64(grp_off[k + 1], dense_cap);
    for (int i = a + 1; i < b; ++i) {
      const int v = w.perm[i];
      const int kv = key2[v];
      int j = i - 1;
      while (j >= a && key2[w.perm[j]] > kv) {
        w.perm[j + 1] = w.perm[j];
        --j;
      }
      w.perm[j + 1] = v;
    }
  }
}

// out[i] = min(grp_off[first[i * stride]], cap), i in [0, n] (the clamp keeps later stages inside
// the dense arrays when they overflowed; the run is then retried with larger ones)
__global__ void k_off_compose(int32_t* out, int n, const int32_t* first, int stride, const int32_t* grp_off,
                              int64_t cap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    out[i] = (int)lst_min64(grp_off[first[(int64_t)i * stride]], cap);
}

}  // namespace

void group_slots(const Ws& w, const GroupArgs& a, const Launch& L) {
  k_grp_count<<<grid_for((int64_t)w.V * 32, 256), 256, 0, L.stream>>>(w, a.cnt, a.cap, a.base, a.slots, a.ovf_word,
                                                                     a.arena_word, a.key1, a.grp_cnt);
  LST_LAUNCH(L);
  scan_exclusive(a.grp_cnt, a.grp_off, a.n_keys, w.scan_tmp, L);
  k_grp_scatter<<<grid_for((int64_t)w.V * 32, 256), 256, 0, L.stream>>>(w, a.base, a.key1, a.grp_off, a.grp_cur,
                                                                       a.dense_cap);
  LST_LAUNCH(L);
  k_grp_sort<<<grid_for(a.n_keys, 256), 256, 0, L.stream>>>(w, a.grp_off, a.n_keys, a.key2, a.dense_cap, a.dense_word);
  LST_LAUNCH(L);
  k_off_compose<<<grid_for(w.V + 1, 256), 256, 0, L.stream>>>(a.mod_off, w.V, a.mod_first, a.mod_first_stride,
                                                             a.grp_off, a.dense_cap);
  LST_LAUNCH(L);
}

void compose_offsets(int32_t* out, int n, const int32_t* first, int stride, const int32_t* grp_off, int64_t cap,
                     const Launch& L) {
  k_off_compose<<<grid_for(n + 1, 256), 256, 0, L.stream>>>(out, n, first, stride, grp_off, cap);
  LST_LAUNCH(L);
}

}  // namespace lst
