// Exclusive prefix sums over int32 counts, used for every count -> offset step of the chain
// (sensor offsets, per-module object offsets, per-key group offsets). Inside a chain run: one
// single-pass kernel per scan (decoupled look-back); elsewhere (the standalone binning entry
// points): three passes (per-tile scan, scan of tile totals, add-back).
#include <vector>

#include "lst_internal.h"

namespace lst {
namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kTile = kScanBlock * kScanItems;

__device__ __forceinline__ int block_excl_scan(int v, int& total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  const int warp_prefix = wid > 0 ? warp_sums[wid - 1] : 0;
  total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

// n_dev (nullable): the entry count is then min(n, *n_dev + n_add), read on the device
__device__ __forceinline__ int64_t scan_count(int64_t n, const int32_t* n_dev, int n_add) {
  return n_dev ? lst_min64(n, (int64_t)*n_dev + n_add) : n;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(const int32_t* in, int32_t* out, int64_t n_max,
                                                           int32_t* tile_sums, const int32_t* n_dev, int n_add) {
  const int64_t n = scan_count(n_max, n_dev, n_add);
  if ((int64_t)blockIdx.x * kTile >= n) {   // a tile past the entries: nothing to scan
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = 0;
    return;
  }
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int local = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    local += v[k];
  }
  int total;
  int pre = block_excl_scan(local, total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(int32_t* tile_sums, int64_t n_tiles, int32_t* out,
                                                          int64_t n_max, const int32_t* n_dev, int n_add) {
  const int64_t n = scan_count(n_max, n_dev, n_add);
  n_tiles = lst_min64(n_tiles, (n + kTile - 1) / kTile);
  int carry = 0;
  for (int64_t b0 = 0; b0 < n_tiles; b0 += kScanBlock) {
    const int64_t i = b0 + threadIdx.x;
    const int v = i < n_tiles ? tile_sums[i] : 0;
    int total;
    const int pre = block_excl_scan(v, total);
    if (i < n_tiles) tile_sums[i] = carry + pre;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_add(int32_t* out, int64_t n_max, const int32_t* tile_sums,
                                                         const int32_t* n_dev, int n_add) {
  const int add = tile_sums[blockIdx.x];
  if (add == 0) return;
  const int64_t n = scan_count(n_max, n_dev, n_add);
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) out[base + k] += add;
}

// Single-pass exclusive scan with decoupled look-back (D. Merrill and M. Garland, "Single-pass
// parallel prefix scan with decoupled look-back", NVIDIA tech. report NVR-2016-002). Each block takes
// the next tile ticket, scans its tile, publishes the tile total, then adds the totals of the
// preceding tiles, walking back until a tile whose inclusive prefix is published, and publishes its
// own inclusive prefix. A block only waits on tiles whose tickets were taken before its own, by
// blocks already running, so the waits end; each is bounded all the same (kSpinMax polls), and a
// wait that gives up counts itself in *err (the run then reports a timeout).
// State word: epoch (30 bits) | flag (2 bits: 1 tile total, 2 inclusive prefix) | value (32 bits).
constexpr int kSpinMax = 1 << 22;   // polls of one wait in the chain (about a second at most)

__device__ __forceinline__ unsigned long long scan_word(unsigned epoch, unsigned flag, int v) {
  return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | (unsigned)v;
}

// What a scan does with each element's exclusive prefix besides storing it.
struct NoEpilogue {
  __device__ void element(int64_t, int, int) const {}
  __device__ void finish(int64_t, int) const {}
};

// Compaction tasks from the scan of per-module weights: task t starts at the first module whose
// prefix is >= t * chunk; an element k with prefix [excl, excl + v) starts the tasks whose t * chunk
// lies in (excl, excl + v] at module k + 1 (task 0 starts at module 0). finish() closes the last
// task at module n.
struct TaskEpilogue {
  int32_t* first;
  int chunk;
  __device__ void element(int64_t k, int excl, int v) const {
    for (int64_t t = (int64_t)excl / chunk + 1; t * chunk <= (int64_t)excl + v; ++t) first[t] = (int)(k + 1);
    if (k == 0) first[0] = 0;
  }
  __device__ void finish(int64_t n, int total) const { first[(total + chunk - 1) / chunk] = (int)n; }
};

template <class Epi>
__global__ void __launch_bounds__(kScanBlock) k_scan_1pass(const int32_t* in, int32_t* out, int64_t n_max,
                                                           const int32_t* n_dev, int n_add,
                                                           unsigned long long* state, int32_t* ticket,
                                                           const int32_t* run, int scan_idx, int32_t* err,
                                                           Epi epi, int spin_max) {
  __shared__ int s_tile, s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1);
  __syncthreads();
  const int tile = s_tile;
  const int64_t n = scan_count(n_max, n_dev, n_add);
  const int64_t last = (n + kTile - 1) / kTile - 1;
  if (tile > last) {
    if (n == 0 && tile == 0 && threadIdx.x == 0) out[0] = 0;
    return;
  }
  const int64_t base = (int64_t)tile * kTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int local = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    local += v[k];
  }
  int total;
  int pre = block_excl_scan(local, total);
  if (threadIdx.x == 0) {
    const unsigned epoch = ((unsigned)*run * kScanMax + (unsigned)scan_idx) & 0x3fffffffu;
    int excl = 0;
    if (tile == 0) {
      atomicExch(&state[0], scan_word(epoch, 2, total));
    } else {
      atomicExch(&state[tile], scan_word(epoch, 1, total));
      int p = tile - 1, spins = 0;
      while (p >= 0) {
        const unsigned long long sw = *reinterpret_cast<volatile unsigned long long*>(&state[p]);
        const unsigned flag = (unsigned)(sw >> 32) & 3u;
        if ((unsigned)(sw >> 34) != epoch || flag == 0) {
          if (++spins > spin_max) {
            atomicAdd(err, 1);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += (int)(unsigned)sw;
        if (flag == 2) break;
        --p;
      }
      atomicExch(&state[tile], scan_word(epoch, 2, excl + total));
    }
    s_excl = excl;
  }
  __syncthreads();
  pre += s_excl;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) {
      out[base + k] = pre;
      epi.element(base + k, pre, v[k]);
    }
    pre += v[k];
  }
  if (tile == last && threadIdx.x == 0) {
    out[n] = s_excl + total;
    epi.finish(n, s_excl + total);
  }
}

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + kTile - 1) / kTile + 1; }

void scan_exclusive_dev(const int32_t* in, int32_t* out, int64_t n, const int32_t* n_dev, int n_add, int32_t* tmp,
                        const Launch& L) {
  const int64_t tiles = (n + kTile - 1) / kTile;
  if (L.scan_state && *L.scan_idx < kScanMax) {
    const int idx = (*L.scan_idx)++;
    k_scan_1pass<<<(unsigned)std::max<int64_t>(tiles, 1), kScanBlock, 0, L.stream>>>(
        in, out, n, n_dev, n_add, L.scan_state, L.scan_ctr + idx, L.scan_run, idx, L.scan_err, NoEpilogue{},
        kSpinMax);
    LST_LAUNCH(L);
    return;
  }
  if (tiles == 0) {
    k_scan_sums<<<1, kScanBlock, 0, L.stream>>>(tmp, 0, out, 0, nullptr, 0);
    LST_LAUNCH(L);
    return;
  }
  k_scan_tiles<<<(unsigned)tiles, kScanBlock, 0, L.stream>>>(in, out, n, tmp, n_dev, n_add);
  k_scan_sums<<<1, kScanBlock, 0, L.stream>>>(tmp, tiles, out, n, n_dev, n_add);
  k_scan_add<<<(unsigned)tiles, kScanBlock, 0, L.stream>>>(out, n, tmp, n_dev, n_add);
  *L.launches += 3;
}

bool scan_tasks(int32_t* data, int64_t n, int32_t* first, int chunk, const Launch& L) {
  if (!L.scan_state || *L.scan_idx >= kScanMax) return false;
  const int64_t tiles = (n + kTile - 1) / kTile;
  const int idx = (*L.scan_idx)++;
  k_scan_1pass<<<(unsigned)std::max<int64_t>(tiles, 1), kScanBlock, 0, L.stream>>>(
      data, data, n, nullptr, 0, L.scan_state, L.scan_ctr + idx, L.scan_run, idx, L.scan_err,
      TaskEpilogue{first, chunk}, kSpinMax);
  LST_LAUNCH(L);
  return true;
}

int scan_wait_selftest(int device, int32_t* gave_up) {
  // three tiles of ones; the ticket counter starts at 1, so no block takes tile 0 and the block of
  // tile 1 waits for a state that is never published, until its bound (spin_max polls)
  constexpr int kTiles = 3;
  constexpr int64_t n = (int64_t)kTiles * kTile;
  if (cudaSetDevice(device) != cudaSuccess) return -1;
  int32_t *in = nullptr, *out = nullptr, *words = nullptr;
  unsigned long long* state = nullptr;
  int rc = -1;
  const int32_t init[3] = {1, 1, 0};   // ticket, run counter, gave-up count
  std::vector<int32_t> ones(n, 1);
  if (cudaMalloc(&in, n * sizeof(int32_t)) == cudaSuccess && cudaMalloc(&out, (n + 1) * sizeof(int32_t)) == cudaSuccess &&
      cudaMalloc(&words, 3 * sizeof(int32_t)) == cudaSuccess &&
      cudaMalloc(&state, kTiles * sizeof(unsigned long long)) == cudaSuccess &&
      cudaMemcpy(in, ones.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(words, init, sizeof(init), cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemset(state, 0, kTiles * sizeof(unsigned long long)) == cudaSuccess) {
    k_scan_1pass<<<kTiles - 1, kScanBlock>>>(in, out, n, nullptr, 0, state, words, words + 1, 0, words + 2,
                                             NoEpilogue{}, 2000);
    int32_t back[3] = {0, 0, 0};
    if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(back, words, sizeof(back), cudaMemcpyDeviceToHost) == cudaSuccess) {
      *gave_up = back[2];
      rc = 0;
    }
  }
  cudaFree(in);
  cudaFree(out);
  cudaFree(words);
  cudaFree(state);
  return rc;
}

void scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, const Launch& L) {
  scan_exclusive_dev(in, out, n, nullptr, 0, tmp, L);
}

}  // namespace lst
