// Hit binning for callers that cannot allocate device memory.
//
// lst_bin_hits() takes its scratch (per-sensor counters, a cursor array and the prefix-sum
// partials) from a context, and creating a context allocates. Some programs that embed this library
// cannot allow that: a trigger or online-reconstruction process that fixes its whole device memory
// budget when it starts and forbids later allocations, or a host framework that owns all device
// memory through its own allocator and does not let a plugin call cudaMalloc (which may also
// synchronize the device in the middle of its event loop). lst_bin_hits_noalloc() serves them: its
// scratch is one file-scope __device__ array of fixed size, which exists on every GPU that loads this
// library for as long as the process runs, so the call itself allocates nothing.
#include <string>

#include "lst_internal.h"

namespace lst {
namespace {

// Largest sensor count the static scratch supports (the toy tracker has 18,276 sensors).
constexpr int kNoAllocMaxSensors = 65536;
// counters [max] + cursors [max] + error word + prefix-sum partials
constexpr int kNoAllocWords = 2 * kNoAllocMaxSensors + 1 + 64;

static __device__ __align__(256) int32_t g_bin_scratch[kNoAllocWords];

// Host code cannot use g_bin_scratch's name as a device address: every call resolves it for the
// current device, with that device current. The lookup allocates nothing; it is not cached, because
// the address belongs to the device's context and changes when that context is destroyed and
// created again (cudaDeviceReset), and a cached address would then point at freed memory.
cudaError_t scratch_for_current_device(int32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<int32_t*>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace lst

extern "C" int lst_bin_hits_noalloc(const int32_t* d_sensor, int32_t n_hits, int32_t n_sensors, int32_t* d_order,
                                    int32_t* d_offsets, void* cuda_stream) {
  using namespace lst;
  if (n_hits < 0 || n_sensors <= 0 || (n_hits > 0 && (!d_sensor || !d_order)) || !d_offsets) {
    set_global_error("lst_bin_hits_noalloc: bad arguments");
    return LST_EINVAL;
  }
  if (n_sensors > kNoAllocMaxSensors) {
    set_global_error("lst_bin_hits_noalloc: more than 65536 sensors (the size of its static scratch)");
    return LST_EINVAL;
  }
  int32_t* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    set_global_error((std::string("lst_bin_hits_noalloc: scratch address: ") + cudaGetErrorString(e)).c_str());
    return LST_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int32_t* cnt = scratch;
  int32_t* cur = cnt + n_sensors;
  int32_t* err = cur + n_sensors;
  int32_t* tmp = err + 1;
  // the array keeps the previous call's contents: counters, cursors and the error word start at zero
  e = cudaMemsetAsync(cnt, 0, (2 * (size_t)n_sensors + 1) * sizeof(int32_t), st);
  if (e != cudaSuccess) {
    set_global_error((std::string("lst_bin_hits_noalloc: ") + cudaGetErrorString(e)).c_str());
    return LST_ECUDA;
  }
  long long launches = 0;
  Launch L;
  L.stream = st;
  L.launches = &launches;
  run_bin_raw(d_sensor, n_hits, n_sensors, d_order, d_offsets, cnt, cur, err, tmp, L);
  int32_t herr = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_global_error((std::string("lst_bin_hits_noalloc: ") + cudaGetErrorString(e)).c_str());
    return LST_ECUDA;
  }
  if (herr) {
    set_global_error("lst_bin_hits_noalloc: sensor id out of range");
    return LST_EINVAL;
  }
  return LST_OK;
}
