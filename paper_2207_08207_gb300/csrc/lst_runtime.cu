// Runtime of the LST library: contexts, resident geometry, arenas, the launch sequence of the chain,
// overflow retries, and the C ABI declared in include/lst.h.
//
// Memory. A context owns two device arenas, both allocated from a per-context CUDA memory pool that
// keeps freed blocks (the stream-ordered counterpart of the caching allocator of paper Sec. 4.2.1):
//  - the input arena: the batch's hits and seeds, event offsets and the per-module capacity
//    overrides that survive a retry;
//  - the work arena: every intermediate and output array, with all counters in one leading region
//    that a single memset clears before each run.
// Arenas grow (never shrink) when a batch needs more room; a run whose objects outgrow the current
// capacities is retried with larger ones.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lst_internal.h"

using namespace lst;

namespace {

__device__ __forceinline__ int find_seg_rt(const int32_t* off, int n, int i) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

struct EvPtr {
  const float *x, *y, *z;
  const int32_t* sensor;
  const lst_pls* pls;
};

// A device-readable address of host memory: any host address where the GPU reads pageable memory
// coherently (then no query is needed: pinned memory has the same address under unified
// addressing), else pinned (page-locked) memory through its mapped device pointer; nullptr when
// neither.
const void* device_view(const void* host, bool pageable_access) {
  if (!host) return nullptr;
  if (pageable_access) return host;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, host) == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer)
    return attr.devicePointer;
  cudaGetLastError();
  return nullptr;
}

// concatenate device-resident events into the input arena
__global__ void k_gather(const EvPtr* tab, Ws w, int H, int P) {
  const int64_t n = (int64_t)H + P;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < H) {
      const int i = (int)k;
      const int e = find_seg_rt(w.ev_hit_off, w.E, i);
      const int l = i - w.ev_hit_off[e];
      w.x[i] = tab[e].x[l];
      w.y[i] = tab[e].y[l];
      w.z[i] = tab[e].z[l];
      w.sensor[i] = tab[e].sensor[l];
    } else {
      const int p = (int)(k - H);
      const int e = find_seg_rt(w.ev_pls_off, w.E, p);
      w.pls[p] = tab[e].pls[p - w.ev_pls_off[e]];
    }
  }
}

// the per-event summary
__global__ void k_ev_stat(Ws w, int n_mods) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w.E; e += gridDim.x * blockDim.x) {
    int* st = w.ev_stat + e * kEvWords;
    const int a = e * n_mods, b = (e + 1) * n_mods;
    const int p0 = w.ev_pls_off[e], p1 = w.ev_pls_off[e + 1];
    st[0] = w.md_off[b] - w.md_off[a];
    st[1] = w.ls_off[b] - w.ls_off[a];
    st[2] = w.t3_off[b] - w.t3_off[a];
    st[3] = w.t5_off[b] - w.t5_off[a];
    st[4] = w.pt3_off[p1] - w.pt3_off[p0];
    st[5] = w.pt5_off[p1] - w.pt5_off[p0];
    const int ntc = w.tc_cnt[e];
    st[6] = ntc;
    // st[7..10] (per-type counts) come from the assembly
    st[11] = w.md_off[a];
    st[12] = w.ls_off[a];
    st[13] = w.t3_off[a];
    st[14] = w.t5_off[a];
    st[15] = w.pt3_off[p0];
    st[16] = w.pt5_off[p0];
    st[17] = w.tcd_off[e];
  }
}

__global__ void k_raise(const int32_t* cnt, int32_t* ovr, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    ovr[i] = max(ovr[i], cnt[i]);
}

// ---------------------------------------------------------------------------------------------
// arena planning
// ---------------------------------------------------------------------------------------------
struct Planner {
  struct Item { void** ptr; size_t bytes; };
  std::vector<Item> items;
  size_t total = 0;
  template <class T>
  void add(T*& p, int64_t n) {
    items.push_back({reinterpret_cast<void**>(&p), (size_t)std::max<int64_t>(n, 1) * sizeof(T)});
  }
  size_t layout() {
    total = 0;
    for (auto& it : items) total += (it.bytes + 255) & ~size_t(255);
    return total;
  }
  void assign(void* base) {
    size_t off = 0;
    for (auto& it : items) {
      *it.ptr = static_cast<char*>(base) + off;
      off += (it.bytes + 255) & ~size_t(255);
    }
  }
};

}  // namespace

// ---------------------------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------------------------
struct lst_ctx {
  int device = 0;
  lst_config cfg{};
  Consts consts{};
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  // geometry
  Geo geo{};
  void* geo_mem = nullptr;
  bool geo_loaded = false;
  int32_t max_degree = 0;
  // arenas
  Ws ws{};
  Caps caps{};          // current work-arena capacities
  Caps in_caps{};       // current input-arena capacities
  void* in_mem = nullptr;
  size_t in_bytes = 0;
  void* work_mem = nullptr;
  size_t work_bytes = 0;
  void* zero_begin = nullptr;
  size_t zero_bytes = 0;
  // host staging
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  int32_t* h_status = nullptr;   // pinned: [ST_N_WORDS + E * kEvWords]
  // capacity multipliers per stage (MD, LS, T3, T5), raised after a stage overflowed so that later
  // batches of the same context rarely need a retry; copied to the device before each run
  float stage_scale[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  size_t h_status_words = 0;
  EvPtr* d_tab = nullptr;
  int tab_cap = 0;
  int32_t* bin_mem = nullptr;   // scratch of lst_bin_hits
  size_t bin_words = 0;
  // last run
  int32_t E = 0, H = 0, P = 0;
  std::vector<int32_t> ev_hits, ev_pls;
  std::vector<lst_counts> counts;
  std::vector<lst_event_out> outs;
  lst_event_out* user_out = nullptr;
  bool pending = false;
  int retries = 0;
  int first_ovf[LST_N_STAGES] = {};
  // instrumentation
  long long launches = 0;
  int n_sm = 152;
  int ls_bps = 0;
  int t3_bps = 0, t5_bps = 0;   // resident blocks per SM of the T3 / T5 candidate kernels
  int pt3_bps = 0, pt5_bps = 0; // and of the pT3 / pT5 pre-filters
  bool pageable_access = false;   // the GPU reads pageable host memory coherently (e.g. NVLink-C2C)
  // CUDA graph of the whole chain for the current arenas (shape-independent within capacities)
  cudaGraphExec_t graph_exec = nullptr;
  long long graph_nodes = 0;
  uint64_t arena_gen = 1, graph_gen = 0;
  bool graph_timing = false;
  bool timing = false;
  cudaEvent_t ev_stage[10] = {};
  cudaEvent_t ev_kern[2 * K_N_TIMED] = {};
  float kern_ms[K_N_TIMED] = {};
  float stage_ms[LST_N_STAGES + 1] = {};
  cudaEvent_t ev_done = nullptr;
  std::string err;
};

static std::string g_create_error;

void lst::set_global_error(const char* msg) { g_create_error = msg; }

namespace {

int fail(lst_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, LST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

Consts make_consts(const lst_config& c) {
  Consts k{};
  Cst<double>& d = k.d;
  d.k = c.k; d.pt_thr = c.pt_thr; d.sin_max = c.sin_max; d.z_lum = c.z_lum; d.d0_max = c.d0_max;
  d.n_sigma = c.n_sigma; d.sigma_rphi = c.sigma_rphi; d.sigma_z = c.sigma_z; d.sigma_r = c.sigma_r;
  d.k2p = (double)c.k / 2.0 / (double)c.pt_thr;
  d.two_rthr = 2.0 * (double)c.pt_thr / (double)c.k;
  d.tol_rphi = (double)c.n_sigma * std::sqrt(2.0) * (double)c.sigma_rphi;
  d.tol_z = (double)c.n_sigma * std::sqrt(2.0) * (double)c.sigma_z;
  d.tol_r = (double)c.n_sigma * std::sqrt(2.0) * (double)c.sigma_r;
  d.chi2_t3 = c.chi2_t3; d.chi2_t5_c = c.chi2_t5_c; d.chi2_t5_rz = c.chi2_t5_rz;
  d.chi2_pt3_xy = c.chi2_pt3_xy; d.chi2_pt3_rz = c.chi2_pt3_rz;
  d.chi2_pt5_xy = c.chi2_pt5_xy; d.chi2_pt5_rz = c.chi2_pt5_rz;
  d.f_t3 = c.f_t3; d.d0_t3 = c.d0_t3; d.c_rel = c.c_rel; d.c_abs = c.c_abs; d.dr_min = c.dr_min;
  d.pt_cap = c.pt_cap; d.pls_dir_err = c.pls_dir_err; d.pls_pt_err = c.pls_pt_err;
  d.sigma_floor = c.sigma_floor; d.t5_overlap_hits = c.t5_overlap_hits;
  Cst<float>& f = k.f;
  f.k = (float)d.k; f.pt_thr = (float)d.pt_thr; f.sin_max = (float)d.sin_max; f.z_lum = (float)d.z_lum;
  f.d0_max = (float)d.d0_max; f.n_sigma = (float)d.n_sigma; f.sigma_rphi = (float)d.sigma_rphi;
  f.sigma_z = (float)d.sigma_z; f.sigma_r = (float)d.sigma_r; f.k2p = (float)d.k2p;
  f.two_rthr = (float)d.two_rthr; f.tol_rphi = (float)d.tol_rphi; f.tol_z = (float)d.tol_z;
  f.tol_r = (float)d.tol_r; f.chi2_t3 = (float)d.chi2_t3; f.chi2_t5_c = (float)d.chi2_t5_c;
  f.chi2_t5_rz = (float)d.chi2_t5_rz; f.chi2_pt3_xy = (float)d.chi2_pt3_xy;
  f.chi2_pt3_rz = (float)d.chi2_pt3_rz; f.chi2_pt5_xy = (float)d.chi2_pt5_xy;
  f.chi2_pt5_rz = (float)d.chi2_pt5_rz; f.f_t3 = (float)d.f_t3; f.d0_t3 = (float)d.d0_t3;
  f.c_rel = (float)d.c_rel; f.c_abs = (float)d.c_abs; f.dr_min = (float)d.dr_min;
  f.pt_cap = (float)d.pt_cap; f.pls_dir_err = (float)d.pls_dir_err; f.pls_pt_err = (float)d.pls_pt_err;
  f.sigma_floor = (float)d.sigma_floor; f.t5_overlap_hits = d.t5_overlap_hits;
  Cst<ff>& x = k.x;
  x.k = ff(d.k); x.pt_thr = ff(d.pt_thr); x.sin_max = ff(d.sin_max); x.z_lum = ff(d.z_lum);
  x.d0_max = ff(d.d0_max); x.n_sigma = ff(d.n_sigma); x.sigma_rphi = ff(d.sigma_rphi);
  x.sigma_z = ff(d.sigma_z); x.sigma_r = ff(d.sigma_r); x.k2p = ff(d.k2p); x.two_rthr = ff(d.two_rthr);
  x.tol_rphi = ff(d.tol_rphi); x.tol_z = ff(d.tol_z); x.tol_r = ff(d.tol_r); x.chi2_t3 = ff(d.chi2_t3);
  x.chi2_t5_c = ff(d.chi2_t5_c); x.chi2_t5_rz = ff(d.chi2_t5_rz); x.chi2_pt3_xy = ff(d.chi2_pt3_xy);
  x.chi2_pt3_rz = ff(d.chi2_pt3_rz); x.chi2_pt5_xy = ff(d.chi2_pt5_xy); x.chi2_pt5_rz = ff(d.chi2_pt5_rz);
  x.f_t3 = ff(d.f_t3); x.d0_t3 = ff(d.d0_t3); x.c_rel = ff(d.c_rel); x.c_abs = ff(d.c_abs);
  x.dr_min = ff(d.dr_min); x.pt_cap = ff(d.pt_cap); x.pls_dir_err = ff(d.pls_dir_err);
  x.pls_pt_err = ff(d.pls_pt_err); x.sigma_floor = ff(d.sigma_floor); x.t5_overlap_hits = d.t5_overlap_hits;
  return k;
}

Launch make_launch(lst_ctx* ctx) {
  Launch L;
  L.stream = ctx->stream;
  L.block_ls = ctx->cfg.block_ls;
  L.warps_px = ctx->cfg.warps_px;
  L.persistent = ctx->cfg.persistent == 2 ? 2 : (ctx->cfg.persistent != 0 ? 1 : 0);
  L.launches = &ctx->launches;
  L.n_sm = ctx->n_sm;
  L.ls_blocks_per_sm = ctx->ls_bps;
  L.t3_blocks_per_sm = ctx->t3_bps;
  L.t5_blocks_per_sm = ctx->t5_bps;
  L.pt3_blocks_per_sm = ctx->pt3_bps;
  L.pt5_blocks_per_sm = ctx->pt5_bps;
  L.kev = ctx->timing ? ctx->ev_kern : nullptr;
  return L;
}

// default object capacities for a batch with H hits and P seeds (generous; a run that needs more
// grows them and is retried)
Caps default_caps(int64_t E, int64_t H, int64_t P, int64_t n_mods) {
  Caps c;
  c.E = E; c.H = H; c.P = P; c.n_mods = n_mods;
  c.md_slots = 4 * H + 4096;
  c.ls_slots = 40 * H + 16384;
  c.t3_slots = 16 * H + 8192;
  c.t5_slots = 2 * H + 4096;
  c.md_dense = H + 4096;
  c.ls_dense = 6 * H + 16384;
  c.t3_dense = 2 * H + 8192;
  c.t5_dense = H / 2 + 4096;
  c.p3_slots = H + 4096;
  c.p5_slots = H / 2 + 4096;
  c.q_md = H / 8 + 4096;
  c.q_ls = H + 8192;
  c.q_t3 = 2 * H + 8192;
  c.q_t5 = H + 8192;
  c.q_p3 = H + 8192;
  c.q_p5 = H / 2 + 8192;
  return c;
}

int plan_input(lst_ctx* ctx, int64_t E, int64_t H, int64_t P) {
  if (ctx->in_mem && E <= ctx->in_caps.E && H <= ctx->in_caps.H && P <= ctx->in_caps.P) return LST_OK;
  Caps c;
  c.E = std::max<int64_t>(E, ctx->in_caps.E);
  c.H = std::max<int64_t>(H + H / 4, ctx->in_caps.H);
  c.P = std::max<int64_t>(P + P / 4, ctx->in_caps.P);
  const int64_t V = c.E * ctx->geo.n_mods;
  Planner pl;
  Ws& w = ctx->ws;
  pl.add(w.x, c.H); pl.add(w.y, c.H); pl.add(w.z, c.H); pl.add(w.sensor, c.H);
  pl.add(w.pls, c.P);
  pl.add(w.ev_hit_off, 2 * (c.E + 1));   // hit offsets, then seed offsets
  pl.add(w.md_ovr, V); pl.add(w.ls_ovr, V); pl.add(w.t3_ovr, V); pl.add(w.t5_ovr, V);
  float* stage_scale = nullptr;
  pl.add(stage_scale, 4);
  const size_t bytes = pl.layout();
  if (ctx->in_mem) CK(cudaFreeAsync(ctx->in_mem, ctx->stream));
  ctx->in_mem = nullptr;
  CK(cudaMallocFromPoolAsync(&ctx->in_mem, bytes, ctx->pool, ctx->stream));
  pl.assign(ctx->in_mem);
  w.ev_pls_off = w.ev_hit_off + (c.E + 1);
  w.stage_scale = stage_scale;
  ctx->in_bytes = bytes;
  ctx->in_caps = c;
  ctx->arena_gen++;
  // overrides start at zero
  CK(cudaMemsetAsync(w.md_ovr, 0, V * sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(w.ls_ovr, 0, V * sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(w.t3_ovr, 0, V * sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(w.t5_ovr, 0, V * sizeof(int32_t), ctx->stream));
  return LST_OK;
}

// Lay out the work arena for capacities c (addresses assigned to ws when base is not null).
// Returns its bytes (zeroed region first, size in *zero_bytes).
size_t layout_work(Ws& w, const Caps& c, int n_mods, void* base, size_t* zero_bytes);

int plan_work(lst_ctx* ctx, const Caps& want) {
  Caps c = want;
  c.E = ctx->in_caps.E;   // event offsets (padded to E) live in the input arena
  c.half = ctx->cfg.half_floats != 0;
  size_t zb = 0;
  const size_t total = layout_work(ctx->ws, c, ctx->geo.n_mods, nullptr, &zb);
  if (ctx->work_mem) CK(cudaFreeAsync(ctx->work_mem, ctx->stream));
  ctx->work_mem = nullptr;
  CK(cudaMallocFromPoolAsync(&ctx->work_mem, total, ctx->pool, ctx->stream));
  layout_work(ctx->ws, c, ctx->geo.n_mods, ctx->work_mem, &zb);
  Ws& w = ctx->ws;
  // single-pass scan states start empty (epoch 0 never matches a run's epochs)
  CK(cudaMemsetAsync(w.scan_state, 0, w.scan_state_n * sizeof(unsigned long long), ctx->stream));
  CK(cudaMemsetAsync(w.scan_run, 0, sizeof(int32_t), ctx->stream));
  ctx->zero_begin = ctx->work_mem;
  ctx->zero_bytes = zb;
  ctx->work_bytes = total;
  ctx->caps = c;
  ctx->arena_gen++;
  w.cap = c;
  w.n_cells = tc_cells_per_event();
  w.tc_capacity = c.P + c.t5_dense;
  // pinned status words
  const size_t words = ST_N_WORDS + (size_t)c.E * kEvWords;
  if (words > ctx->h_status_words) {
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    ctx->h_status = nullptr;
    CK(cudaMallocHost(&ctx->h_status, words * sizeof(int32_t)));
    ctx->h_status_words = words;
  }
  return LST_OK;
}

size_t layout_work(Ws& w, const Caps& c, int n_mods, void* base, size_t* zero_bytes) {
  const int64_t V = c.E * n_mods;
  const int64_t S = 2 * V;
  const int64_t NC = (int64_t)c.E * tc_cells_per_event();
  const int64_t tc_cap = c.P + c.t5_dense;
  Planner z, pl;   // z: cleared before every run
  z.add(w.status, ST_N_WORDS + c.E * kEvWords);   // status words, then the per-event words
  z.add(w.tc_cnt, c.E);
  z.add(w.sens_cnt, S); z.add(w.sens_cur, S);
  z.add(w.md_cnt, V); z.add(w.ls_cnt, V); z.add(w.t3_cnt, V); z.add(w.t5_cnt, V);
  z.add(w.t3_bound, V); z.add(w.t5_bound, V);
  z.add(w.p3_cnt, c.P); z.add(w.p3_cur, c.P); z.add(w.p5_cnt, c.P); z.add(w.p5_cur, c.P);
  z.add(w.h5_cnt, c.H + 1); z.add(w.h5_cur, c.H + 1);
  z.add(w.cell_cnt, NC); z.add(w.cell_cur, NC);
  z.add(w.work_cnt, 32); z.add(w.work_cur, 32);
  z.add(w.scan_ctr, kScanMax);
  z.add(w.ext_qn, 5);
  z.add(w.ls_head, 1);
  // binning
  pl.add(w.hit_vs, c.H); pl.add(w.sens_off, S + 1); pl.add(w.bidx, c.H);
  pl.add(w.bx, c.H); pl.add(w.by, c.H); pl.add(w.bz, c.H); pl.add(w.borig, c.H);
  // compaction scratch, LS work list
  pl.add(w.eff, V + 1);
  pl.add(w.grp_key, std::max(c.H, c.t3_dense) + 2);
  pl.add(w.grp_pos, std::max({c.md_dense, c.ls_dense, c.t3_dense, c.t5_dense}));
  pl.add(w.grp_key12, std::max({c.md_dense, c.ls_dense, c.t3_dense, c.t5_dense}));
  pl.add(w.grp_task, (std::max({c.md_slots, c.ls_slots, c.t3_slots, c.t5_slots}) + V) / 64 + 2);
  pl.add(w.work, kLsMaxChunks * V); pl.add(w.work_c, kLsMaxChunks * V); pl.add(w.work_bucket, V);
  pl.add(w.work_nch, V); pl.add(w.work_off, 33);
  pl.add(w.perm, std::max({c.md_dense, c.ls_dense, c.t3_dense, c.t5_dense}));
  // MD
  pl.add(w.md_cap, V); pl.add(w.md_base, V + 1); pl.add(w.md_off, V + 1);
  pl.add(w.ms_lo, c.md_slots); pl.add(w.ms_up, c.md_slots); pl.add(w.ms_dpc, c.md_slots); pl.add(w.ms_pte, c.md_slots);
  pl.add(w.md_lo, c.md_dense); pl.add(w.md_up, c.md_dense); pl.add(w.md_vm, c.md_dense);
  pl.add(w.md_rlo, c.md_dense);
  // output-only floats: float32 arrays, or binary16 ones when c.half (the others stay nullptr)
  auto out_f = [&](float*& f32, uint16_t*& f16, int64_t n) {
    f32 = nullptr;
    f16 = nullptr;
    if (c.half) pl.add(f16, n);
    else pl.add(f32, n);
  };
  out_f(w.md_dpc, w.md_dpc_h, c.md_dense); out_f(w.md_pte, w.md_pte_h, c.md_dense);
  pl.add(w.md_ec, c.md_dense);
  pl.add(w.md_xyzr, c.md_dense); pl.add(w.md_sa, c.md_dense); pl.add(w.md_rphi, c.md_dense);
  pl.add(w.md_rmin, V); pl.add(w.md_rmax, V); pl.add(w.md_win, V);
  // LS
  pl.add(w.ls_cap, V); pl.add(w.ls_base, V + 1); pl.add(w.ls_off, V + 1); pl.add(w.lsin_off, c.md_dense + 2);
  pl.add(w.lss_in, c.ls_slots); pl.add(w.lss_out, c.ls_slots); pl.add(w.lss_dphi, c.ls_slots);
  pl.add(w.ls_in, c.ls_dense); pl.add(w.ls_out, c.ls_dense);
  out_f(w.ls_z0, w.ls_z0_h, c.ls_dense); out_f(w.ls_dphi, w.ls_dphi_h, c.ls_dense);
  pl.add(w.ls_xy_out, c.ls_dense);
  // T3
  pl.add(w.t3_cap, V); pl.add(w.t3_base, V + 1); pl.add(w.t3_off, V + 1);
  pl.add(w.t3s_a, c.t3_slots); pl.add(w.t3s_b, c.t3_slots); pl.add(w.t3s_R, c.t3_slots); pl.add(w.t3s_xc, c.t3_slots);
  pl.add(w.t3s_yc, c.t3_slots); pl.add(w.t3s_chi2, c.t3_slots); pl.add(w.t3s_pte, c.t3_slots);
  pl.add(w.t3_a, c.t3_dense); pl.add(w.t3_b, c.t3_dense); pl.add(w.t3_md0, c.t3_dense); pl.add(w.t3_md1, c.t3_dense);
  pl.add(w.t3_md2, c.t3_dense); pl.add(w.t3_R, c.t3_dense);
  out_f(w.t3_xc, w.t3_xc_h, c.t3_dense); out_f(w.t3_yc, w.t3_yc_h, c.t3_dense);
  out_f(w.t3_chi2, w.t3_chi2_h, c.t3_dense); out_f(w.t3_pte, w.t3_pte_h, c.t3_dense);
  pl.add(w.t3_anc, 3 * c.t3_dense); pl.add(w.t3_anc_rlo, 3 * c.t3_dense); pl.add(w.t3_ecm, c.t3_dense);
  pl.add(w.t3md_off, c.md_dense + 2);
  // T5
  pl.add(w.t5_cap, V); pl.add(w.t5_base, V + 1); pl.add(w.t5_off, V + 1);
  pl.add(w.t5s_a, c.t5_slots); pl.add(w.t5s_b, c.t5_slots); pl.add(w.t5s_f, 8 * c.t5_slots);
  pl.add(w.t5_a, c.t5_dense); pl.add(w.t5_b, c.t5_dense); pl.add(w.t5_md, 5 * c.t5_dense); pl.add(w.t5_f, 8 * c.t5_dense);
  w.t5_h = nullptr;
  if (c.half) pl.add(w.t5_h, 3 * c.t5_dense);
  pl.add(w.t5_anc, 5 * c.t5_dense); pl.add(w.t5_anc_rlo, 5 * c.t5_dense); pl.add(w.t5_ecm, c.t5_dense);
  pl.add(w.t5_kept, c.t5_dense); pl.add(w.acc5t, c.t5_dense);
  pl.add(w.box3, 2 * V); pl.add(w.box5, 2 * V);
  // pixel
  pl.add(w.pls_bin, c.P); pl.add(w.pls_ev, c.P); pl.add(w.pls_seed, 2 * c.P); pl.add(w.pls_seed_ff, 9 * c.P);
  pl.add(w.p3a_pls, c.p3_slots); pl.add(w.p3a_obj, c.p3_slots); pl.add(w.p3a_xy, c.p3_slots);
  pl.add(w.p3a_rz, c.p3_slots); pl.add(w.p3a_sc, c.p3_slots); pl.add(w.pt3_off, c.P + 1);
  pl.add(w.pt3_pls, c.p3_slots); pl.add(w.pt3_obj, c.p3_slots);
  out_f(w.pt3_xy, w.pt3_xy_h, c.p3_slots); out_f(w.pt3_rz, w.pt3_rz_h, c.p3_slots); pl.add(w.pt3_sc, c.p3_slots);
  pl.add(w.p5a_pls, c.p5_slots); pl.add(w.p5a_obj, c.p5_slots); pl.add(w.p5a_xy, c.p5_slots);
  pl.add(w.p5a_rz, c.p5_slots); pl.add(w.p5a_sc, c.p5_slots); pl.add(w.pt5_off, c.P + 1);
  pl.add(w.pt5_pls, c.p5_slots); pl.add(w.pt5_obj, c.p5_slots);
  out_f(w.pt5_xy, w.pt5_xy_h, c.p5_slots); out_f(w.pt5_rz, w.pt5_rz_h, c.p5_slots); pl.add(w.pt5_sc, c.p5_slots);
  pl.add(w.grp_tmp, std::max(c.p3_slots, c.p5_slots));
  // track candidates
  pl.add(w.best5, c.P); pl.add(w.best3, c.P); pl.add(w.pls_member, c.P); pl.add(w.acc3, c.P); pl.add(w.accl, c.P);
  pl.add(w.h5_off, c.H + 2); pl.add(w.h5_idx, 10 * c.t5_dense);
  pl.add(w.t5_hit, 10 * c.t5_dense);
  pl.add(w.cell_off, NC + 1); pl.add(w.cell_item, c.P + c.t5_dense);
  pl.add(w.tc_code, tc_cap); pl.add(w.tc_perm, tc_cap); pl.add(w.tc_n, 4 * c.E); pl.add(w.tc_key, tc_cap); pl.add(w.tc_hit_key, 14 * tc_cap);
  pl.add(w.tc_type, tc_cap); pl.add(w.tc_obj, tc_cap); pl.add(w.tc_hits, 14 * tc_cap);
  pl.add(w.tc_pt, tc_cap); pl.add(w.tc_eta, tc_cap); pl.add(w.tc_phi, tc_cap);
  pl.add(w.tcd_off, c.E + 1);
  pl.add(w.tcd_type, tc_cap); pl.add(w.tcd_obj, tc_cap); pl.add(w.tcd_hits, 14 * tc_cap);
  pl.add(w.tcd_pt, tc_cap); pl.add(w.tcd_eta, tc_cap); pl.add(w.tcd_phi, tc_cap);
  pl.add(w.tcd_ext_t3, tc_cap); pl.add(w.tcd_ext_n, tc_cap); pl.add(w.tcd_ext_hits, 4 * tc_cap);
  pl.add(w.tcd_ext_c, tc_cap); pl.add(w.tcd_ext_rz, tc_cap);
  w.ext_qcap = tc_cap / 2 + 1024;   // candidates per anchor count (about one per candidate row in all)
  pl.add(w.ext_cnt, tc_cap); pl.add(w.ext_ref, kExtRefs * tc_cap); pl.add(w.ext_slow, tc_cap);
  pl.add(w.ext_q, 4 * w.ext_qcap); pl.add(w.ext_res, 4 * w.ext_qcap);
  // event-local outputs
  pl.add(w.o_md_lo, c.md_dense); pl.add(w.o_md_up, c.md_dense); pl.add(w.o_md_mod, c.md_dense);
  pl.add(w.o_ls_in, c.ls_dense); pl.add(w.o_ls_out, c.ls_dense);
  pl.add(w.o_t3_a, c.t3_dense); pl.add(w.o_t3_b, c.t3_dense);
  pl.add(w.o_t5_a, c.t5_dense); pl.add(w.o_t5_b, c.t5_dense);
  pl.add(w.o_pt3_pls, c.p3_slots); pl.add(w.o_pt3_obj, c.p3_slots);
  pl.add(w.o_pt5_pls, c.p5_slots); pl.add(w.o_pt5_obj, c.p5_slots);
  // queues
  pl.add(w.q_md, c.q_md); pl.add(w.q_ls, c.q_ls); pl.add(w.q_t3, c.q_t3); pl.add(w.q_t5, c.q_t5);
  pl.add(w.q_p3, c.q_p3); pl.add(w.q_p5, c.q_p5);
  const int64_t scan_n = std::max({S + 1, V + 1, c.H + 2, c.md_dense + 2, c.ls_dense + 2, c.t3_dense + 2, NC + 1, c.P + 1});
  pl.add(w.scan_tmp, scan_tmp_elems(scan_n) + 8);
  w.scan_state_n = scan_tmp_elems(scan_n) + 8;
  pl.add(w.scan_state, w.scan_state_n);
  pl.add(w.scan_run, 1);
  const size_t zb = z.layout();
  const size_t pb = pl.layout();
  if (base) {
    z.assign(base);
    pl.assign(static_cast<char*>(base) + zb);
    w.ev_stat = w.status + ST_N_WORDS;
  }
  *zero_bytes = zb;
  return zb + pb;
}

int ensure_pinned(lst_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->pinned_bytes) return LST_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  CK(cudaMallocHost(&ctx->pinned, bytes));
  ctx->pinned_bytes = bytes;
  return LST_OK;
}

// Enqueue the whole chain on ctx->stream. Every launch is shaped by the arena capacities, never by
// the batch (kernels read the actual hit / seed counts from the padded event offsets), so the same
// sequence serves every batch that fits and can be captured once as a CUDA graph.
int enqueue_chain(lst_ctx* ctx, bool capturing) {
  Ws& w = ctx->ws;
  w.E = (int32_t)ctx->caps.E;
  w.H = (int32_t)ctx->caps.H;
  w.P = (int32_t)ctx->caps.P;
  w.V = w.E * ctx->geo.n_mods;
  w.S = 2 * w.V;
  w.cap_scale = ctx->cfg.cap_scale;
  // a small batch has too few modules to balance the LS kernel's warps: its heavy modules are split
  // into chunks of outer MDs (for 64 events the whole-module items already balance)
  w.ls_chunk = w.E < 8 ? 64 : (1 << 30);
  w.cycle_budget = ctx->cfg.cycle_budget;
  Launch L = make_launch(ctx);
  int scan_idx = 0;
  L.scan_state = w.scan_state;
  L.scan_ctr = w.scan_ctr;
  L.scan_run = w.scan_run;
  L.scan_err = &w.status[ST_TIMEOUT];
  L.scan_idx = &scan_idx;
  const Geo& g = ctx->geo;
  const Consts& c = ctx->consts;
  L.capturing = capturing;
  CK(cudaMemsetAsync(ctx->zero_begin, 0, ctx->zero_bytes, ctx->stream));
  int ei = 0;
  // the first stage after which an error is pending (named in the error message)
  const char* failed_at = nullptr;
  auto mark = [&](const char* stage) {
    if (ctx->timing) KT_REC(L, ctx->ev_stage[ei++]);
    if (!failed_at && cudaPeekAtLastError() != cudaSuccess) failed_at = stage;
  };
  mark("start");
  run_binning(w, g, L);
  run_md(w, g, c, L);
  mark("hit binning and MD");
  run_ls(w, g, c, L);
  mark("LS");
  run_t3(w, g, c, L);
  mark("T3");
  run_t5(w, g, c, L);
  mark("T5");
  run_pixel(w, g, c, L);
  mark("pT3 / pT5");
  run_tc(w, g, c, L);
  mark("TC");
  // (the event-local copies of member indices are written with the dense objects)
  k_ev_stat<<<grid_for(w.E, 64), 64, 0, ctx->stream>>>(w, g.n_mods);
  ctx->launches += 1;
  mark("summary");
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess)
    return fail(ctx, LST_ECUDA, std::string("chain launch (first error after: ") + (failed_at ? failed_at : "?") +
                                    "): " + cudaGetErrorString(le));
  CK(cudaMemcpyAsync(ctx->h_status, w.status, (ST_N_WORDS + (size_t)w.E * kEvWords) * sizeof(int32_t),
                     cudaMemcpyDeviceToHost, ctx->stream));
  return LST_OK;
}

int launch_chain(lst_ctx* ctx) {
  const bool graph = ctx->cfg.use_graph != 0;
  if (!graph) {
    int rc = enqueue_chain(ctx, false);
    if (rc) return rc;
  } else {
    // the timing events, when enabled, are captured as event-record nodes of the graph
    if (!ctx->graph_exec || ctx->graph_gen != ctx->arena_gen || ctx->graph_timing != ctx->timing) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      const long long before = ctx->launches;
      const int rc = enqueue_chain(ctx, true);
      cudaGraph_t gr = nullptr;
      const cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
      if (rc) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return fail(ctx, LST_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      const cudaError_t ei = cudaGraphInstantiate(&ctx->graph_exec, gr, 0);
      cudaGraphDestroy(gr);
      if (ei != cudaSuccess) {
        ctx->graph_exec = nullptr;
        return fail(ctx, LST_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
      }
      ctx->graph_nodes = ctx->launches - before;
      ctx->launches = before;
      ctx->graph_gen = ctx->arena_gen;
      ctx->graph_timing = ctx->timing;
    }
    CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->launches += ctx->graph_nodes;
  }
  CK(cudaEventRecord(ctx->ev_done, ctx->stream));
  return LST_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

void lst_config_default(lst_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->k = 0.0114f;
  c->pt_thr = 0.8f;
  c->sin_max = 0.95f;
  c->z_lum = 15.0f;
  c->d0_max = 0.1f;
  c->n_sigma = 3.0f;
  c->sigma_rphi = 0.003f;
  c->sigma_z = 0.1f;
  c->sigma_r = 0.1f;
  c->chi2_t3 = 9.0f;
  c->chi2_t5_c = 20.0f;
  c->chi2_t5_rz = 16.0f;
  c->chi2_pt3_xy = 16.0f;
  c->chi2_pt3_rz = 16.0f;
  c->chi2_pt5_xy = 25.0f;
  c->chi2_pt5_rz = 25.0f;
  c->f_t3 = 0.8f;
  c->d0_t3 = 2.0f;
  c->c_rel = 0.2f;
  c->c_abs = 1.5e-4f;
  c->dr_min = 0.01f;
  c->pt_cap = 1.0e4f;
  c->pls_dir_err = 1.0e-3f;
  c->pls_pt_err = 0.01f;
  c->sigma_floor = 1.0e-4f;
  c->t5_overlap_hits = 7;
  c->persistent = 2;
  c->use_graph = 0;
  c->block_ls = 128;
  c->warps_px = 4;
  c->cap_scale = 1.0f;
  c->max_retries = 4;
  c->cycle_budget = 0;
  c->half_floats = 0;
}

int lst_create(lst_ctx** out, const lst_config* cfg, int device) {
  lst_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, LST_EINVAL, "lst_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail(nullptr, LST_ECUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
  if (device < 0 || device >= ndev) return fail(nullptr, LST_EINVAL, "lst_create: no such device");
  ctx = new lst_ctx();
  ctx->device = device;
  if (cfg) ctx->cfg = *cfg;
  else lst_config_default(&ctx->cfg);
  if (ctx->cfg.block_ls != 64 && ctx->cfg.block_ls != 128 && ctx->cfg.block_ls != 256) ctx->cfg.block_ls = 128;
  if (ctx->cfg.warps_px < 1 || ctx->cfg.warps_px > 8) ctx->cfg.warps_px = 4;
  if (!(ctx->cfg.cap_scale >= 0.25f)) ctx->cfg.cap_scale = 1.0f;
  if (ctx->cfg.max_retries < 0) ctx->cfg.max_retries = 0;
  if (!(ctx->cfg.pt_thr > 0.f) || !(ctx->cfg.k > 0.f)) {
    delete ctx;
    return fail(nullptr, LST_EINVAL, "lst_create: pt_thr and k must be positive");
  }
  ctx->consts = make_consts(ctx->cfg);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return fail(nullptr, LST_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if ((e = cudaMemPoolCreate(&ctx->pool, &props)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming)) != cudaSuccess) {
    lst_destroy(ctx);
    return fail(nullptr, LST_ECUDA, std::string("lst_create: ") + cudaGetErrorString(e));
  }
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  for (auto& ev : ctx->ev_stage) cudaEventCreate(&ev);
  for (auto& ev : ctx->ev_kern) cudaEventCreate(&ev);
  ctx->stream = ctx->own_stream;
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (ctx->n_sm <= 0) ctx->n_sm = 152;
  int pageable = 0;
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
  ctx->pageable_access = pageable != 0;
  tc_configure();
  *out = ctx;
  return LST_OK;
}

void lst_destroy(lst_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
  if (ctx->in_mem) cudaFreeAsync(ctx->in_mem, ctx->own_stream);
  if (ctx->work_mem) cudaFreeAsync(ctx->work_mem, ctx->own_stream);
  if (ctx->d_tab) cudaFreeAsync(ctx->d_tab, ctx->own_stream);
  if (ctx->bin_mem) cudaFreeAsync(ctx->bin_mem, ctx->own_stream);
  if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->geo_mem) cudaFree(ctx->geo_mem);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  for (auto& ev : ctx->ev_stage)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : ctx->ev_kern)
    if (ev) cudaEventDestroy(ev);
  if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
}

int lst_check_geometry(const lst_module* mods, int32_t n_mods, const int32_t* conn_off, const int32_t* conn_tgt,
                       const int32_t* pix_off, const int32_t* pix_tgt, int32_t n_pix_bins, int32_t* max_degree) {
  lst_ctx* none = nullptr;   // messages go to lst_last_error(NULL)
  if (!mods || n_mods <= 0 || !conn_off) return fail(none, LST_EINVAL, "lst_load_geometry: empty module table");
  if (n_pix_bins < 0 || (n_pix_bins > 0 && !pix_off)) return fail(none, LST_EINVAL, "lst_load_geometry: bad pixel map");
  if (n_pix_bins > 0 && n_pix_bins != kPixNEta * kPixNPhi * 2)
    return fail(none, LST_EINVAL, "lst_load_geometry: the pixel map must have 100 x 128 x 2 bins");
  if (conn_off[0] != 0) return fail(none, LST_EINVAL, "lst_load_geometry: conn_off[0] != 0");
  int32_t maxdeg = 0;
  for (int32_t m = 0; m < n_mods; ++m) {
    if (mods[m].id != m) return fail(none, LST_EINVAL, "lst_load_geometry: module ids must equal their index");
    if (mods[m].subdet != 0 && mods[m].subdet != 1) return fail(none, LST_EINVAL, "lst_load_geometry: bad subdet");
    if (!(mods[m].spacing > 0.f)) return fail(none, LST_EINVAL, "lst_load_geometry: spacing must be positive");
    const int32_t d = conn_off[m + 1] - conn_off[m];
    if (d < 0) return fail(none, LST_EINVAL, "lst_load_geometry: conn_off not monotone");
    maxdeg = std::max(maxdeg, d);
  }
  if (maxdeg > 256) return fail(none, LST_EINVAL, "lst_load_geometry: a module has more than 256 connections");
  const int32_t n_conn = conn_off[n_mods];
  if (n_conn > 0 && !conn_tgt) return fail(none, LST_EINVAL, "lst_load_geometry: conn_tgt is NULL");
  for (int32_t k = 0; k < n_conn; ++k)
    if (conn_tgt[k] < 0 || conn_tgt[k] >= n_mods)
      return fail(none, LST_EINVAL, "lst_load_geometry: conn_tgt out of range");
  if (n_pix_bins > 0) {
    if (pix_off[0] != 0) return fail(none, LST_EINVAL, "lst_load_geometry: pix_off[0] != 0");
    for (int32_t b = 0; b < n_pix_bins; ++b)
      if (pix_off[b + 1] < pix_off[b]) return fail(none, LST_EINVAL, "lst_load_geometry: pix_off not monotone");
    const int32_t n_pix = pix_off[n_pix_bins];
    if (n_pix > 0 && !pix_tgt) return fail(none, LST_EINVAL, "lst_load_geometry: pix_tgt is NULL");
    for (int32_t k = 0; k < n_pix; ++k)
      if (pix_tgt[k] < 0 || pix_tgt[k] >= n_mods)
        return fail(none, LST_EINVAL, "lst_load_geometry: pix_tgt out of range");
  }
  if (max_degree) *max_degree = maxdeg;
  return LST_OK;
}

int lst_load_geometry(lst_ctx* ctx, const lst_module* mods, int32_t n_mods, const int32_t* conn_off,
                      const int32_t* conn_tgt, const int32_t* pix_off, const int32_t* pix_tgt,
                      int32_t n_pix_bins) {
  if (!ctx) return LST_EINVAL;
  if (ctx->pending) return fail(ctx, LST_ESTATE, "lst_load_geometry: a run is in flight");
  int32_t maxdeg = 0;
  const int vrc = lst_check_geometry(mods, n_mods, conn_off, conn_tgt, pix_off, pix_tgt, n_pix_bins, &maxdeg);
  if (vrc != LST_OK) return fail(ctx, vrc, g_create_error);
  const int32_t n_conn = conn_off[n_mods];
  const int32_t n_pix = n_pix_bins > 0 ? pix_off[n_pix_bins] : 0;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<uint8_t> ec(n_mods);
  std::vector<float> sp(n_mods), pc(n_mods);
  for (int32_t m = 0; m < n_mods; ++m) {
    ec[m] = (uint8_t)mods[m].subdet;
    sp[m] = mods[m].spacing;
    // centre azimuth in [0, 2 pi) (used only to order hits and to centre search windows; any value
    // is valid, a module's true centre keeps its hits away from the wrap at +-pi)
    double c = 0.5 * ((double)mods[m].phi_lo + (double)mods[m].phi_hi);
    c = std::fmod(c, 6.283185307179586);
    if (!(c >= 0.0)) c = std::isfinite(c) ? c + 6.283185307179586 : 0.0;
    pc[m] = (float)c;
  }
  // per connection: the module's centre azimuth minus the connected module's, in (-pi, pi] (the LS
  // kernel maps azimuths between the two modules' frames with it)
  std::vector<float> dpc(std::max<int32_t>(n_conn, 1));
  for (int32_t m = 0; m < n_mods; ++m)
    for (int32_t k = conn_off[m]; k < conn_off[m + 1]; ++k) {
      float d = pc[m] - pc[conn_tgt[k]];
      if (d > 3.14159265f) d -= 6.28318531f;
      if (d <= -3.14159265f) d += 6.28318531f;
      dpc[k] = d;
    }
  Planner pl;
  uint8_t* d_ec = nullptr; float *d_sp = nullptr, *d_pc = nullptr, *d_dpc = nullptr;
  int32_t *d_co = nullptr, *d_ct = nullptr, *d_po = nullptr, *d_pt = nullptr;
  pl.add(d_ec, n_mods); pl.add(d_sp, n_mods); pl.add(d_pc, n_mods); pl.add(d_co, n_mods + 1); pl.add(d_ct, n_conn);
  pl.add(d_dpc, n_conn);
  pl.add(d_po, n_pix_bins + 1); pl.add(d_pt, n_pix);
  const size_t bytes = pl.layout();
  if (ctx->geo_mem) CK(cudaFree(ctx->geo_mem));
  ctx->geo_mem = nullptr;
  ctx->geo_loaded = false;
  CK(cudaMalloc(&ctx->geo_mem, bytes));
  pl.assign(ctx->geo_mem);
  CK(cudaMemcpy(d_ec, ec.data(), n_mods, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_sp, sp.data(), n_mods * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_pc, pc.data(), n_mods * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_co, conn_off, (n_mods + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (n_conn) CK(cudaMemcpy(d_ct, conn_tgt, n_conn * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (n_conn) CK(cudaMemcpy(d_dpc, dpc.data(), n_conn * sizeof(float), cudaMemcpyHostToDevice));
  if (n_pix_bins > 0) {
    CK(cudaMemcpy(d_po, pix_off, (n_pix_bins + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (n_pix) CK(cudaMemcpy(d_pt, pix_tgt, n_pix * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  ctx->geo.n_mods = n_mods;
  ctx->geo.n_pix_bins = n_pix_bins;
  ctx->geo.endcap = d_ec;
  ctx->geo.spacing = d_sp;
  ctx->geo.phic = d_pc;
  ctx->geo.conn_off = d_co;
  ctx->geo.conn_tgt = d_ct;
  ctx->geo.conn_dpc = d_dpc;
  ctx->geo.pix_off = d_po;
  ctx->geo.pix_tgt = d_pt;
  ctx->max_degree = maxdeg;
  ctx->geo.ls_tcap = std::max(32, (maxdeg + 31) / 32 * 32);
  ctx->ls_bps = ls_resident_blocks(ctx->cfg.block_ls, ctx->geo.ls_tcap);
  ctx->t3_bps = t3_pre_resident_blocks();
  ctx->t5_bps = t5_pre_resident_blocks();
  ctx->pt3_bps = pt_pre_resident_blocks(3, ctx->cfg.warps_px);
  ctx->pt5_bps = pt_pre_resident_blocks(5, ctx->cfg.warps_px);
  ctx->geo_loaded = true;
  // arenas depend on the module count
  if (ctx->in_mem) CK(cudaFreeAsync(ctx->in_mem, ctx->stream));
  if (ctx->work_mem) CK(cudaFreeAsync(ctx->work_mem, ctx->stream));
  ctx->in_mem = ctx->work_mem = nullptr;
  ctx->in_caps = Caps{};
  ctx->caps = Caps{};
  ctx->arena_gen++;
  return LST_OK;
}

int lst_reserve(lst_ctx* ctx, int32_t n_events, int32_t max_hits, int32_t max_pls) {
  if (!ctx) return LST_EINVAL;
  if (!ctx->geo_loaded) return fail(ctx, LST_ESTATE, "lst_reserve: no geometry loaded");
  if (ctx->pending) return fail(ctx, LST_ESTATE, "lst_reserve: a run is in flight");
  if (n_events <= 0 || max_hits < 0 || max_pls < 0) return fail(ctx, LST_EINVAL, "lst_reserve: bad sizes");
  CK(cudaSetDevice(ctx->device));
  const int64_t H = (int64_t)n_events * max_hits, P = (int64_t)n_events * max_pls;
  int rc = plan_input(ctx, n_events, H, P);
  if (rc) return rc;
  Caps want = default_caps(n_events, ctx->in_caps.H, ctx->in_caps.P, ctx->geo.n_mods);
  want.E = ctx->in_caps.E;
  return plan_work(ctx, want);
}

int lst_run_events(lst_ctx* ctx, const lst_event_in* ev, int32_t n_ev, lst_event_out* out, void* cuda_stream) {
  if (!ctx) return LST_EINVAL;
  if (!ctx->geo_loaded) return fail(ctx, LST_ESTATE, "lst_run_events: no geometry loaded");
  if (ctx->pending) return fail(ctx, LST_ESTATE, "lst_run_events: the previous run was not synced");
  if (n_ev <= 0 || !ev) return fail(ctx, LST_EINVAL, "lst_run_events: no events");
  int64_t H = 0, P = 0;
  bool any_dev = false, any_host = false;
  for (int32_t e = 0; e < n_ev; ++e) {
    if (ev[e].n_hits < 0 || ev[e].n_pls < 0) return fail(ctx, LST_EINVAL, "lst_run_events: negative size");
    if (ev[e].n_hits > 0 && (!ev[e].x || !ev[e].y || !ev[e].z || !ev[e].sensor))
      return fail(ctx, LST_EINVAL, "lst_run_events: NULL hit array");
    if (ev[e].n_pls > 0 && !ev[e].pls) return fail(ctx, LST_EINVAL, "lst_run_events: NULL seed array");
    if (ev[e].mem_space != LST_MEM_HOST && ev[e].mem_space != LST_MEM_DEVICE &&
        ev[e].mem_space != LST_MEM_HOST_ASYNC)
      return fail(ctx, LST_EINVAL, "lst_run_events: bad mem_space");
    (ev[e].mem_space == LST_MEM_DEVICE ? any_dev : any_host) = true;
    H += ev[e].n_hits;
    P += ev[e].n_pls;
  }
  if (H >= (1ll << 29) || P >= (1ll << 28)) return fail(ctx, LST_EINVAL, "lst_run_events: batch too large");
  if (any_dev && any_host) return fail(ctx, LST_EINVAL, "lst_run_events: mixed host and device events");
  CK(cudaSetDevice(ctx->device));
  ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
  int rc = plan_input(ctx, n_ev, H, P);
  if (rc) return rc;
  if (!ctx->work_mem || ctx->caps.E != ctx->in_caps.E || H > ctx->caps.H || P > ctx->caps.P) {
    Caps want = default_caps(std::max<int64_t>(n_ev, ctx->caps.E), std::max<int64_t>(ctx->in_caps.H, ctx->caps.H),
                             std::max<int64_t>(ctx->in_caps.P, ctx->caps.P), ctx->geo.n_mods);
    want.E = std::max<int64_t>(ctx->in_caps.E, want.E);
    rc = plan_work(ctx, want);
    if (rc) return rc;
  }
  ctx->E = n_ev;
  ctx->H = (int32_t)H;
  ctx->P = (int32_t)P;
  ctx->ev_hits.resize(n_ev);
  ctx->ev_pls.resize(n_ev);
  // event offsets padded with empty events up to the arena's event capacity
  const int32_t Ecap = (int32_t)ctx->in_caps.E;
  std::vector<int32_t> hoff(Ecap + 1, 0), poff(Ecap + 1, 0);
  for (int32_t e = 0; e < Ecap; ++e) {
    hoff[e + 1] = hoff[e] + (e < n_ev ? ev[e].n_hits : 0);
    poff[e + 1] = poff[e] + (e < n_ev ? ev[e].n_pls : 0);
  }
  for (int32_t e = 0; e < n_ev; ++e) {
    ctx->ev_hits[e] = ev[e].n_hits;
    ctx->ev_pls[e] = ev[e].n_pls;
  }
  Ws& w = ctx->ws;
  // stage the inputs. Device events, and LST_MEM_HOST_ASYNC events the GPU can read where they are
  // (pinned, or pageable with coherent access), are gathered by one kernel straight into the input
  // arena; other host events are packed into the context's pinned buffer before this call returns and
  // copied with one transfer per array.
  std::vector<EvPtr> views(n_ev);
  bool direct = true;
  for (int32_t e = 0; e < n_ev; ++e) {
    if (ev[e].mem_space == LST_MEM_DEVICE) {
      views[e] = EvPtr{ev[e].x, ev[e].y, ev[e].z, ev[e].sensor, ev[e].pls};
      continue;
    }
    if (ev[e].mem_space == LST_MEM_HOST) {
      direct = false;
      continue;
    }
    views[e] = EvPtr{static_cast<const float*>(device_view(ev[e].x, ctx->pageable_access)),
                     static_cast<const float*>(device_view(ev[e].y, ctx->pageable_access)),
                     static_cast<const float*>(device_view(ev[e].z, ctx->pageable_access)),
                     static_cast<const int32_t*>(device_view(ev[e].sensor, ctx->pageable_access)),
                     static_cast<const lst_pls*>(device_view(ev[e].pls, ctx->pageable_access))};
    if ((ev[e].n_hits && (!views[e].x || !views[e].y || !views[e].z || !views[e].sensor)) ||
        (ev[e].n_pls && !views[e].pls))
      direct = false;
  }
  if (direct) any_host = false;
  const size_t off_bytes = 2 * ((size_t)Ecap + 1) * sizeof(int32_t);
  const size_t host_bytes = any_host ? (size_t)H * 16 + (size_t)P * sizeof(lst_pls) : 0;
  rc = ensure_pinned(ctx, off_bytes + host_bytes + (size_t)n_ev * sizeof(EvPtr) + 64);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));   // the staging buffer may still feed the previous copy
  char* hp = static_cast<char*>(ctx->pinned);
  std::memcpy(hp, hoff.data(), ((size_t)Ecap + 1) * sizeof(int32_t));
  std::memcpy(hp + ((size_t)Ecap + 1) * sizeof(int32_t), poff.data(), ((size_t)Ecap + 1) * sizeof(int32_t));
  CK(cudaMemcpyAsync(w.ev_hit_off, hp, off_bytes, cudaMemcpyHostToDevice, ctx->stream));
  if (any_host) {
    float* hx = reinterpret_cast<float*>(hp + off_bytes);
    float* hy = hx + H;
    float* hz = hy + H;
    int32_t* hs = reinterpret_cast<int32_t*>(hz + H);
    lst_pls* hpl = reinterpret_cast<lst_pls*>(hs + H);
    for (int32_t e = 0; e < n_ev; ++e) {
      const size_t n = ev[e].n_hits, o = hoff[e];
      if (n) {
        std::memcpy(hx + o, ev[e].x, n * sizeof(float));
        std::memcpy(hy + o, ev[e].y, n * sizeof(float));
        std::memcpy(hz + o, ev[e].z, n * sizeof(float));
        std::memcpy(hs + o, ev[e].sensor, n * sizeof(int32_t));
      }
      if (ev[e].n_pls) std::memcpy(hpl + poff[e], ev[e].pls, ev[e].n_pls * sizeof(lst_pls));
    }
    if (H) {
      CK(cudaMemcpyAsync(w.x, hx, H * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(w.y, hy, H * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(w.z, hz, H * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(w.sensor, hs, H * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (P) CK(cudaMemcpyAsync(w.pls, hpl, P * sizeof(lst_pls), cudaMemcpyHostToDevice, ctx->stream));
  } else {
    if (n_ev > ctx->tab_cap) {
      if (ctx->d_tab) CK(cudaFreeAsync(ctx->d_tab, ctx->stream));
      ctx->d_tab = nullptr;
      CK(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ctx->d_tab), n_ev * sizeof(EvPtr), ctx->pool, ctx->stream));
      ctx->tab_cap = n_ev;
    }
    EvPtr* ht = reinterpret_cast<EvPtr*>(hp + off_bytes);
    for (int32_t e = 0; e < n_ev; ++e) ht[e] = views[e];
    CK(cudaMemcpyAsync(ctx->d_tab, ht, n_ev * sizeof(EvPtr), cudaMemcpyHostToDevice, ctx->stream));
    w.E = Ecap;
    if (H + P > 0) {
      k_gather<<<grid_for(H + P, 256), 256, 0, ctx->stream>>>(ctx->d_tab, w, (int)H, (int)P);
      ctx->launches++;
    }
  }
  // capacity overrides belong to one batch
  const int64_t V = (int64_t)Ecap * ctx->geo.n_mods;
  CK(cudaMemsetAsync(w.md_ovr, 0, V * sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(w.ls_ovr, 0, V * sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(w.t3_ovr, 0, V * sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(w.t5_ovr, 0, V * sizeof(int32_t), ctx->stream));
  ctx->retries = 0;
  std::memset(ctx->first_ovf, 0, sizeof(ctx->first_ovf));
  ctx->user_out = out;
  CK(cudaMemcpyAsync(const_cast<float*>(w.stage_scale), ctx->stage_scale, sizeof(ctx->stage_scale),
                     cudaMemcpyHostToDevice, ctx->stream));
  rc = launch_chain(ctx);
  if (rc) return rc;
  ctx->pending = true;
  return LST_OK;
}

int lst_query(lst_ctx* ctx) {
  if (!ctx) return -LST_EINVAL;
  if (!ctx->pending) return 1;
  cudaError_t e = cudaEventQuery(ctx->ev_done);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  fail(ctx, LST_ECUDA, std::string("lst_query: ") + cudaGetErrorString(e));
  return -LST_ECUDA;
}

int lst_sync(lst_ctx* ctx, int32_t* status_per_event) {
  if (!ctx) return LST_EINVAL;
  if (!ctx->pending) return fail(ctx, LST_ESTATE, "lst_sync: nothing to wait for");
  CK(cudaSetDevice(ctx->device));
  for (;;) {
    cudaError_t e = cudaEventSynchronize(ctx->ev_done);
    if (e != cudaSuccess) {
      ctx->pending = false;
      return fail(ctx, LST_ECUDA, std::string("lst_sync: ") + cudaGetErrorString(e));
    }
    const int32_t* st = ctx->h_status;
    if (ctx->retries == 0) {
      ctx->first_ovf[LST_STAGE_MD] = st[ST_OVF_MD];
      ctx->first_ovf[LST_STAGE_LS] = st[ST_OVF_LS];
      ctx->first_ovf[LST_STAGE_T3] = st[ST_OVF_T3];
      ctx->first_ovf[LST_STAGE_T5] = st[ST_OVF_T5];
      ctx->first_ovf[LST_STAGE_PT3] = std::max<int64_t>(0, (int64_t)st[ST_N_PT3] - ctx->caps.p3_slots);
      ctx->first_ovf[LST_STAGE_PT5] = std::max<int64_t>(0, (int64_t)st[ST_N_PT5] - ctx->caps.p5_slots);
      // slot arenas too small for the predicted capacities
      const int64_t arena_need[8] = {st[ST_ARENA_MD], st[ST_ARENA_LS], st[ST_ARENA_T3], st[ST_ARENA_T5],
                                     st[ST_DENSE_MD], st[ST_DENSE_LS], st[ST_DENSE_T3], st[ST_DENSE_T5]};
      const int64_t arena_cap[8] = {ctx->caps.md_slots, ctx->caps.ls_slots, ctx->caps.t3_slots, ctx->caps.t5_slots,
                                    ctx->caps.md_dense, ctx->caps.ls_dense, ctx->caps.t3_dense, ctx->caps.t5_dense};
      for (int k = 0; k < 8; ++k)
        if (arena_need[k] > arena_cap[k]) ctx->first_ovf[k % 4] += (int)(arena_need[k] - arena_cap[k]);
      // float64 decision queues
      const int64_t qn[6] = {st[ST_Q_MD], st[ST_Q_LS], st[ST_Q_T3], st[ST_Q_T5], st[ST_Q_PT3], st[ST_Q_PT5]};
      const int64_t qc[6] = {ctx->caps.q_md, ctx->caps.q_ls, ctx->caps.q_t3, ctx->caps.q_t5, ctx->caps.q_p3, ctx->caps.q_p5};
      for (int k = 0; k < 6; ++k)
        if (qn[k] > qc[k]) ctx->first_ovf[LST_STAGE_QUEUE] += (int)(qn[k] - qc[k]);
    }
    // capacity problems: grow arenas / queues, raise per-module capacities, run again
    Caps c = ctx->caps;
    bool grow = false, raise = false;
    auto need = [&](int64_t used, int64_t& cap) {
      if (used > cap) { cap = std::max<int64_t>(used + used / 4, 2 * cap); grow = true; }
    };
    need(st[ST_ARENA_MD], c.md_slots);
    need(st[ST_ARENA_LS], c.ls_slots);
    need(st[ST_ARENA_T3], c.t3_slots);
    need(st[ST_ARENA_T5], c.t5_slots);
    need(st[ST_DENSE_MD], c.md_dense);
    need(st[ST_DENSE_LS], c.ls_dense);
    need(st[ST_DENSE_T3], c.t3_dense);
    need(st[ST_DENSE_T5], c.t5_dense);
    need(st[ST_N_PT3], c.p3_slots);
    need(st[ST_N_PT5], c.p5_slots);
    need(st[ST_Q_MD], c.q_md);
    need(st[ST_Q_LS], c.q_ls);
    need(st[ST_Q_T3], c.q_t3);
    need(st[ST_Q_T5], c.q_t5);
    need(st[ST_Q_PT3], c.q_p3);
    need(st[ST_Q_PT5], c.q_p5);
    raise = st[ST_OVF_MD] || st[ST_OVF_LS] || st[ST_OVF_T3] || st[ST_OVF_T5];
    if (!(st[ST_ERROR]) && !st[ST_TIMEOUT] && (grow || raise)) {
      if (ctx->retries >= ctx->cfg.max_retries) {
        ctx->pending = false;
        for (int32_t ev = 0; ev < ctx->E; ++ev) {
          if (status_per_event) status_per_event[ev] = LST_EOVERFLOW_UNRESOLVED;
        }
        return fail(ctx, LST_EOVERFLOW_UNRESOLVED, "lst_sync: object capacity still exceeded after retries");
      }
      ctx->retries++;
      const int ovf_word[4] = {ST_OVF_MD, ST_OVF_LS, ST_OVF_T3, ST_OVF_T5};
      for (int k = 0; k < 4; ++k)
        if (st[ovf_word[k]]) ctx->stage_scale[k] = std::min(ctx->stage_scale[k] * 1.5f, 8.0f);
      if (raise) {
        const int V = (int)ctx->caps.E * ctx->geo.n_mods;
        const Ws& w = ctx->ws;
        if (st[ST_OVF_MD]) k_raise<<<grid_for(V, 256), 256, 0, ctx->stream>>>(w.md_cnt, w.md_ovr, V);
        if (st[ST_OVF_LS]) k_raise<<<grid_for(V, 256), 256, 0, ctx->stream>>>(w.ls_cnt, w.ls_ovr, V);
        if (st[ST_OVF_T3]) k_raise<<<grid_for(V, 256), 256, 0, ctx->stream>>>(w.t3_cnt, w.t3_ovr, V);
        if (st[ST_OVF_T5]) k_raise<<<grid_for(V, 256), 256, 0, ctx->stream>>>(w.t5_cnt, w.t5_ovr, V);
        ctx->launches += 4;
      }
      if (grow) {
        int rc = plan_work(ctx, c);
        if (rc) { ctx->pending = false; return rc; }
      }
      int rc = launch_chain(ctx);
      if (rc) { ctx->pending = false; return rc; }
      continue;
    }
    break;
  }
  ctx->pending = false;
  // per-event results
  const int32_t* st = ctx->h_status;
  ctx->counts.assign(ctx->E, lst_counts{});
  ctx->outs.assign(ctx->E, lst_event_out{});
  int first_err = LST_OK;
  if (ctx->timing) {
    for (int s = 0; s < LST_N_STAGES + 1; ++s) ctx->stage_ms[s] = 0.f;
    float ms;
    const int map[7] = {LST_STAGE_MD, LST_STAGE_LS, LST_STAGE_T3, LST_STAGE_T5, LST_STAGE_PT3, LST_STAGE_TC, LST_STAGE_QUEUE};
    for (int k = 0; k < 7; ++k)
      if (cudaEventElapsedTime(&ms, ctx->ev_stage[k], ctx->ev_stage[k + 1]) == cudaSuccess) ctx->stage_ms[map[k]] += ms;
    if (cudaEventElapsedTime(&ms, ctx->ev_stage[0], ctx->ev_stage[7]) == cudaSuccess) ctx->stage_ms[LST_N_STAGES] = ms;
    for (int k = 0; k < K_N_TIMED; ++k) {
      ctx->kern_ms[k] = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev_kern[2 * k], ctx->ev_kern[2 * k + 1]) == cudaSuccess) ctx->kern_ms[k] = ms;
    }
    // the pT3 and pT5 kernels interleave in one pixel stage: pT5's share is its two candidate
    // kernels, the rest (seed preparation, module boxes, pT3 kernels, grouping) stays with pT3
    const float pt5 = ctx->kern_ms[K_PT5_PRE] + ctx->kern_ms[K_PT5_DECIDE];
    if (pt5 > 0.f && pt5 <= ctx->stage_ms[LST_STAGE_PT3]) {
      ctx->stage_ms[LST_STAGE_PT5] = pt5;
      ctx->stage_ms[LST_STAGE_PT3] -= pt5;
    }
  }
  const Ws& w = ctx->ws;
  for (int32_t ev = 0; ev < ctx->E; ++ev) {
    const int32_t* es = st + ST_N_WORDS + ev * kEvWords;
    lst_counts& c = ctx->counts[ev];
    c.n_hits = ctx->ev_hits[ev];
    c.n_pls = ctx->ev_pls[ev];
    c.n_md = es[0]; c.n_ls = es[1]; c.n_t3 = es[2]; c.n_t5 = es[3]; c.n_pt3 = es[4]; c.n_pt5 = es[5]; c.n_tc = es[6];
    for (int k = 0; k < 4; ++k) c.n_tc_type[k] = es[7 + k];
    c.n_tc_ext = es[kEvExt];
    c.n_ls_pairs = (int64_t)(((uint64_t)(uint32_t)st[ST_LS_PAIRS_HI] << 32) | (uint32_t)st[ST_LS_PAIRS]);
    for (int s = 0; s < LST_N_STAGES; ++s) c.overflow[s] = ctx->first_ovf[s];
    c.recheck[LST_STAGE_MD] = st[ST_REC_MD];
    c.recheck[LST_STAGE_LS] = st[ST_REC_LS];
    c.recheck[LST_STAGE_T3] = st[ST_Q_T3];
    c.recheck[LST_STAGE_T5] = st[ST_Q_T5];
    c.recheck[LST_STAGE_PT3] = st[ST_Q_PT3];
    c.recheck[LST_STAGE_PT5] = st[ST_Q_PT5];
    c.retries = ctx->retries;
    c.status = es[kEvErr] ? LST_EINVAL : (st[ST_TIMEOUT] ? LST_ETIMEOUT : LST_OK);
    if (c.status == LST_ETIMEOUT && !first_err) {
      first_err = c.status;
      ctx->err = "lst_sync: " + std::to_string(st[ST_TIMEOUT]) +
                 " warps of the candidate kernels ran out of their cycle budget; results are incomplete";
    } else if (c.status && !first_err) {
      first_err = c.status;
      ctx->err = "lst_sync: invalid input in event " + std::to_string(ev) +
                 ((es[kEvErr] & ERR_BAD_SENSOR) ? " (sensor id out of range)" : "") +
                 ((es[kEvErr] & ERR_BAD_COORD) ? " (non-finite coordinate)" : "") +
                 ((es[kEvErr] & ERR_BAD_PLS) ? " (bad pixel seed)" : "");
    }
    if (status_per_event) status_per_event[ev] = c.status;
    lst_event_out& o = ctx->outs[ev];
    o.counts = c;
    const int bmd = es[11], bls = es[12], bt3 = es[13], bt5 = es[14], bp3 = es[15], bp5 = es[16], btc = es[17];
    const int64_t S5 = ctx->caps.t5_dense;
    o.md_hit_lo = w.o_md_lo + bmd; o.md_hit_up = w.o_md_up + bmd; o.md_module = w.o_md_mod + bmd;
    // float32 output columns, or their binary16 twins (the other pointer NULL)
    auto f32 = [](const float* a, int64_t off) -> const float* { return a ? a + off : nullptr; };
    auto f16 = [](const uint16_t* a, int64_t off) -> const uint16_t* { return a ? a + off : nullptr; };
    o.md_dphichange = f32(w.md_dpc, bmd); o.md_pt_est = f32(w.md_pte, bmd);
    o.md_dphichange_h = f16(w.md_dpc_h, bmd); o.md_pt_est_h = f16(w.md_pte_h, bmd);
    o.ls_md_in = w.o_ls_in + bls; o.ls_md_out = w.o_ls_out + bls;
    o.ls_z0 = f32(w.ls_z0, bls); o.ls_dphi = f32(w.ls_dphi, bls);
    o.ls_z0_h = f16(w.ls_z0_h, bls); o.ls_dphi_h = f16(w.ls_dphi_h, bls);
    o.t3_ls_in = w.o_t3_a + bt3; o.t3_ls_out = w.o_t3_b + bt3; o.t3_r = w.t3_R + bt3;
    o.t3_xc = f32(w.t3_xc, bt3); o.t3_yc = f32(w.t3_yc, bt3); o.t3_chi2_rz = f32(w.t3_chi2, bt3);
    o.t3_pt_est = f32(w.t3_pte, bt3);
    o.t3_xc_h = f16(w.t3_xc_h, bt3); o.t3_yc_h = f16(w.t3_yc_h, bt3); o.t3_chi2_rz_h = f16(w.t3_chi2_h, bt3);
    o.t3_pt_est_h = f16(w.t3_pte_h, bt3);
    o.t5_t3_in = w.o_t5_a + bt5; o.t5_t3_out = w.o_t5_b + bt5;
    const bool h5 = w.t5_h != nullptr;
    o.t5_kappa_in = h5 ? nullptr : w.t5_f + 0 * S5 + bt5; o.t5_kappa_out = h5 ? nullptr : w.t5_f + 1 * S5 + bt5;
    o.t5_kappa_fit = w.t5_f + 2 * S5 + bt5; o.t5_chi2_c = w.t5_f + 3 * S5 + bt5;
    o.t5_chi2_rz = h5 ? nullptr : w.t5_f + 4 * S5 + bt5; o.t5_eta = w.t5_f + 5 * S5 + bt5;
    o.t5_phi = w.t5_f + 6 * S5 + bt5; o.t5_pt = w.t5_f + 7 * S5 + bt5;
    o.t5_kappa_in_h = h5 ? w.t5_h + 0 * S5 + bt5 : nullptr; o.t5_kappa_out_h = h5 ? w.t5_h + 1 * S5 + bt5 : nullptr;
    o.t5_chi2_rz_h = h5 ? w.t5_h + 2 * S5 + bt5 : nullptr;
    o.pt3_pls = w.o_pt3_pls + bp3; o.pt3_t3 = w.o_pt3_obj + bp3;
    o.pt3_chi2_xy = f32(w.pt3_xy, bp3); o.pt3_chi2_rz = f32(w.pt3_rz, bp3);
    o.pt3_chi2_xy_h = f16(w.pt3_xy_h, bp3); o.pt3_chi2_rz_h = f16(w.pt3_rz_h, bp3);
    o.pt5_pls = w.o_pt5_pls + bp5; o.pt5_t5 = w.o_pt5_obj + bp5;
    o.pt5_chi2_xy = f32(w.pt5_xy, bp5); o.pt5_chi2_rz = f32(w.pt5_rz, bp5);
    o.pt5_chi2_xy_h = f16(w.pt5_xy_h, bp5); o.pt5_chi2_rz_h = f16(w.pt5_rz_h, bp5);
    o.tc_type = w.tcd_type + btc; o.tc_obj = w.tcd_obj + btc; o.tc_hits = w.tcd_hits + (int64_t)btc * 14;
    o.tc_pt = w.tcd_pt + btc; o.tc_eta = w.tcd_eta + btc; o.tc_phi = w.tcd_phi + btc;
    o.tc_ext_t3 = w.tcd_ext_t3 + btc; o.tc_ext_n_md = w.tcd_ext_n + btc;
    o.tc_ext_hits = w.tcd_ext_hits + (int64_t)btc * 4;
    o.tc_ext_chi2_c = w.tcd_ext_c + btc; o.tc_ext_chi2_rz = w.tcd_ext_rz + btc;
    if (ctx->user_out) ctx->user_out[ev] = o;
  }
  return first_err;
}

int lst_bin_hits(lst_ctx* ctx, const int32_t* d_sensor, int32_t n_hits, int32_t* d_order, int32_t* d_offsets,
                 void* cuda_stream) {
  if (!ctx) return LST_EINVAL;
  if (!ctx->geo_loaded) return fail(ctx, LST_ESTATE, "lst_bin_hits: no geometry loaded");
  if (n_hits < 0 || (n_hits > 0 && (!d_sensor || !d_order)) || !d_offsets)
    return fail(ctx, LST_EINVAL, "lst_bin_hits: bad arguments");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
  const int n_sens = 2 * ctx->geo.n_mods;
  const size_t words = 2 * (size_t)n_sens + 1 + (size_t)scan_tmp_elems(n_sens + 1) + 8;
  if (words > ctx->bin_words) {
    if (ctx->bin_mem) CK(cudaFreeAsync(ctx->bin_mem, st));
    ctx->bin_mem = nullptr;
    CK(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ctx->bin_mem), words * sizeof(int32_t), ctx->pool, st));
    ctx->bin_words = words;
  }
  int32_t* cnt = ctx->bin_mem;
  int32_t* cur = cnt + n_sens;
  int32_t* err = cur + n_sens;
  int32_t* tmp = err + 1;
  CK(cudaMemsetAsync(cnt, 0, (2 * (size_t)n_sens + 1) * sizeof(int32_t), st));
  Launch L = make_launch(ctx);
  L.stream = st;
  run_bin_raw(d_sensor, n_hits, n_sens, d_order, d_offsets, cnt, cur, err, tmp, L);
  int32_t herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(ctx, LST_EINVAL, "lst_bin_hits: sensor id out of range");
  return LST_OK;
}

int lst_get_counts(const lst_ctx* ctx, int32_t ev, lst_counts* c) {
  if (!ctx || !c) return LST_EINVAL;
  if (ev < 0 || ev >= (int32_t)ctx->counts.size()) return LST_EINVAL;
  *c = ctx->counts[ev];
  return LST_OK;
}

int lst_copy_tc(lst_ctx* ctx, int32_t ev, int32_t* type, int32_t* obj, int32_t* hits, float* pt, float* eta,
                float* phi) {
  if (!ctx) return LST_EINVAL;
  if (ev < 0 || ev >= (int32_t)ctx->outs.size()) return fail(ctx, LST_EINVAL, "lst_copy_tc: no such event");
  CK(cudaSetDevice(ctx->device));
  const lst_event_out& o = ctx->outs[ev];
  const size_t n = o.counts.n_tc;
  if (n == 0) return LST_OK;
  if (type) CK(cudaMemcpyAsync(type, o.tc_type, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (obj) CK(cudaMemcpyAsync(obj, o.tc_obj, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (hits) CK(cudaMemcpyAsync(hits, o.tc_hits, n * 14 * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (pt) CK(cudaMemcpyAsync(pt, o.tc_pt, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (eta) CK(cudaMemcpyAsync(eta, o.tc_eta, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (phi) CK(cudaMemcpyAsync(phi, o.tc_phi, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LST_OK;
}

int lst_copy_tc_ext(lst_ctx* ctx, int32_t ev, int32_t* t3, int32_t* n_md, int32_t* hits, float* chi2_c,
                    float* chi2_rz) {
  if (!ctx) return LST_EINVAL;
  if (ev < 0 || ev >= (int32_t)ctx->outs.size()) return fail(ctx, LST_EINVAL, "lst_copy_tc_ext: no such event");
  CK(cudaSetDevice(ctx->device));
  const lst_event_out& o = ctx->outs[ev];
  const size_t n = o.counts.n_tc;
  if (n == 0) return LST_OK;
  if (t3) CK(cudaMemcpyAsync(t3, o.tc_ext_t3, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (n_md) CK(cudaMemcpyAsync(n_md, o.tc_ext_n_md, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (hits) CK(cudaMemcpyAsync(hits, o.tc_ext_hits, n * 4 * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (chi2_c) CK(cudaMemcpyAsync(chi2_c, o.tc_ext_chi2_c, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (chi2_rz) CK(cudaMemcpyAsync(chi2_rz, o.tc_ext_chi2_rz, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LST_OK;
}

int64_t lst_tc_total(const lst_ctx* ctx) {
  if (!ctx) return -LST_EINVAL;
  int64_t n = 0;
  for (const lst_counts& c : ctx->counts) n += c.n_tc;
  return n;
}

int lst_copy_tc_all(lst_ctx* ctx, int32_t* offsets, int32_t* type, int32_t* obj, int32_t* hits, float* pt,
                    float* eta, float* phi) {
  if (!ctx) return LST_EINVAL;
  if (ctx->outs.empty()) return fail(ctx, LST_ESTATE, "lst_copy_tc_all: no completed run");
  CK(cudaSetDevice(ctx->device));
  const int32_t E = (int32_t)ctx->outs.size();
  const int64_t n = lst_tc_total(ctx);
  if (offsets) {
    int64_t acc = 0;
    for (int32_t e = 0; e < E; ++e) {
      offsets[e] = (int32_t)acc;
      acc += ctx->counts[e].n_tc;
    }
    offsets[E] = (int32_t)acc;
  }
  if (n == 0) return LST_OK;
  const Ws& w = ctx->ws;
  // rows of events 0..E-1 are contiguous from row 0 of the dense arrays
  if (type) CK(cudaMemcpyAsync(type, w.tcd_type, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (obj) CK(cudaMemcpyAsync(obj, w.tcd_obj, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (hits) CK(cudaMemcpyAsync(hits, w.tcd_hits, n * 14 * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (pt) CK(cudaMemcpyAsync(pt, w.tcd_pt, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (eta) CK(cudaMemcpyAsync(eta, w.tcd_eta, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  if (phi) CK(cudaMemcpyAsync(phi, w.tcd_phi, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LST_OK;
}

int lst_set_timing(lst_ctx* ctx, int enable) {
  if (!ctx) return LST_EINVAL;
  ctx->timing = enable != 0;
  return LST_OK;
}

int lst_get_stage_ms(const lst_ctx* ctx, float* stage_ms) {
  if (!ctx || !stage_ms) return LST_EINVAL;
  for (int s = 0; s < LST_N_STAGES + 1; ++s) stage_ms[s] = ctx->stage_ms[s];
  return LST_OK;
}

int lst_get_kernel_ms(const lst_ctx* ctx, float* ms, int32_t n) {
  if (!ctx || !ms || n < 0) return LST_EINVAL;
  for (int k = 0; k < n && k < K_N_TIMED; ++k) ms[k] = ctx->kern_ms[k];
  return K_N_TIMED;
}

int64_t lst_predict_bytes(const lst_ctx* ctx, int32_t n_events, int64_t n_hits, int64_t n_pls) {
  if (!ctx || !ctx->geo_loaded || n_events <= 0 || n_hits < 0 || n_pls < 0) return -LST_EINVAL;
  Caps c = default_caps(n_events, n_hits, n_pls, ctx->geo.n_mods);
  c.half = ctx->cfg.half_floats != 0;
  Ws tmp{};
  size_t zb = 0;
  const size_t work = layout_work(tmp, c, ctx->geo.n_mods, nullptr, &zb);
  const size_t in = (size_t)n_hits * 16 + (size_t)n_pls * sizeof(lst_pls) + 8 * (size_t)(n_events + 1) +
                    16 * (size_t)n_events * ctx->geo.n_mods;
  return (int64_t)(work + in);
}

int64_t lst_launch_count(const lst_ctx* ctx) { return ctx ? ctx->launches : 0; }

int lst_selftest_bounded_wait(int device, int32_t* gave_up) {
  if (!gave_up) return LST_EINVAL;
  *gave_up = 0;
  return scan_wait_selftest(device, gave_up) == 0 ? LST_OK : LST_ECUDA;
}

const char* lst_last_error(const lst_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"
