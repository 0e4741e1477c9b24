// Internal layout of the LST library: resident geometry, the per-batch workspace, status words and
// the host-side launchers of each stage. Shared by the .cu files of the library; not installed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lst.h"
#include "lst_common.cuh"

namespace lst {

// Resident geometry (device pointers).
struct Geo {
  int32_t n_mods = 0;
  int32_t n_pix_bins = 0;
  const uint8_t* endcap = nullptr;   // [n_mods] 1 for endcap modules
  const float* spacing = nullptr;    // [n_mods]
  const float* phic = nullptr;       // [n_mods] centre azimuth of each module, (phi_lo + phi_hi) / 2
  int32_t ls_tcap = 32;              // connected-module slots per warp of the LS kernel: the largest
                                     // module-map degree rounded up to 32
  const int32_t* conn_off = nullptr; // [n_mods + 1]
  const int32_t* conn_tgt = nullptr;
  const float* conn_dpc = nullptr;   // [conn_off[n_mods]] centre azimuth of the module minus that of
                                     // the connected module, wrapped to (-pi, pi]
  const int32_t* pix_off = nullptr;  // [n_pix_bins + 1]
  const int32_t* pix_tgt = nullptr;
};

// Status words (int32, device; copied to the host after each run).
enum StatusWord : int {
  ST_ERROR = 0,          // bit flags, below
  ST_OVF_MD, ST_OVF_LS, ST_OVF_T3, ST_OVF_T5, ST_OVF_PT3, ST_OVF_PT5,   // objects beyond capacity
  ST_ARENA_MD, ST_ARENA_LS, ST_ARENA_T3, ST_ARENA_T5, ST_ARENA_PT3, ST_ARENA_PT5,  // slot totals
  ST_Q_MD, ST_Q_LS, ST_Q_T3, ST_Q_T5, ST_Q_PT3, ST_Q_PT5,   // queue pushes attempted
  ST_REC_MD, ST_REC_LS,  // float64 re-decisions of MD / LS candidates
  ST_N_PT3, ST_N_PT5,    // appended pT3 / pT5 objects
  ST_DENSE_MD, ST_DENSE_LS, ST_DENSE_T3, ST_DENSE_T5,   // dense totals beyond the dense capacity
  ST_TIMEOUT,            // blocks that ran out of their cycle budget
  ST_LS_PAIRS,           // (with the next word: one 64-bit count) (inner MD, outer MD) pairs the LS
  ST_LS_PAIRS_HI,        //   kernel evaluated, inside its azimuth windows
  ST_N_WORDS
};
static_assert(ST_LS_PAIRS % 2 == 0, "the 64-bit pair count needs an 8-byte aligned word");
enum ErrorBit : int { ERR_BAD_SENSOR = 1, ERR_BAD_COORD = 2, ERR_BAD_PLS = 4 };

// Per-event summary written by the final kernel: object counts [0..6] (MD, LS, T3, T5, pT3, pT5, TC),
// TC counts per type [7..10], first dense index of the event in each object array [11..17]
// (same order; TC: first row), extended TCs [kEvExt], error bits [kEvErr].
constexpr int kEvWords = 24;
constexpr int kEvErr = 23;
constexpr int kEvExt = 18;
constexpr int kExtRefs = 16;   // candidate references stored per track candidate

// Capacities of one workspace (element counts).
struct Caps {
  int64_t E = 0, H = 0, P = 0;
  int64_t md_slots = 0, ls_slots = 0, t3_slots = 0, t5_slots = 0, p3_slots = 0, p5_slots = 0;
  int64_t md_dense = 0, ls_dense = 0, t3_dense = 0, t5_dense = 0;   // dense (compacted) objects
  int64_t q_md = 0, q_ls = 0, q_t3 = 0, q_t5 = 0, q_p3 = 0, q_p5 = 0;
  int64_t n_mods = 0;
  int64_t half = 0;   // 1: the output-only per-object floats are stored as binary16
};

// Per-batch workspace: every device array the chain uses. Passed to kernels by value.
struct Ws {
  // capacities of the launch shape (events, virtual modules / sensors, hits, seeds); the actual
  // counts are on the device: event offsets are padded with empty events up to E
  int32_t E = 0, V = 0, S = 0, H = 0, P = 0;
  __device__ __forceinline__ int n_hits() const { return ev_hit_off[E]; }
  __device__ __forceinline__ int n_pls() const { return ev_pls_off[E]; }
  Caps cap;
  float cap_scale = 1.0f;
  const float* stage_scale = nullptr;   // [4] device: adaptive capacity multipliers (MD, LS, T3, T5)
  long long cycle_budget = 0;
  // inputs (concatenated events)
  float *x = nullptr, *y = nullptr, *z = nullptr;
  int32_t* sensor = nullptr;
  int32_t* ev_hit_off = nullptr;  // [E + 1]
  int32_t* ev_pls_off = nullptr;  // [E + 1]
  lst_pls* pls = nullptr;
  // binning
  int32_t *hit_vs = nullptr, *sens_cnt = nullptr, *sens_off = nullptr, *sens_cur = nullptr;
  int32_t* bidx = nullptr;
  float *bx = nullptr, *by = nullptr, *bz = nullptr;
  int32_t* borig = nullptr;
  // MD
  int32_t *md_cap = nullptr, *md_base = nullptr, *md_cnt = nullptr, *md_ovr = nullptr;
  int32_t *ms_lo = nullptr, *ms_up = nullptr;
  float *ms_dpc = nullptr, *ms_pte = nullptr;
  int32_t* md_off = nullptr;
  int32_t *md_lo = nullptr, *md_up = nullptr, *md_vm = nullptr;
  float4* md_xyzr = nullptr;     // [md_dense] (x, y, z, r) of each MD anchor (the lower hit)
  float *md_rlo = nullptr;       // [md_dense] r + md_rlo = the anchor radius to ~2^-47 (float pair)
  float2* md_sa = nullptr;       // [md_dense] (arc length at R_thr, alpha_thr(r) = asin(min(r k / (2 pT_thr), sin_max)))
  float *md_dpc = nullptr, *md_pte = nullptr;
  uint8_t* md_ec = nullptr;
  // binary16 storage of the output-only per-object floats (lst_config.half_floats; nullptr
  // otherwise, and then their float32 arrays are used): MD dPhiChange, pT estimate; LS z0, dphi;
  // T3 centre, r-z chi2, pT estimate; T5 kappa_in, kappa_out, r-z chi2 ([3][t5_dense]); pT3 / pT5
  // chi2_xy, chi2_rz
  uint16_t *md_dpc_h = nullptr, *md_pte_h = nullptr, *ls_z0_h = nullptr, *ls_dphi_h = nullptr;
  uint16_t *t3_xc_h = nullptr, *t3_yc_h = nullptr, *t3_chi2_h = nullptr, *t3_pte_h = nullptr, *t5_h = nullptr;
  uint16_t *pt3_xy_h = nullptr, *pt3_rz_h = nullptr, *pt5_xy_h = nullptr, *pt5_rz_h = nullptr;
  float* md_rphi = nullptr;      // [md_dense] anchor azimuth relative to its module's centre, (-pi, pi]:
                                 // the MDs of a module are ordered by it (hits are binned in azimuth order)
  int32_t *md_rmin = nullptr, *md_rmax = nullptr;   // [V] smallest / largest anchor radius of each
                                                    // module's MDs (float bits; set by k_md_dense)
  float2* md_win = nullptr;   // [V] (alpha_thr of the largest anchor radius, 1 / the smallest) of each
                              // module's MDs, the LS azimuth windows' inputs (set by k_ls_caps)
  // LS
  int32_t *ls_cap = nullptr, *ls_base = nullptr, *ls_cnt = nullptr, *ls_ovr = nullptr;
  int32_t *lss_in = nullptr, *lss_out = nullptr;
  float* lss_dphi = nullptr;   // (z0 is computed again, in float-float, for the dense LS)
  int32_t* ls_off = nullptr;
  int32_t *ls_in = nullptr, *ls_out = nullptr;
  float *ls_z0 = nullptr, *ls_dphi = nullptr;
  float2* ls_xy_out = nullptr;   // (x, y) of each dense LS's outer anchor (T3 candidate loop)
  int32_t* lsin_off = nullptr;   // LS grouped by inner MD
  // T3
  int32_t *t3_cap = nullptr, *t3_base = nullptr, *t3_cnt = nullptr, *t3_ovr = nullptr;
  int32_t *t3s_a = nullptr, *t3s_b = nullptr;
  float *t3s_R = nullptr, *t3s_xc = nullptr, *t3s_yc = nullptr, *t3s_chi2 = nullptr, *t3s_pte = nullptr;
  int32_t* t3_off = nullptr;
  int32_t *t3_a = nullptr, *t3_b = nullptr, *t3_md0 = nullptr, *t3_md1 = nullptr, *t3_md2 = nullptr;
  float *t3_R = nullptr, *t3_xc = nullptr, *t3_yc = nullptr, *t3_chi2 = nullptr, *t3_pte = nullptr;
  int32_t* t3md_off = nullptr;   // [md_dense + 2] T3 by first MD (their group offsets)
  float4* t3_anc = nullptr;      // [3][t3_dense] anchor (x, y, z, r) of each member MD
  float* t3_anc_rlo = nullptr;   // [3][t3_dense] low part of each anchor's radius (r + rlo to ~2^-47)
  uint8_t* t3_ecm = nullptr;     // endcap bit per anchor
  // T5
  int32_t *t5_cap = nullptr, *t5_base = nullptr, *t5_cnt = nullptr, *t5_ovr = nullptr;
  int32_t *t5s_a = nullptr, *t5s_b = nullptr;
  float* t5s_f = nullptr;   // [8][t5_slots]: kin, kout, kfit, chi2c, chi2rz, eta, phi, pt
  int32_t* t5_off = nullptr;
  int32_t *t5_a = nullptr, *t5_b = nullptr;
  int32_t* t5_md = nullptr;  // [5][t5_dense]
  float* t5_f = nullptr;     // [8][t5_dense]
  float4* t5_anc = nullptr;      // [5][t5_dense]
  float* t5_anc_rlo = nullptr;   // [5][t5_dense]
  uint8_t* t5_ecm = nullptr;
  // per module: lo[vm], hi[V + vm] = bounding box (x, y, z, r) of the first anchors of its T3 / T5
  float4* box3 = nullptr;
  float4* box5 = nullptr;
  // pixel seeds and pT3 / pT5: passing objects are appended, then grouped by seed
  int32_t* pls_bin = nullptr;
  int32_t* pls_ev = nullptr;     // [P] event of each seed
  float4* pls_seed = nullptr;    // [2][P] float32 seed helix: (x0, y0, z0, rho), (|kappa|, sin phi, cos phi, cot theta)
  float2* pls_seed_ff = nullptr; // [P][9] the same in double-float (x0, y0, z0, rho, |kappa|, sin, cos, cot, R)
  int32_t *p3a_pls = nullptr, *p3a_obj = nullptr;
  float *p3a_xy = nullptr, *p3a_rz = nullptr, *p3a_sc = nullptr;
  int32_t *p3_cnt = nullptr, *p3_cur = nullptr, *pt3_off = nullptr;   // [P], [P], [P + 1]
  int32_t *pt3_pls = nullptr, *pt3_obj = nullptr;
  float *pt3_xy = nullptr, *pt3_rz = nullptr, *pt3_sc = nullptr;
  int32_t *p5a_pls = nullptr, *p5a_obj = nullptr;
  float *p5a_xy = nullptr, *p5a_rz = nullptr, *p5a_sc = nullptr;
  int32_t *p5_cnt = nullptr, *p5_cur = nullptr, *pt5_off = nullptr;
  int32_t *pt5_pls = nullptr, *pt5_obj = nullptr;
  float *pt5_xy = nullptr, *pt5_rz = nullptr, *pt5_sc = nullptr;
  // track candidates
  int32_t *best5 = nullptr, *best3 = nullptr;   // [P]
  uint8_t *pls_member = nullptr, *acc3 = nullptr, *accl = nullptr;   // [P]
  uint8_t *t5_kept = nullptr, *acc5t = nullptr;  // [t5_dense]
  int32_t *h5_cnt = nullptr, *h5_off = nullptr, *h5_cur = nullptr, *h5_idx = nullptr;  // hit -> T5
  int32_t* t5_hit = nullptr;     // [t5_dense][10] hits of each T5 (lower, upper of each member MD)
  int32_t *cell_cnt = nullptr, *cell_off = nullptr, *cell_cur = nullptr, *cell_item = nullptr;
  int32_t n_cells = 0;   // per event
  int32_t* tc_cnt = nullptr;   // [E]
  int32_t* tc_code = nullptr;  // [tc_capacity] candidate codes (type << 29 | index), per-event regions
  int32_t* tc_perm = nullptr;  // [tc_capacity] source (collected index) of each ordered row
  int32_t* tc_n = nullptr;     // [4 E] candidates collected per (event, type)
  unsigned long long* tc_key = nullptr;   // [tc_capacity] sort keys
  int32_t* tc_hit_key = nullptr;          // [tc_capacity][14] sorted hit tuples
  int32_t* grp_tmp = nullptr;             // [max(p3_slots, p5_slots)] grouping scratch
  int32_t *tc_type = nullptr, *tc_obj = nullptr, *tc_hits = nullptr;   // per-event regions
  float *tc_pt = nullptr, *tc_eta = nullptr, *tc_phi = nullptr;
  int32_t* tcd_off = nullptr;   // [E + 1] first dense row of each event
  int32_t *tcd_type = nullptr, *tcd_obj = nullptr, *tcd_hits = nullptr;   // dense over the batch
  float *tcd_pt = nullptr, *tcd_eta = nullptr, *tcd_phi = nullptr;
  // track extensions of the dense rows: extending T3 (event-local, -1: none), MDs added, the added
  // hits ([4] per row, -1 padded), chi2 of the extended track's circle and r-z fits
  int32_t *tcd_ext_t3 = nullptr, *tcd_ext_n = nullptr, *tcd_ext_hits = nullptr;
  float *tcd_ext_c = nullptr, *tcd_ext_rz = nullptr;
  // their candidates: per row the count and up to kExtRefs references into the candidate queues
  // (one region of ext_qcap entries per anchor count 4..7: (row, T3 | overlap << 30) and the
  // result (score, chi2_c, chi2_rz, passed))
  int32_t* ext_cnt = nullptr;     // [tc_cap]
  int32_t* ext_ref = nullptr;     // [tc_cap][kExtRefs]: region << 28 | position
  int2* ext_q = nullptr;          // [4][ext_qcap]
  float4* ext_res = nullptr;      // [4][ext_qcap]
  int32_t* ext_qn = nullptr;      // [5] entries pushed per region, then the slow rows (zeroed every run)
  int32_t* ext_slow = nullptr;    // [tc_cap] rows with candidates beyond their references or the queues
  int64_t ext_qcap = 0;
  int64_t tc_capacity = 0;
  // event-local output copies
  int32_t *o_md_lo = nullptr, *o_md_up = nullptr, *o_md_mod = nullptr;
  int32_t *o_ls_in = nullptr, *o_ls_out = nullptr, *o_t3_a = nullptr, *o_t3_b = nullptr;
  int32_t *o_t5_a = nullptr, *o_t5_b = nullptr, *o_pt3_pls = nullptr, *o_pt3_obj = nullptr;
  int32_t *o_pt5_pls = nullptr, *o_pt5_obj = nullptr;
  // float64 decision queues
  int4 *q_md = nullptr, *q_ls = nullptr;
  int2 *q_t3 = nullptr, *q_t5 = nullptr, *q_p3 = nullptr, *q_p5 = nullptr;
  // scan scratch and status
  int32_t* scan_tmp = nullptr;
  int32_t* eff = nullptr;    // [V + 1] weights (valid slots + 1) per module of the stage being compacted, then their scan
  int32_t* grp_key = nullptr;       // [max(H, t3_dense) + 2] per-key counts / group starts (compaction)
  int32_t* grp_pos = nullptr;       // [max dense] objects placed by group (compaction)
  int2* grp_key12 = nullptr;        // [max dense] their (first, second) members
  unsigned long long* scan_state = nullptr;   // single-pass scan tile states (zeroed at allocation)
  int32_t* scan_ctr = nullptr;      // [kScanMax] their tile tickets (zeroed every run)
  int32_t* scan_run = nullptr;      // chain runs so far (zeroed at allocation; advanced by k_bin_count)
  int64_t scan_state_n = 0;         // entries of scan_state
  int32_t* grp_task = nullptr;      // [(max slots + V) / 64 + 2] first module of each compaction task
  unsigned long long* t3_bound = nullptr;   // [V] T3 candidates per module (summed over its dense LS)
  unsigned long long* t5_bound = nullptr;   // [V] T5 candidates per module (summed over its dense T3)
  int32_t* perm = nullptr;   // [max dense] slot of each dense object of the stage being compacted
  int32_t* status = nullptr;   // [ST_N_WORDS]
  int32_t* ev_stat = nullptr;  // [E][kEvWords]
  // persistent LS kernel: modules ordered by descending predicted cost (log2 buckets)
  int32_t* work = nullptr;        // [kLsMaxChunks V] work items: module
  int32_t* work_c = nullptr;      // [kLsMaxChunks V] work items: chunk of the module's outer MDs
  int32_t* work_bucket = nullptr; // [V] cost bucket of each module's chunks (-1: no candidates)
  int32_t* work_nch = nullptr;    // [V] chunks of each module
  int ls_chunk = 1 << 30;         // outer MDs per chunk of a module's LS work (small batches split)
  int32_t* work_cnt = nullptr;    // [32] items per bucket
  int32_t* work_cur = nullptr;    // [32]
  int32_t* work_off = nullptr;    // [33]
  int32_t* ls_head = nullptr;     // device-queue head of the LS work list (persistent = 2; zeroed every run)
};

// Launch settings (from lst_config).
struct Launch {
  cudaStream_t stream = nullptr;
  int block_ls = 128;
  int warps_px = 4;
  int persistent = 0;   // 0 grid-stride, 1 static cost-ordered deal, 2 device queue
  int n_sm = 152;
  int ls_blocks_per_sm = 0;        // resident blocks of the Line-Segment kernel (0: not queried)
  int t3_blocks_per_sm = 0;        // resident blocks of the T3 / T5 candidate kernels (0: not queried)
  int t5_blocks_per_sm = 0;
  int pt3_blocks_per_sm = 0;       // resident blocks of the pT3 / pT5 pre-filters at warps_px warps
  int pt5_blocks_per_sm = 0;       //   per block (0: not queried)
  long long* launches = nullptr;   // host counter
  bool capturing = false;          // the chain is being captured into a CUDA graph
  cudaEvent_t* kev = nullptr;      // when set: [2 * kernel id] start / end events of timed kernels
  // single-pass scans of the chain (nullptr: three-pass scans). Tile states are tagged with an
  // epoch = run * kScanMax + scan index, where the run counter is advanced on the device once per
  // chain run, so that no state needs clearing between scans or runs.
  unsigned long long* scan_state = nullptr;   // [tiles of the largest scan], zeroed once
  int32_t* scan_ctr = nullptr;                // [kScanMax] tile tickets, zeroed every run
  const int32_t* scan_run = nullptr;          // device run counter
  int32_t* scan_err = nullptr;                // incremented when a look-back gives up
  int* scan_idx = nullptr;                    // host: next scan index of the chain being enqueued
};
constexpr int kScanMax = 64;   // single-pass scans per chain run at most
constexpr int kLsMaxChunks = 8;   // LS work items per module at most

// kernels timed individually when timing is enabled (index order of lst_get_kernel_ms)
enum KernelId : int {
  K_BIN = 0, K_MD, K_MD_COMPACT, K_LS, K_LS_COMPACT, K_T3_PRE, K_T3_DECIDE, K_T3_COMPACT, K_T5_PRE,
  K_T5_DECIDE, K_PT3_PRE, K_PT5_PRE, K_PT3_DECIDE, K_PT5_DECIDE, K_TC_CLEAN, K_TC_ASSEMBLE, K_TC_EXT, K_N_TIMED
};
// (recorded as external events while the chain is captured, so that inside the CUDA graph they
// become event-record nodes that can be timed; plain records otherwise, where the external flag is
// not allowed)
#define KT_REC(L, ev) \
  cudaEventRecordWithFlags((ev), (L).stream, (L).capturing ? cudaEventRecordExternal : cudaEventRecordDefault)
#define KT_BEGIN(L, id) \
  if ((L).kev) KT_REC(L, (L).kev[2 * (id)])
#define KT_END(L, id) \
  if ((L).kev) KT_REC(L, (L).kev[2 * (id) + 1])

// resident blocks per SM of the Line-Segment kernel at `block` threads (0 when the query fails)
int ls_resident_blocks(int block, int targets);
// resident blocks per SM of the T3 and T5 candidate kernels (their grids hold exactly these, so that
// their statically divided work runs in one wave); 0 when the query fails
int t3_pre_resident_blocks();
int t5_pre_resident_blocks();
// the same for the pT3 (n = 3) and pT5 (n = 5) pre-filters with `warps` warps per block
int pt_pre_resident_blocks(int n, int warps);

// scan: out[0..n] exclusive prefix sums of in[0..n-1] (out[n] = total); in and out may alias
void scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, const Launch& L);
// In-place single-pass scan of n positive weights that also writes the compaction task starts:
// first[t] = the first k whose prefix is >= t * chunk, for t up to ceil(total / chunk) (that one = n).
// Only inside a chain run (single-pass scans); returns false when it cannot run (the caller then
// scans and searches separately).
bool scan_tasks(int32_t* data, int64_t n, int32_t* first, int chunk, const Launch& L);
// The single-pass scan with its first tile withheld (see lst_selftest_bounded_wait); 0 or -1.
int scan_wait_selftest(int device, int32_t* gave_up);
// the same with the entry count min(n, *n_dev + n_add) read on the device (n sizes the launch);
// out[count] receives the total
void scan_exclusive_dev(const int32_t* in, int32_t* out, int64_t n, const int32_t* n_dev, int n_add, int32_t* tmp,
                        const Launch& L);
int64_t scan_tmp_elems(int64_t n);

// compaction of one stage's slots into ordered dense arrays (lst_group.cu)
struct GroupArgs {
  const int32_t *cnt, *cap, *base;   // per-module counts, capacities, slot bases (base[V] = total)
  int64_t slots;
  int ovf_word, arena_word;
  const int32_t *key1, *key2;        // first / second member of each slot
  const int32_t* key_map;            // group key of a first member k1: key_map[k1] (monotone), or k1 if nullptr
  int32_t* grp_off;                  // out: [n_keys + 1] objects whose group key is below each key
                                     // (nullptr: not needed by a later stage; scratch is used)
  int64_t n_keys;                    // group key range (capacity)
  const int32_t* n_keys_dev;         // device: the actual number of keys (<= n_keys); grp_off is
                                     // defined on [0, *n_keys_dev]. The group sizes are counted by the
                                     // producing kernels into grp_off (or grp_key) at [group + 1].
  int64_t dense_cap;
  int dense_word;
  int32_t* mod_off;                  // [V + 1] out: per-module dense offsets
  const int32_t* mod_first;          // first key of each module, at [vm * stride]
  int mod_first_stride;
  int dense_out = -1;                // what the rank pass writes (kDensePerm / kDenseLs / kDenseT3)
};
// kDensePerm: the permutation (perm[dense position] = slot; the stage's own kernel gathers the
// dense arrays); kDenseLs / kDenseT3: the dense LS / T3 arrays themselves (ls_dense_write,
// t3_dense_write)
enum { kDensePerm = 0, kDenseLs = 1, kDenseT3 = 2 };
void group_slots(const Ws& w, const GroupArgs& a, const Launch& L);


// message returned by lst_last_error(NULL) (calls that have no context)
void set_global_error(const char* msg);

// single-event hit binning on plain device arrays; cnt, cur (n_sens each) and err must be zero
void run_bin_raw(const int32_t* sensor, int n, int n_sens, int32_t* order, int32_t* offsets, int32_t* cnt,
                 int32_t* cur, int32_t* err, int32_t* scan_tmp, const Launch& L);

// stages
void run_binning(const Ws& w, const Geo& g, const Launch& L);
void run_md(const Ws& w, const Geo& g, const Consts& c, const Launch& L);
void run_ls(const Ws& w, const Geo& g, const Consts& c, const Launch& L);
void run_t3(const Ws& w, const Geo& g, const Consts& c, const Launch& L);
void run_t5(const Ws& w, const Geo& g, const Consts& c, const Launch& L);
void run_pixel(const Ws& w, const Geo& g, const Consts& c, const Launch& L);
void run_tc(const Ws& w, const Geo& g, const Consts& c, const Launch& L);
void run_finalize(const Ws& w, const Geo& g, const Launch& L);
int tc_cells_per_event();
void tc_configure();
// after an overflowing run: raise the per-module capacity overrides to the observed counts
void run_raise_overrides(const Ws& w, const Launch& L);

// Cycle budget of the candidate kernels (lst_config.cycle_budget, 0 = none): checked by whole warps at
// the head of each work item; a warp past its budget counts itself in ST_TIMEOUT and stops taking
// work, so a pathological batch ends with LST_ETIMEOUT instead of occupying the GPU.
__device__ __forceinline__ bool warp_over_budget(const Ws& w, long long t0) {
  const bool over = w.cycle_budget > 0 && clock64() - t0 > w.cycle_budget;
  if (__any_sync(0xffffffffu, over)) {
    if ((threadIdx.x & 31) == 0) atomicAdd(&w.status[ST_TIMEOUT], 1);
    return true;
  }
  return false;
}

// counters[key] += v over the lanes of a warp (all lanes call it; inactive lanes pass v = 0):
// lanes with the same key are summed first, one atomic per distinct key
__device__ __forceinline__ void warp_add_keyed(unsigned long long* counters, int key, unsigned v) {
  const unsigned grp = __match_any_sync(0xffffffffu, key);
  const unsigned sum = __reduce_add_sync(grp, v);
  if ((threadIdx.x & 31) == __ffs(grp) - 1 && sum) atomicAdd(&counters[key], (unsigned long long)sum);
}

// Group counts of a compaction: the producing kernels count each stored object at E[group + 1] of an
// array zeroed on [0, n] before them (by the stage's capacity kernel; all threads of its grid call
// this).
__device__ __forceinline__ void zero_group_counts(int32_t* E, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) E[k] = 0;
}

// After a dense overflow of the previous stage its group offsets E[0..n] are clamped to the dense
// capacity before the next stage reads them (done by the next stage's capacity kernel; all threads
// of its grid call this)
__device__ __forceinline__ void clamp_group_offsets(int32_t* E, int n, int64_t cap, bool overflowed) {
  if (!overflowed) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x)
    if (E[k] > cap) E[k] = (int)cap;
}

// E[key] += 1 for every lane with pred, one atomic per distinct key of the warp (all lanes call it)
__device__ __forceinline__ void warp_count_keyed(bool pred, int key, int32_t* E) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (pred) {
    const unsigned grp = __match_any_sync(m, key);
    if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&E[key], __popc(grp));
  }
}

// The dense LS at position d (ordered by (inner MD a, outer MD b)) from slot s: members (global and
// event-local), z0, dphi, the outer anchor cache, and each LS's count of outer partners (the T3 candidates it starts, from
// the LS-by-inner-MD offsets lsin_off) summed per module for the T3 capacities. All lanes of the
// warp call it; n is the number of dense LS.
__device__ __forceinline__ void ls_dense_write(const Ws& w, bool valid, int d, int s, int a, int b,
                                               const int32_t* lsin_off, int n) {
  int vm = 0;
  unsigned outs = 0;
  if (valid) {
    w.ls_in[d] = a;
    w.ls_out[d] = b;
    // z0 = (z1 r2 - z2 r1) / (r2 - r1) with the radii in float-float: the float32 rounding of the
    // radii would be amplified up to ~20x for endcap pairs
    const float4 pa = w.md_xyzr[a], pb = w.md_xyzr[b];
    const float r1l = w.md_rlo[a], r2l = w.md_rlo[b];
    const float num = diff_prod(pa.z, pb.w, pb.z, pa.w) + (pa.z * r2l - pb.z * r1l);
    const float den = (pb.w - pa.w) + (r2l - r1l);
    store_out(w.ls_z0, w.ls_z0_h, d, num / den);
    store_out(w.ls_dphi, w.ls_dphi_h, d, w.lss_dphi[s]);
    w.ls_xy_out[d] = make_float2(pb.x, pb.y);
    vm = w.md_vm[a];
    outs = (unsigned)(min(lsin_off[b + 1], n) - min(lsin_off[b], n));
    // event-local member indices (the MDs of the event start at the first MD of its first module)
    const int n_mods = w.V / w.E;
    const int first_md = w.md_off[vm - vm % n_mods];
    w.o_ls_in[d] = a - first_md;
    w.o_ls_out[d] = b - first_md;
  }
  warp_add_keyed(w.t3_bound, vm, outs);
}

// The dense T3 at position d (ordered by first MD, then (inner LS a, outer LS b)) from slot s:
// members (global and event-local), member MDs, fit values, an anchor cache for the pT3 stage, and
// each T3's count of outer partners (the T5 candidates it starts, from the T3-by-first-MD offsets
// t3md_off) summed per module for the T5 capacities. All lanes of the warp call it; n is the number
// of dense T3.
__device__ __forceinline__ void t3_dense_write(const Ws& w, bool valid, int d, int s, int a, int b,
                                               const int32_t* t3md_off, int n) {
  int vm = 0;
  unsigned outs = 0;
  if (valid) {
    const int64_t T = w.cap.t3_dense;
    w.t3_a[d] = a;
    w.t3_b[d] = b;
    const int md[3] = {w.ls_in[a], w.ls_out[a], w.ls_out[b]};
    w.t3_md0[d] = md[0];
    w.t3_md1[d] = md[1];
    w.t3_md2[d] = md[2];
    w.t3_R[d] = w.t3s_R[s];
    store_out(w.t3_xc, w.t3_xc_h, d, w.t3s_xc[s]);
    store_out(w.t3_yc, w.t3_yc_h, d, w.t3s_yc[s]);
    store_out(w.t3_chi2, w.t3_chi2_h, d, w.t3s_chi2[s]);
    store_out(w.t3_pte, w.t3_pte_h, d, w.t3s_pte[s]);
    uint8_t ecm = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      w.t3_anc[k * T + d] = w.md_xyzr[md[k]];
      w.t3_anc_rlo[k * T + d] = w.md_rlo[md[k]];
      ecm |= (uint8_t)(w.md_ec[md[k]] << k);
    }
    w.t3_ecm[d] = ecm;
    vm = w.md_vm[md[0]];
    outs = (unsigned)(min(t3md_off[md[2] + 1], n) - min(t3md_off[md[2]], n));
    // event-local member indices (the LS of the event start at the first LS of its first module)
    const int n_mods = w.V / w.E;
    const int first_ls = w.ls_off[vm - vm % n_mods];
    w.o_t3_a[d] = a - first_ls;
    w.o_t3_b[d] = b - first_ls;
  }
  warp_add_keyed(w.t5_bound, vm, outs);
}

inline int grid_for(int64_t n, int block, int max_blocks = 152 * 32) {
  int64_t b = (n + block - 1) / block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

#define LST_LAUNCH(L) (++*(L).launches)

}  // namespace lst
