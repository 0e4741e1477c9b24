/*
 * lst.h - C ABI of the GB300 (sm_103a) Line Segment Tracking library, liblst.so.
 *
 * Line Segment Tracking (arXiv:2207.08207) builds tracks bottom-up in the CMS outer tracker:
 *   hits, binned by detector module                      (Sec. 4.2, "pre-processing the hits")
 *   -> Mini-Doublets (MD): hit pairs in a module's two sensors            (Sec. 2.2)
 *   -> Line Segments (LS): MD pairs in modules linked by the module map   (Sec. 2.2)
 *   -> Triplets (T3): two LS sharing an MD; Quintuplets (T5): two T3 sharing an MD  (Sec. 2.3)
 *   -> pixel seeds (pLS) linked to T3 / T5 as pT3 / pT5                  (Sec. 2.4)
 *   -> Track Candidates (TC): pT5, pT3, T5, pLS in that order, cross-cleaned in eta-phi (Sec. 2.5)
 * The paper's statement of the problem (Fig. "GPU implementation flowchart", Sec. 4.2) is: hits and
 * pixel tracks in, MD/LS/T3/T5/pT3/pT5/TC objects out, track candidates copied to the CPU. The
 * calls below follow it.
 *
 * Conventions
 *  - Every function returns an lst_status (0 = LST_OK). No exception crosses this boundary and
 *    nothing aborts the process; lst_last_error() gives a one-line reason for the last failure.
 *  - Pointers are plain host or device pointers; sizes are element counts unless stated.
 *  - A context (lst_ctx) owns its device memory (object arenas, allocated from a per-context CUDA
 *    memory pool) and is used by one host thread at a time. Several contexts may share a device.
 *  - Units: cm, GeV, Tesla; the solenoid field is along +z.
 */
#ifndef LST_H_
#define LST_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LST_OK = 0,
  LST_EINVAL = 1,                 /* bad argument or input (ids out of range, NaN coordinates) */
  LST_ENOMEM = 2,                 /* device or pinned-host allocation failed */
  LST_ECUDA = 3,                  /* a CUDA runtime call failed (see lst_last_error) */
  LST_ETIMEOUT = 4,               /* a kernel exceeded its cycle budget and stopped early */
  LST_EOVERFLOW_UNRESOLVED = 5,   /* object capacity still exceeded after the retry limit */
  LST_ESTATE = 6                  /* call out of order (e.g. no geometry loaded) */
} lst_status;

/* Where an event's input arrays live. LST_MEM_HOST: host memory, copied before lst_run_events
 * returns. LST_MEM_DEVICE: device memory of the context's device. LST_MEM_HOST_ASYNC: host memory
 * that the caller keeps unchanged until lst_sync returns; where the GPU can read it in place (pinned
 * memory, or pageable memory on a coherent host link such as NVLink-C2C) the device gathers it
 * directly inside the run, else it is copied like LST_MEM_HOST. */
enum { LST_MEM_HOST = 0, LST_MEM_DEVICE = 1, LST_MEM_HOST_ASYNC = 2 };

/* Stage indices used by the per-stage arrays of lst_counts. */
enum {
  LST_STAGE_MD = 0, LST_STAGE_LS = 1, LST_STAGE_T3 = 2, LST_STAGE_T5 = 3,
  LST_STAGE_PT3 = 4, LST_STAGE_PT5 = 5, LST_STAGE_TC = 6, LST_STAGE_QUEUE = 7, LST_N_STAGES = 8
};

/* Track-candidate types, in the order the paper adds them to the collection (Sec. 2.5). */
enum { LST_TC_PT5 = 0, LST_TC_PT3 = 1, LST_TC_T5 = 2, LST_TC_PLS = 3 };

/*
 * Selection constants and execution settings. The paper prints no cut value except the pT
 * threshold (0.8 GeV, Sec. 2.2); every other constant is this library's reading, fixed here once.
 * lst_config_default() fills the values below. The float fields are the cut constants; the
 * integer fields control execution only and never change which objects are built.
 */
typedef struct {
  float k;             /* pT = k * R [GeV/cm]; 0.003 * 3.8 T = 0.0114 */
  float pt_thr;        /* pT threshold (Sec. 2.2), 0.8 */
  float sin_max;       /* cap on sin(alpha_thr), 0.95 */
  float z_lum;         /* luminous-region half length, 15 cm */
  float d0_max;        /* impact-parameter allowance of MD/LS windows, 0.1 cm */
  float n_sigma;       /* window width in resolutions, 3 */
  float sigma_rphi;    /* hit resolution in r-phi, 0.003 cm */
  float sigma_z;       /* barrel hit resolution in z, 0.1 cm */
  float sigma_r;       /* endcap hit resolution in r, 0.1 cm */
  float chi2_t3;       /* T3 r-z chi2 cut, 9 */
  float chi2_t5_c;     /* T5 global circle-fit chi2 cut, 20 */
  float chi2_t5_rz;    /* T5 r-z chi2 cut, 16 */
  float chi2_pt3_xy, chi2_pt3_rz;   /* pT3 cuts, 16 / 16 */
  float chi2_pt5_xy, chi2_pt5_rz;   /* pT5 cuts, 25 / 25 */
  float f_t3;          /* T3 pT estimate >= f_t3 * pt_thr, 0.8 */
  float d0_t3;         /* T3 circle impact parameter, 2 cm */
  float c_rel, c_abs;  /* T5 curvature compatibility, 0.2 and 1.5e-4 / cm */
  float dr_min;        /* eta-phi cross-cleaning distance, 0.01 */
  float pt_cap;        /* cap on pT estimates, 1e4 GeV */
  float pls_dir_err;   /* pixel-seed direction uncertainty, 1e-3 rad */
  float pls_pt_err;    /* pixel-seed relative pT uncertainty, 0.01 */
  float sigma_floor;   /* floor on r-z per-anchor uncertainties, 1e-4 cm */
  int32_t t5_overlap_hits;  /* T5 duplicate removal: >= this many of 10 hits shared, 7 */

  /* execution settings (chosen by the autotuner; defaults are safe) */
  int32_t persistent;       /* LS kernel over a cost-ordered list of (event, module) work items, heavy
                               modules split in small batches: 2 (default) persistent warps take the
                               items from a device queue (one atomic head); 1 persistent warps with a
                               static boustrophedon deal of the list; 0: grid-stride over modules */
  int32_t use_graph;        /* 1: capture the MD->TC chain in a CUDA graph and replay it */
  int32_t block_ls;         /* threads per LS block (64, 128, 256) */
  int32_t warps_px;         /* warps per block in the pT3/pT5 candidate kernels (1..8; else 4) */
  float cap_scale;          /* multiplier on predicted per-module capacities (>= 0.25) */
  int32_t max_retries;      /* capacity-overflow retries before LST_EOVERFLOW_UNRESOLVED */
  int64_t cycle_budget;     /* per-warp clock64 budget of the candidate kernels (MD, LS, T3, pT3/pT5 loops);
                               0 = none. A warp past it stops taking work and the run ends with
                               LST_ETIMEOUT (results incomplete; the context stays usable) */
  int32_t half_floats;      /* 1: store the output-only per-object floats as IEEE binary16 (round to
                               nearest) instead of float32, halving their device memory and copy-out
                               bytes (the "half precision" storage of Sec. 5): MD dPhiChange and pT
                               estimate, LS z0 and dphi, T3 centre, r-z chi2 and pT estimate, T5
                               kappa_in, kappa_out and r-z chi2, pT3 / pT5 chi2_xy and chi2_rz. No
                               selection reads these values, so every object and every other output
                               is the same; their float32 pointers in lst_event_out are then NULL and
                               the *_h pointers hold them. binary16 spans +-65504: larger magnitudes
                               (the centre of a nearly straight T3's circle, a huge chi2) are stored as
                               +-inf, as the round-to-nearest conversion gives. Default 0. */
} lst_config;

/* One detector module (a pair of closely spaced sensors, "bi-layer pT module", Sec. 1). */
typedef struct {
  int32_t id;        /* must equal its index */
  int32_t subdet;    /* 0 barrel, 1 endcap */
  int32_t layer;     /* barrel layer 1..6 or endcap disk 1..5 */
  int32_t side;      /* 0 barrel, -1 / +1 endcap side */
  int32_t type;      /* 0 PS, 1 2S */
  float surf;        /* radius (barrel) or |z| (endcap) of the lower sensor */
  float spacing;     /* sensor separation */
  float phi_lo, phi_hi, w_lo, w_hi;   /* patch bounds: phi and z (barrel) or r (endcap) */
} lst_module;

/* A pixel seed, used as a line segment (pLS, Sec. 2.4). The helix is given at (x0, y0, z0) with
 * direction phi, pseudorapidity eta and charge; pix_hit are the seed's 4 hit ids (any int32 ids
 * that do not collide with the event's outer-tracker hit indices). */
typedef struct {
  float pt, eta, phi, x0, y0, z0;
  int32_t charge;
  int32_t pix_hit[4];
  int32_t pad;
} lst_pls;

/* One event. sensor[i] = 2 * module + (0 lower sensor | 1 upper sensor). LST_MEM_HOST and
 * LST_MEM_DEVICE inputs are read during lst_run_events (copied into the context) and may be released
 * when it returns; LST_MEM_HOST_ASYNC inputs must stay valid until lst_sync returns. */
typedef struct {
  const float* x;
  const float* y;
  const float* z;
  const int32_t* sensor;
  int32_t n_hits;
  const lst_pls* pls;
  int32_t n_pls;
  int32_t mem_space;   /* LST_MEM_HOST, LST_MEM_DEVICE or LST_MEM_HOST_ASYNC, for all five arrays */
} lst_event_in;

/* Per-event object counts and status. overflow[s] counts, for the whole batch the event was part
 * of, the objects that did not fit stage s's capacities on the first pass (per-module capacity or
 * the stage's slot arena; overflow[LST_STAGE_QUEUE]: entries beyond an exact-decision queue); they
 * were recovered by a retry (retries > 0) unless status is LST_EOVERFLOW_UNRESOLVED.
 * recheck[s] (batch totals) counts candidates decided in the exact path (float64 for MD and LS,
 * double-float for T3 / T5 / pT3 / pT5): for MD and LS those whose float32 cut margins were too
 * close to a threshold, for the others every candidate that survived the float32 pre-filter. */
typedef struct {
  int32_t n_hits, n_pls;
  int32_t n_md, n_ls, n_t3, n_t5, n_pt3, n_pt5, n_tc;
  int32_t n_tc_type[4];
  int32_t overflow[LST_N_STAGES];
  int32_t recheck[LST_N_STAGES];
  int32_t retries;
  int32_t status;
  int32_t n_tc_ext;   /* track candidates that were extended (Sec. 2.5.1) */
  int64_t n_ls_pairs; /* batch total: (inner MD, outer MD) candidate pairs the LS search evaluated
                         (those inside its azimuth windows; Sec. 2.2), a measure of its work */
} lst_counts;

/*
 * Device pointers to one event's objects, inside the context's arenas. Valid until the next
 * lst_run_events on the same context. Objects of each type are dense and ordered: MD by
 * (module, lower hit, upper hit) where a module's hits are taken in order of azimuth about the module
 * centre (ties by input index), LS by (inner MD, outer MD), T3 by (inner LS, outer LS), T5 by
 * (inner T3, outer T3), pT3 / pT5 by (seed, object), TC by (type, sorted hit tuple).
 * Member indices (ls_md_in, t3_ls_in, ...) are event-local indices into the same event's arrays.
 * Hit indices are the event's input hit indices.
 */
typedef struct {
  lst_counts counts;
  const int32_t *md_hit_lo, *md_hit_up, *md_module;
  const float *md_dphichange, *md_pt_est;
  const int32_t *ls_md_in, *ls_md_out;
  const float *ls_z0, *ls_dphi;
  const int32_t *t3_ls_in, *t3_ls_out;
  const float *t3_r, *t3_xc, *t3_yc, *t3_chi2_rz, *t3_pt_est;
  const int32_t *t5_t3_in, *t5_t3_out;
  const float *t5_kappa_in, *t5_kappa_out, *t5_kappa_fit, *t5_chi2_c, *t5_chi2_rz, *t5_eta,
      *t5_phi, *t5_pt;
  const int32_t *pt3_pls, *pt3_t3;
  const float *pt3_chi2_xy, *pt3_chi2_rz;
  const int32_t *pt5_pls, *pt5_t5;
  const float *pt5_chi2_xy, *pt5_chi2_rz;
  const int32_t *tc_type, *tc_obj, *tc_hits;   /* tc_hits: [n_tc][14], -1 padded */
  const float *tc_pt, *tc_eta, *tc_phi;
  /* Track extensions (Sec. 2.5.1), one per TC row: the T3 that continues the candidate outward
   * (event-local T3 index, -1 when the candidate is not extended), the MDs it adds (1 or 2; 0 when
   * none), their hits ([n_tc][4], lower and upper hit of each added MD inner to outer, -1 padded),
   * and the chi2 of the extended track's circle and r-z line fits. A pT5, pT3 or T5 candidate with
   * MDs m_1..m_K is extended by a T3 that starts at m_K (adding two MDs) or at m_(K-1) with its
   * second MD m_K (adding one), whose curvature agrees with the candidate's (|k_T3 - k_TC| <=
   * c_rel max + c_abs; k_TC from the seed's pT or the T5 fit), and for which the n-anchor extended
   * track passes the r-z line fit with chi2 <= chi2_t5_rz (n - 2) / 3 (the T5 cut per degree of
   * freedom); of several, the lowest (circle chi2 + r-z chi2, sorted hit tuple of the T3), the circle
   * chi2 being that of Karimaki's fit of the n anchors (reported, not cut on). pLS candidates are
   * not extended. */
  const int32_t *tc_ext_t3, *tc_ext_n_md, *tc_ext_hits;
  const float *tc_ext_chi2_c, *tc_ext_chi2_rz;
  /* With lst_config.half_floats = 1: the output-only columns as IEEE binary16 bit patterns (the
   * float32 pointers of the same columns are then NULL); NULL otherwise. */
  const uint16_t *md_dphichange_h, *md_pt_est_h, *ls_z0_h, *ls_dphi_h;
  const uint16_t *t3_xc_h, *t3_yc_h, *t3_chi2_rz_h, *t3_pt_est_h;
  const uint16_t *t5_kappa_in_h, *t5_kappa_out_h, *t5_chi2_rz_h;
  const uint16_t *pt3_chi2_xy_h, *pt3_chi2_rz_h, *pt5_chi2_xy_h, *pt5_chi2_rz_h;
} lst_event_out;

typedef struct lst_ctx lst_ctx;

/* Fill cfg with the default constants and execution settings. Host only; needs no GPU. */
void lst_config_default(lst_config* cfg);

/* Create a context on CUDA device `device` (ownership of *out passes to the caller, release with
 * lst_destroy). cfg may be NULL for defaults; it is copied. */
int lst_create(lst_ctx** out, const lst_config* cfg, int device);

/* Release every device and host resource of the context. Waits for its pending work first, so it
 * is safe to call while a run is in flight. NULL is ignored. */
void lst_destroy(lst_ctx* ctx);

/*
 * Load the detector geometry (host arrays, copied once into resident device tables).
 *  mods[n_mods]: module table, mods[i].id == i.
 *  conn_off[n_mods + 1], conn_tgt[conn_off[n_mods]]: the module map as CSR - the modules of the
 *    next layer reachable from each module by helices above the pT threshold (Sec. 2.2).
 *  pix_off[n_pix_bins + 1], pix_tgt[...]: pixel-seed map as CSR over (eta, phi, charge) bins:
 *    bin = ((floor(20 eta + 50)) * 128 + floor(phi_[0,2pi) * 64 / pi)) * 2 + (charge > 0); the
 *    targets are modules where a seed's T3 / T5 may start. n_pix_bins may be 0 (no seeds used).
 * Returns LST_EINVAL on inconsistent tables (ids, offsets not monotone, targets out of range).
 */
int lst_load_geometry(lst_ctx* ctx, const lst_module* mods, int32_t n_mods, const int32_t* conn_off,
                      const int32_t* conn_tgt, const int32_t* pix_off, const int32_t* pix_tgt,
                      int32_t n_pix_bins);

/*
 * The checks lst_load_geometry applies to its tables, on the host alone (no context, no GPU):
 * module ids equal their index, subdet is 0 or 1, spacing > 0; conn_off starts at 0 and never
 * decreases, no module has more than 256 connections, every conn_tgt is a module; the pixel map,
 * when n_pix_bins > 0, has exactly 100 x 128 x 2 bins, pix_off starts at 0 and never decreases, and
 * every pix_tgt is a module. Returns LST_OK (and the largest module-map degree in *max_degree, which
 * may be NULL) or LST_EINVAL with the reason in lst_last_error(NULL).
 */
int lst_check_geometry(const lst_module* mods, int32_t n_mods, const int32_t* conn_off, const int32_t* conn_tgt,
                       const int32_t* pix_off, const int32_t* pix_tgt, int32_t n_pix_bins, int32_t* max_degree);

/*
 * Reserve arenas for batches of up to n_events events of up to max_hits hits and max_pls seeds
 * each (optional: lst_run_events grows the arenas on demand).
 */
int lst_reserve(lst_ctx* ctx, int32_t n_events, int32_t max_hits, int32_t max_pls);

/*
 * Enqueue the whole chain for n_ev events on `cuda_stream` (a cudaStream_t; NULL means the
 * context's own stream) and return without waiting. out[n_ev] (host array, may be NULL) receives
 * the per-event device pointers once lst_sync returns. Events are independent: the objects of one
 * event never depend on another event in the batch.
 */
int lst_run_events(lst_ctx* ctx, const lst_event_in* ev, int32_t n_ev, lst_event_out* out,
                   void* cuda_stream);

/*
 * Wait for the last lst_run_events. Re-runs the batch with enlarged capacities if any stage
 * overflowed (at most cfg.max_retries times). status_per_event[n_ev] (may be NULL) receives each
 * event's lst_status. Returns the first non-OK event status, or a context-level error.
 */
int lst_sync(lst_ctx* ctx, int32_t* status_per_event);

/*
 * Bin one event's hits by sensor on the device (the hit pre-processing of Sec. 4.2): a counting sort
 * that is stable in the input order.
 *  d_sensor[n_hits] (device, in): sensor ids, 0 <= id < 2 * n_mods of the loaded geometry.
 *  d_order[n_hits] (device, out): input index of the hit at each binned position; the hits of one
 *    sensor are contiguous and in input order.
 *  d_offsets[2 * n_mods + 1] (device, out): first binned position of each sensor; the last entry is
 *    n_hits.
 * Scratch memory comes from the context. Runs on cuda_stream (NULL: the context's stream) and
 * waits for it before returning, because it reports an out-of-range sensor id as LST_EINVAL (the
 * outputs are then unspecified).
 */
int lst_bin_hits(lst_ctx* ctx, const int32_t* d_sensor, int32_t n_hits, int32_t* d_order,
                 int32_t* d_offsets, void* cuda_stream);

/*
 * The same binning as lst_bin_hits, for callers that may not allocate device memory at all: for
 * example a trigger process whose device memory is fixed when it starts, or a plugin inside a
 * framework that owns every device allocation. It needs no context. Its scratch is a fixed array in
 * the library's device memory (about 0.5 MB, present on every GPU that loads the library until the
 * process exits), so it handles at most 65536 sensors and returns LST_EINVAL for more.
 * The paper has no counterpart of this call; it exists for such embedding constraints only.
 *  d_sensor[n_hits] (device, in), d_order[n_hits] and d_offsets[n_sensors + 1] (device, out): as in
 *    lst_bin_hits, with the sensor count given explicitly.
 * Each call looks up the scratch array's address on the current device (the lookup allocates
 * nothing and is not cached, so it stays right after the device's context is reset). Every call on
 * a device shares the one scratch array, so calls whose work overlaps on the GPU (several streams,
 * or several host threads) race and must be serialized by the caller. The call waits for
 * cuda_stream (NULL: the legacy default stream) before returning, because it reads the error word
 * back to the host. Errors: LST_EINVAL for bad sizes or an out-of-range sensor id, LST_ECUDA for a
 * CUDA failure; lst_last_error(NULL) says which.
 */
int lst_bin_hits_noalloc(const int32_t* d_sensor, int32_t n_hits, int32_t n_sensors, int32_t* d_order,
                         int32_t* d_offsets, void* cuda_stream);

/* Non-blocking: 1 if the last run (including retries it needs) has finished, 0 otherwise, <0 on
 * error. A run that needs a retry is finished only after lst_sync. */
int lst_query(lst_ctx* ctx);

/* Counts of event `ev` of the last completed run (host copy). */
int lst_get_counts(const lst_ctx* ctx, int32_t ev, lst_counts* c);

/*
 * Copy event `ev`'s track candidates to host memory: type[n], obj[n], hits[n * 14], pt/eta/phi[n]
 * with n = counts.n_tc (any pointer may be NULL to skip that array).
 */
int lst_copy_tc(lst_ctx* ctx, int32_t ev, int32_t* type, int32_t* obj, int32_t* hits, float* pt,
                float* eta, float* phi);

/*
 * Copy event `ev`'s track extensions to host memory, one per TC row (see lst_event_out): t3[n],
 * n_md[n], hits[n * 4], chi2_c[n], chi2_rz[n] with n = counts.n_tc (any pointer may be NULL).
 */
int lst_copy_tc_ext(lst_ctx* ctx, int32_t ev, int32_t* t3, int32_t* n_md, int32_t* hits, float* chi2_c,
                    float* chi2_rz);

/*
 * Copy the track candidates of every event of the last completed run to host memory with one
 * transfer per array (the "copy track candidates to the CPU" step of Sec. 4.2). Event e's rows are
 * [offsets[e], offsets[e + 1]) (offsets has n_ev + 1 entries); type / obj / pt / eta / phi hold
 * lst_tc_total(ctx) rows and hits 14 per row. Any array pointer may be NULL. Pinned host memory
 * gives the fastest transfer. Waits for the copies.
 */
int64_t lst_tc_total(const lst_ctx* ctx);
int lst_copy_tc_all(lst_ctx* ctx, int32_t* offsets, int32_t* type, int32_t* obj, int32_t* hits, float* pt,
                    float* eta, float* phi);

/* Device time of each stage of the last run, in ms (CUDA events on the run's stream), indexed by
 * LST_STAGE_*; stage_ms[LST_N_STAGES] receives the whole chain. Needs lst_set_timing(ctx, 1). The
 * pT3 and pT5 kernels run interleaved in one pixel stage: LST_STAGE_PT5 holds the time of pT5's two
 * candidate kernels (pre-filter and decision), LST_STAGE_PT3 the rest of that stage. */
int lst_set_timing(lst_ctx* ctx, int enable);
int lst_get_stage_ms(const lst_ctx* ctx, float* stage_ms);

/*
 * Device time, in ms, of individual kernels of the last run (CUDA events on the run's stream;
 * needs lst_set_timing(ctx, 1)). Index order: hit binning sort/gather, MD, MD compaction, LS,
 * LS compaction, T3 pre-filter, T3 float64 decision, T3 compaction, T5 pre-filter, T5 decision,
 * pT3 pre-filter, pT5 pre-filter, pT3 decision, pT5 decision, T5 duplicate removal, TC assembly,
 * track extensions. Writes min(n, count) values and returns the count (17), or a negative
 * lst_status on error.
 */
int lst_get_kernel_ms(const lst_ctx* ctx, float* ms, int32_t n);

/*
 * Device bytes the context's arenas need for a batch of n_events events with n_hits hits and n_pls
 * seeds in total, at the default capacity predictions (what a serving loop admits work against).
 * Needs a loaded geometry; allocates nothing. Returns a negative lst_status on error.
 */
int64_t lst_predict_bytes(const lst_ctx* ctx, int32_t n_events, int64_t n_hits, int64_t n_pls);

/* Number of kernel launches issued by this context since creation (graph replays count each
 * kernel node). */
int64_t lst_launch_count(const lst_ctx* ctx);

/* Self-test of the one place where blocks wait on other blocks: the chain's single-pass scans
 * (each block adds the published totals of the tiles before it). Runs such a scan over three tiles
 * on `device` with the first tile withheld, so that the next tile's wait can never be satisfied and
 * must give up at its bound (2000 polls here; about a second in the chain, where a wait that gives
 * up ends the run with LST_ETIMEOUT). *gave_up receives the number of waits that gave up: >= 1 when
 * the bound works. No fault is involved; the device stays usable. Returns LST_OK or LST_ECUDA. */
int lst_selftest_bounded_wait(int device, int32_t* gave_up);

/* One-line description of the last error on this context (or of the last failed lst_create when
 * ctx is NULL). Never NULL. */
const char* lst_last_error(const lst_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LST_H_ */
