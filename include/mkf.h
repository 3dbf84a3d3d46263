/* mkf.h -- C ABI of the GB300 (sm_103a) Kalman-filter track-building library.
 *
 * The operations follow the problem statement of the paper (CHEP 2019 mkFit
 * status report): a lightweight detector of barrel layers at an average radius
 * and endcap disks at an average z, with a material thickness and a uniform
 * field (Sec. 2); hits given by their 3-D positions (Sec. 1, Sec. 2); seeds
 * that start the search (Sec. 1, Sec. 3); combinatorial building that keeps
 * only the best-ranking candidates up to a per-seed cap (Sec. 2), counts
 * missing hits and ranks by a score (Sec. 3), keeps short candidates (abstract)
 * and removes duplicates in a final step (abstract); and the Kalman fit over a
 * fixed hit assignment (Sec. 1).
 *
 * Conventions (every entry point):
 *  - Array arguments are caller-owned DEVICE pointers unless stated otherwise;
 *    the library never frees or retains them past the call's stream work.
 *    Structure of arrays: "[6][S]" means 6 rows of S contiguous floats.
 *  - Track parameters p = (x, y, z, kappa = q/pT, phi, theta) in cm, 1/GeV,
 *    rad.  A covariance is the packed lower triangle in row order,
 *    index(i, j) = i*(i+1)/2 + j for i >= j (21 entries).
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Argument errors are reported by
 *    the return code before anything is enqueued.  Errors detected on the
 *    device (capacity overflow, bounded waits that expired) are latched in a
 *    device status word and returned by the next mkf_sync().
 *  - A context is bound to one device and is not thread safe: use one per
 *    host thread.  It owns a workspace that grows on demand (cudaMalloc).
 *  - Streams: mkf_bin_hits, mkf_build_tracks and mkf_dedup_tracks use the
 *    context's binning and building workspace, so calls of these on one
 *    context must be ordered (same stream, or events).  mkf_fit_tracks,
 *    mkf_fit_backward and mkf_fit_tracks_adjoint touch no workspace: they may
 *    run concurrently on different streams once their inputs are ready (an
 *    adjoint next to the inward fit, for instance).
 *  - No C++ exception crosses this interface.
 */
#ifndef MKF_H
#define MKF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mkf_status;
#define MKF_OK 0
#define MKF_ERR_ARG (-1)       /* invalid argument (null pointer, size out of range) */
#define MKF_ERR_OOM (-2)       /* workspace allocation failed */
#define MKF_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define MKF_ERR_TIMEOUT (-4)   /* a bounded device-side wait expired */
#define MKF_ERR_STATE (-5)     /* call out of order (e.g. no geometry, hits not binned) */
#define MKF_ERR_CAPACITY (-6)  /* a device-side fixed-size buffer overflowed; results invalid */

/* Track flags written by mkf_build_tracks / mkf_dedup_tracks. */
#define MKF_TRK_SHORT 0        /* best candidate has fewer than min_hits hits (or none) */
#define MKF_TRK_KEPT 1         /* kept after duplicate removal */
#define MKF_TRK_DUP 2          /* removed as a duplicate of a better-scoring track */

#define MKF_MAX_LAYERS 64
#define MKF_MAX_CANDS 8

typedef struct mkf_ctx mkf_ctx;

/* Create a context on CUDA device `device`.  *out is set to NULL on failure. */
mkf_status mkf_create(mkf_ctx** out, int device);
/* Release the context and its workspace (synchronises the device first). */
void mkf_destroy(mkf_ctx* ctx);
/* Text of the last error on this context ("" if none).  Owned by the context. */
const char* mkf_last_error(const mkf_ctx* ctx);
/* Wait for all work of the context on `stream`, then read and clear the device
 * status word: MKF_OK, MKF_ERR_CAPACITY or MKF_ERR_TIMEOUT. */
mkf_status mkf_sync(mkf_ctx* ctx, void* stream);

/* One detector surface (Sec. 2: barrel layers collapsed at their average
 * radius, endcap layers at their average z, no modules). */
typedef struct {
  int kind;          /* 0: barrel cylinder r = pos; 1: endcap disk z = pos (signed) */
  float pos;         /* cm */
  float lo, hi;      /* acceptance: barrel z range, disk r range (cm) */
  float x_over_x0;   /* material thickness at normal incidence, radiation lengths */
  int n_phi_bins;    /* hit-lookup bins in phi (0: library default 64) */
  int n_w_bins;      /* hit-lookup bins in z (barrel) or r (disk) (0: default 16) */
} mkf_layer;

/* Load the detector description and the uniform field Bz (tesla).  `layers`
 * is a HOST array of n_layers (1..MKF_MAX_LAYERS) entries; it is copied. */
mkf_status mkf_load_geometry(mkf_ctx* ctx, const mkf_layer* layers, int n_layers, float bz_tesla);

/* Bin the hits of n_events events for position-based lookup (Sec. 2: the
 * search relies only on the 3-D hit positions): key = (event, layer, phi bin,
 * z bin for a barrel / r bin for a disk); counting sort + exclusive scan;
 * inside one bin hits keep ascending original index.  The binned copy stays in
 * the context for the following mkf_build_tracks calls.
 *   xyz [3][H]          global hit positions (cm)
 *   lcov [3][H]         local covariance (var_rphi, var_b, cov) with b = z on a
 *                       barrel and r on a disk (cm^2)
 *   layer [H]           layer index 0..n_layers-1 (out of range: MKF_ERR_ARG at sync)
 *   ev_hit_off [E+1]    int64 CSR offsets of each event's hits, ev_hit_off[0] = 0,
 *                       ev_hit_off[E] = H
 * Hit ids in every output are the caller's indices 0..H-1. */
mkf_status mkf_bin_hits(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                        const int64_t* ev_hit_off, int n_events, void* stream);

/* Iterative tracking (Sec. 3: hits used by the tracks of an iteration are
 * masked for the following iterations).  mkf_bin_hits_masked bins like
 * mkf_bin_hits but leaves out every hit h with mask[h] != 0 (DEVICE uint8 [H],
 * NULL = none): no later mkf_build_tracks can return it, and it does not enter
 * the window bounds; the bin offsets then cover only the hits left in.
 * mkf_used_hits sets mask[h] = 1 (DEVICE uint8 [n_hits], not cleared first)
 * for every hit of the tracks whose flag is MKF_TRK_KEPT (hits [T][L] caller
 * hit ids, -1 = none; flags [T] as written by mkf_build_tracks); an id outside
 * 0..n_hits-1 is skipped and reported as MKF_ERR_ARG by mkf_sync. */
mkf_status mkf_bin_hits_masked(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                               const int64_t* ev_hit_off, int n_events, const uint8_t* mask, void* stream);
mkf_status mkf_used_hits(mkf_ctx* ctx, const int* hits, int L, const int* flags, int64_t n_tracks, int64_t n_hits,
                         uint8_t* mask, void* stream);

/* Strip clustering (Sec. 4, the step before building that turns raw strip
 * data into hits): in every row r = event * n_modules + module of adc, seed
 * strips have ADC above 3 times the strip's noise; a cluster adds every strip
 * above twice the noise that is consecutive or separated only by bad strips,
 * at most max_bad_gap of them in a row (bad strips carry no charge); it is
 * kept if sqrt(sum ADC^2) > 5 sqrt(sum noise^2) over its strips and sum ADC
 * >= q_min.
 *   adc [n_events * n_modules][n_strips]  uint16 ADC counts (DEVICE)
 *   noise_q, bad [n_modules][n_strips]    uint16 noise in 1/8 ADC counts (so
 *                                         every test is exact in integers),
 *                                         uint8 bad-strip flag (DEVICE)
 *   out_row, out_first, out_last, out_charge [max_out] int32, out_center
 *   [max_out] float (charge-weighted strip index) (DEVICE): one entry per
 *   cluster, in no particular order;
 *   out_count (DEVICE uint64): number of clusters found, also when it is
 *   above max_out (then only max_out are written and mkf_sync returns
 *   MKF_ERR_CAPACITY).
 * MKF_ERR_ARG for bad sizes or null arrays.  With n_strips a multiple of 16,
 * at most 65536, and 16-byte aligned adc, noise_q and bad, rows are staged by TMA (tensor
 * maps encoded on each call; MKF_ERR_CUDA if the driver cannot encode them);
 * any other shape takes a plain kernel with the same results. */
mkf_status mkf_cluster_strips(mkf_ctx* ctx, const uint16_t* adc, const uint16_t* noise_q, const uint8_t* bad,
                              int n_events, int n_modules, int n_strips, int max_bad_gap, int q_min, int* out_row,
                              int* out_first, int* out_last, int* out_charge, float* out_center, int64_t max_out,
                              unsigned long long* out_count, void* stream);

/* Hit-based seeding of prompt tracks from the four innermost barrel layers
 * (Sec. 3: the initial iteration seeds from the four innermost pixel layers
 * and targets prompt tracks; the rules are this library's reading).  Uses the
 * hits of the last mkf_bin_hits / mkf_bin_hits_masked, all events:
 *  - a pair (layer 0, layer 1) defines the circle through the beam line
 *    (origin) and both hits and the line z = z0 + s cot(theta) in the
 *    transverse path s; it passes if its curvature |omega| <= alpha Bz / pt_min
 *    (pt_min in GeV) and |z0| <= z_max (cm);
 *  - that helix predicts layer 2: a hit passes if its transverse residual
 *    R2 sin(phi_hit - phi_pred) and its z residual are within rphi_tol and
 *    z_tol (cm); the helix through the origin and the layer-0 and layer-2
 *    hits predicts layer 3 the same way;
 *  - the layer-1 hit lies within 90 degrees of the layer-0 hit in azimuth,
 *    the layer-2 and layer-3 hits within 90 degrees of their predictions;
 *  - every passing quadruplet is a seed; its state is on the beam line,
 *    (0, 0, z0, kappa, phi, theta), from the circle through the origin and the
 *    layer-1 and layer-3 hits and the line through the layer-0 and layer-3
 *    hits, with a fixed diagonal covariance (sigma x, y 0.01 cm, z 0.05 cm,
 *    kappa 5 % + 0.01 /GeV, phi and theta 5 mrad).
 * Decisions are taken in FP32.  By default the call synchronises `stream` once
 * (it reads back the number of hit triplets to size its working memory), so
 * it cannot be captured in a CUDA graph; with a fixed triplet capacity set by
 * mkf_set_seed_config it does not synchronise and can be captured.  Outputs
 * (DEVICE, caller-owned):
 *   ev_seed_off [n_events + 1] int64: seeds of event e are [off[e], off[e+1]);
 *     n = ev_seed_off[n_events] is the number found;
 *   seed_par [6][n], seed_cov [21][n] float: laid out with column stride n
 *     (so the first 6 n and 21 n floats are ready for mkf_build_tracks), or
 *     with column stride max_seeds under a fixed triplet capacity (so that
 *     mkf_build_tracks can be called with n_seeds = max_seeds before n is known
 *     on the host; see there); buffers hold max_seeds columns;
 *   seed_hits [n][4] int: caller hit ids on layers 0..3.
 * If n > max_seeds nothing but ev_seed_off is written and mkf_sync returns
 * MKF_ERR_CAPACITY.  The seeds are in a fixed order (event, then layer-0 hit
 * by bin and id, then the search order).  MKF_ERR_STATE without geometry or
 * binned hits; MKF_ERR_ARG for fewer than four barrel layers, non-positive
 * cuts, pt_min so low that a circle of the largest allowed curvature does not
 * reach 1.1 times the layer-3 radius, or rphi_tol >= R2 / 2. */
mkf_status mkf_seed_tracks(mkf_ctx* ctx, float pt_min, float z_max, float rphi_tol, float z_tol, int64_t max_seeds,
                           float* seed_par, float* seed_cov, int* seed_hits, int64_t* ev_seed_off, void* stream);

/* Fixed triplet capacity of mkf_seed_tracks.  max_triplets = 0 (default):
 * the triplet list is sized from its count, read back once per call (the call
 * synchronises its stream).  max_triplets > 0: the list holds that many
 * triplets, nothing is read back, and the call can be captured in a CUDA
 * graph; a list that does not fit is not searched, ev_seed_off then counts no
 * seeds of the events past the fit, and mkf_sync returns MKF_ERR_CAPACITY.
 * The paper has no counterpart.  MKF_ERR_ARG outside 0..2^31-2. */
mkf_status mkf_set_seed_config(mkf_ctx* ctx, int64_t max_triplets);

/* Work counters of the last mkf_seed_tracks (synchronises `stream`): [0]
 * layer-1 hits examined in the pair windows, [1] pairs that passed, [2]
 * layer-2 hits examined, [3] triplets, [4] layer-3 hits examined, [5] seeds.
 * HOST output of n <= 6 values (zeros before the first call). */
mkf_status mkf_get_seed_stats(mkf_ctx* ctx, int64_t* out, int n, void* stream);

/* Recovery of hits in overlapping detector modules (Sec. 3: more than one hit
 * per layer assigned to a track; the paper plans the feature without a rule,
 * so this is the library's reading).  For each track the forward fit of
 * mkf_fit_tracks runs over its hits (same steps, FP32); after the update with
 * its hit h on layer l, the overlap hit of that crossing is the other hit of
 * layer l (in h's event, among the binned hits of the last mkf_bin_hits, which
 * must be these hits) inside the adjacent-module box around h -- |R sin(phi -
 * phi_h)| <= max_drphi with cos > 0 (R the layer radius on a barrel, h's
 * radius on a disk) and |w - w_h| <= max_dw (w = z on a barrel, r on a disk),
 * in cm -- with the smallest predicted chi2 against the updated state, if
 * below chi2_cut (ties: smaller id).  The state is not updated with
 * it.  Inputs as for mkf_fit_tracks (no alignment or thickness override).
 * Outputs (DEVICE): out_hit [T][K] caller hit id or -1 for each slot,
 * out_chi2 [T][K] its chi2 (0 when none).  Slots after a surface that is not
 * reached stay -1.  MKF_ERR_STATE without geometry or binned hits,
 * MKF_ERR_ARG if n_hits differs from the binned hits. */
mkf_status mkf_find_overlaps(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                             const int* hits, int K, const float* init_par, const float* init_cov, int64_t n_tracks,
                             float chi2_cut, float max_drphi, float max_dw, int* out_hit, float* out_chi2,
                             void* stream);

/* Launch shape of mkf_find_overlaps: lanes_per_track 1 (one thread per track),
 * 8 (eight lanes per track run its fit together and share the hits of each
 * search window), or 0 = by track count (8 below 128 tracks per SM).  Speed
 * only: the overlap hits and chi2 values are the same in every shape.  The
 * paper has no counterpart.  MKF_ERR_ARG for any other value. */
mkf_status mkf_set_overlap_config(mkf_ctx* ctx, int lanes_per_track);

/* Work counters of the last mkf_find_overlaps (synchronises `stream`): [0]
 * track hits fitted, [1] candidate hits whose chi2 was evaluated, [2] overlap
 * hits found.  HOST output of n <= 3 values. */
mkf_status mkf_get_overlap_stats(mkf_ctx* ctx, int64_t* out, int n, void* stream);

/* Read back the binning (for inspection and tests): perm [H] original id of
 * each sorted position, bin_off [n_bins_total+1] first sorted position of each
 * (event, layer, bin), n_bins_total = n_events * sum_l(n_phi_l * n_w_l).
 * The first call after mkf_bin_hits sorts each bin by original id (a kernel on
 * `stream`), so the order read back is a stable sort by bin; building does not
 * depend on the order inside a bin and does not wait for this sort.
 * DEVICE output pointers; either may be NULL.  Returns n_bins_total in *n_bins. */
mkf_status mkf_get_binning(mkf_ctx* ctx, int* perm, int* bin_off, int64_t* n_bins, void* stream);

/* Combinatorial Kalman-filter track building for all seeds of all binned
 * events (Sec. 1: propagate layer N-1 -> N, update with the hit; Sec. 2: only
 * the best-ranking candidates are kept per layer, up to max_cands per seed;
 * Sec. 3: missing hits (holes) counted, candidates ranked by a score;
 * abstract: short candidates preserved, duplicates removed at the end).
 * Per step every active candidate moves outward to its next reachable
 * surface, its covariance is transported and inflated for multiple
 * scattering, chi2 is evaluated against the hits in a conservative window,
 * children are formed (one per hit with chi2 < chi2_cut, plus a hole child
 * while holes <= max_holes), the max_cands best children by
 * score = 10 n_hits - 10 n_holes - sum chi2 (ties: parent slot, hit id, hole
 * last) are updated and kept.  A candidate with no next surface or no child
 * is finished.  The best finished candidate of a seed is its track; tracks
 * with at least min_hits hits go through greedy duplicate removal per event
 * (drop a track sharing more than dup_frac of min(n_a, n_b) hits with a
 * better-scoring kept track).
 *   seed_par [6][S], seed_cov [21][S]   seed states
 *   ev_seed_off [E+1]                    int64 CSR offsets of each event's seeds;
 *                                        when ev_seed_off[E] (read on the device)
 *                                        is below S, only those seeds are built
 *                                        and rows ev_seed_off[E]..S-1 are written
 *                                        as empty tracks (no hits, zero state,
 *                                        MKF_TRK_SHORT): hit-based seeds with a
 *                                        fixed triplet capacity build with
 *                                        S = max_seeds and no host read-back
 *   max_cands 1..MKF_MAX_CANDS, max_holes >= 0, min_hits >= 0, 0 <= dup_frac <= 1
 * Outputs ([S] arrays, DEVICE; out_layers, out_counts may be NULL):
 *   out_hits [S][L]     hit id at the k-th crossed surface, -1 for a hole or past the end
 *   out_layers [S][L]   surface index of the k-th crossing, -1 past the end
 *   out_par [6][S], out_cov [21][S]  state of the track at its last surface
 *   out_score [S], out_chi2 [S]      score and sum of chi2
 *   out_counts [3][S]   n_hits, n_holes, n_steps
 *   out_flags [S]       MKF_TRK_* */
mkf_status mkf_build_tracks(mkf_ctx* ctx, const float* seed_par, const float* seed_cov, const int64_t* ev_seed_off,
                            int64_t n_seeds, float chi2_cut, int max_cands, int max_holes, int min_hits,
                            float dup_frac, int* out_hits, int* out_layers, float* out_par, float* out_cov,
                            float* out_score, float* out_chi2, int* out_counts, int* out_flags, void* stream);

/* Launch shape of the building kernel: warps per thread block (1, 2, 4 or 8;
 * default 4) and lanes per seed (a power of two up to 32, at least max_cands;
 * 0 = max_cands rounded up).  More lanes per seed shorten the search of wide
 * windows, fewer keep more seeds in flight.  Chosen by the autotuner
 * (paper_2002_06295_gb300/tune.py); it changes speed only, never results. */
mkf_status mkf_set_build_config(mkf_ctx* ctx, int warps_per_block, int lanes_per_seed);

/* Duplicate removal inside mkf_build_tracks (abstract: an additional
 * processing step after building).  enabled = 1 (default): mkf_build_tracks
 * ends with it and writes out_flags.  enabled = 0: mkf_build_tracks leaves
 * out_flags of the built seeds unwritten (rows past ev_seed_off[E] are still
 * written MKF_TRK_SHORT), and the caller runs mkf_dedup_tracks on the built
 * tracks (nhits = out_counts[0]), which gives the same flags.  Because the fits
 * do not read the flags, that call may then run on another stream beside
 * mkf_fit_tracks.  MKF_ERR_ARG unless 0 or 1. */
mkf_status mkf_set_build_dedup(mkf_ctx* ctx, int enabled);

/* Work split of mkf_cluster_strips (TMA path): strips per staged chunk,
 * events per work item (an item is 32 consecutive modules of that many events,
 * whose calibration is staged once per chunk) and pipeline stages per warp.
 * Built splits (chunk, events, stages): (32,1,1) (32,1,2) (32,1,3) (32,1,4) (32,2,2)
 * (64,1,2) (64,1,3) (64,2,2); 0, 0, 0 = default: (32,1,1).
 * Speed only: the clusters found are the same (their order in the output is
 * not fixed anyway).  MKF_ERR_ARG for any other triple.  The paper has no
 * counterpart. */
mkf_status mkf_set_strip_config(mkf_ctx* ctx, int chunk, int events_per_item, int stages);

/* Launch shape of mkf_fit_tracks_adjoint: lanes_per_track 1 (one thread per
 * track), 8 (eight lanes per track share the dual-number passes), or 0 =
 * choose by the number of tracks (8 below 128 tracks per SM).  The paper has
 * no counterpart (the adjoint is not in the paper).  Speed only: both shapes
 * compute the same contribution of every track bit for bit (sums over tracks
 * are accumulated by atomics, so they agree to rounding).  MKF_ERR_ARG for any
 * other value. */
mkf_status mkf_set_adjoint_config(mkf_ctx* ctx, int lanes_per_track);

/* Debug switch for mkf_build_tracks: when on, every candidate step also
 * evaluates chi2 against every hit of the layer and counts accepted hits that
 * lay outside its search window (statistic 4 of mkf_get_stats; it must be 0). */
mkf_status mkf_set_debug(mkf_ctx* ctx, int brute_force_window_check);

/* Work counters of the last mkf_build_tracks (synchronises `stream`):
 * [0] candidate steps, [1] candidate-hit pairs examined in the search windows
 * (each gets the window box test), [2] hit updates, [3] tracks kept,
 * [4] window violations (debug), [5] navigation surface tests whose crossing was
 * computed, [6] seeds,
 * [7] pairs that passed the box test and had their chi2 computed.
 * HOST output of n <= 8 values. */
mkf_status mkf_get_stats(mkf_ctx* ctx, int64_t* out, int n, void* stream);

/* Kernel timing.  When on, the library records CUDA events on the launch
 * stream around its kernels; mkf_get_timings returns the device time of the
 * most recent call of each stage in milliseconds (synchronises `stream`):
 * [0] track-building kernel, [1] hit binning (all its kernels), [2] duplicate
 * removal, [3] forward fit, [4] fit adjoint, [5] backward fit.  A stage not run
 * since timing was switched on reads as -1.  HOST output of n <= 8 floats. */
mkf_status mkf_set_timing(mkf_ctx* ctx, int on);
mkf_status mkf_get_timings(mkf_ctx* ctx, float* ms, int n, void* stream);

/* Duplicate removal alone on given tracks (same rule as in mkf_build_tracks):
 *   hits [S][L] hit ids (-1 none), score [S], nhits [S], ev_seed_off [E+1]
 *   out_flags [S]  MKF_TRK_*  */
mkf_status mkf_dedup_tracks(mkf_ctx* ctx, const int* hits, int L, const float* score, const int* nhits,
                            const int64_t* ev_seed_off, int n_events, int64_t n_seeds, int64_t n_hits_total,
                            int min_hits, float dup_frac, int* out_flags, void* stream);

/* Duplicate removal without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run (a trigger or online process that reserves its
 * whole memory budget at start-up, or a thread that must not take the implicit
 * device synchronisation of cudaMalloc).  Same rule and arguments as
 * mkf_dedup_tracks, but no context: its working memory is one fixed 8.5 MB
 * array in the library's device image, which every GPU that loads the library
 * holds until the process exits.  Limits: n_seeds <= 16384,
 * n_hits_total <= 524288, L <= MKF_MAX_LAYERS; larger inputs return
 * MKF_ERR_CAPACITY and nothing is enqueued.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  That address is
 * kept for the life of the process, so it assumes the device's primary context
 * stays alive: do not call this entry point again after cudaDeviceReset.  All
 * calls share the array: calls whose work can overlap on the GPU race and must
 * be serialised by the caller.  Device-side problems are written as MKF status
 * bits to out_status (DEVICE int, cleared by the call; may be NULL): 2
 * resolution did not converge, 4 an input index out of range (a hit id, or an
 * event offset outside 0..n_seeds, which is clamped into that range so that
 * nothing is read or written past the track arrays). */
mkf_status mkf_dedup_tracks_noalloc(const int* hits, int L, const float* score, const int* nhits,
                                    const int64_t* ev_seed_off, int n_events, int64_t n_seeds, int64_t n_hits_total,
                                    int min_hits, float dup_frac, int* out_flags, int* out_status, void* stream);

/* Kalman fit over a fixed hit assignment (Sec. 1: "fitting simply applies the
 * KF procedure to all hits identified during building").  For each listed hit
 * in crossing order: propagate to that hit's surface, add its material,
 * update with the hit (no cut).
 *   xyz [3][H], lcov [3][H], layer [H]   hits (as for mkf_bin_hits)
 *   hits [T][K]          hit ids in crossing order, -1 entries skipped
 *   init_par [6][T], init_cov [21][T]
 *   align [L][3] or NULL  per-layer (dr, dphi, dz): barrel radius and hits
 *                         shift by dr (radially), hit azimuths by dphi, hit z by
 *                         dz; for a disk its z and the hits' z shift by dz,
 *                         hit radii by dr, azimuths by dphi
 *   x0 [L] or NULL        per-layer thickness overriding the geometry's
 * Outputs: out_par [6][T], out_cov [21][T], out_chi2 [T] (sum of chi2),
 *   out_ok [T] or NULL: 1 every surface reached; 2 every surface reached, and
 *     a transport onto an endcap disk spans a full turn of the helix or more
 *     (|s omega| >= 2 pi: a slow particle near theta = pi/2 drifting from disk
 *     to disk over several turns), on which mkf_fit_tracks_adjoint's FP32
 *     reverse sweep is not accurate, so it leaves the track out; 0 a surface
 *     not reached,
 *   ckpt [K][27][T] or NULL: state (6 parameters, 21 covariance) before step k,
 *   needed by mkf_fit_tracks_adjoint.
 * A row with no listed hit returns init_par and init_cov unchanged, chi2 0,
 * ok 1; n_tracks = 0 launches nothing. */
mkf_status mkf_fit_tracks(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                          const int* hits, int K, const float* init_par, const float* init_cov, int64_t n_tracks,
                          const float* align, const float* x0, float* out_par, float* out_cov, float* out_chi2,
                          int* out_ok, float* ckpt, void* stream);

/* Backward (inward) fit: starts from init_par = the forward result at the
 * outermost listed hit, with the covariance reset to 100 x the seed-style
 * diagonal (0.01, 0.01, 0.01 cm^2, (0.05 kappa)^2, 0.0025, 0.0025), updates
 * with the outermost hit in place, then propagates inward (negative path) to
 * each earlier hit, adds its material and updates.  Arguments as
 * mkf_fit_tracks (init_cov is ignored; ckpt unsupported, pass NULL).  A row
 * with no listed hit returns init_par with that reset covariance, chi2 0, ok 1.
 * Arithmetic: FP64 (the multiple-scattering term in FP32); outputs rounded
 * to FP32.  The prior makes the first updates shrink variances by up to 1e5,
 * and on built tracks that carry wrong picks the updates move the state by
 * hundreds of standard deviations, which an FP32 state (also one with U-D
 * factorised covariance) does not carry to 1e-4 on every track. */
mkf_status mkf_fit_backward(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer, int64_t n_hits,
                            const int* hits, int K, const float* init_par, int64_t n_tracks, const float* align,
                            const float* x0, float* out_par, float* out_cov, float* out_chi2, int* out_ok,
                            void* stream);

/* Adjoint (reverse mode) of mkf_fit_tracks.  Not in the paper: gradient of
 *   loss = sum_t g_chi2[t] chi2_t + g_par[.][t] . p_t + g_cov[.][t] . C_t
 * (C_t packed) with respect to the hit positions, the per-layer alignment and
 * the per-layer thickness.  Needs the checkpoints written by the forward call
 * with the same inputs; recomputes each step's propagation from them.
 *   g_chi2 [T], g_par [6][T], g_cov [21][T]: upstream gradients, any may be NULL
 * Outputs (overwritten): g_hit_xyz [3][H], g_align [L][3], g_x0 [L].
 * Tracks that the forward fit reports with out_ok = 2 contribute nothing
 * (the test is repeated here on the checkpointed states, so the two agree). */
mkf_status mkf_fit_tracks_adjoint(mkf_ctx* ctx, const float* xyz, const float* lcov, const int* layer,
                                  int64_t n_hits, const int* hits, int K, const float* init_par,
                                  const float* init_cov, int64_t n_tracks, const float* align, const float* x0,
                                  const float* ckpt, const float* g_chi2, const float* g_par, const float* g_cov,
                                  float* g_hit_xyz, float* g_align, float* g_x0, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MKF_H */
