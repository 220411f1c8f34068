/*
 * tpctrack.h — C-ABI of the GB300 TPC sector-tracking library (libtpctrack.so).
 *
 * The library implements the standalone TPC sector tracking of the synchronous reconstruction
 * described in "Overview of online and offline reconstruction in ALICE for LHC Run 3"
 * (arXiv:2009.07515): clusters of a continuous-readout time frame in (Sec. 2: native row/time
 * coordinates, z unknown until a vertex time is known), sector tracks with helix parameters,
 * covariances and cluster indices out (Sec. 6: TPC tracking runs standalone, without space-charge,
 * field or hit-error corrections; the algorithm derives from the Run-2 HLT tracker). Every stage
 * runs as a CUDA kernel on one GPU: per-row search grid, cellular-automaton neighbour finding and
 * cleaning, start-hit selection, Kalman-filter tracklet construction in the solenoid field, and
 * tracklet selection.
 *
 * Conventions
 *   - Every call returns TPC_OK (0) or a negative TPC_E_* code. No call aborts, traps or waits
 *     without a bound; tpc_last_error() gives a one-line description of the last failure.
 *   - A context (tpc_ctx) is used by one host thread at a time.
 *   - Coordinates: sector s in [0,36) (s/18 = drift side A/C, s%18 = 20-degree phi sector), pad
 *     row r in [0,152) at radius x_r = 85 + r*160/151 cm (sector-local x), y = local coordinate
 *     along the pad row (cm), w = v_drift * t_arrival (cm): the drift-time coordinate of continuous
 *     readout (Sec. 2). Track parameters are (y, w, sin(phi), dw/ds, q/pT) at x = x_ref in the
 *     sector frame; s is the path length in the bending plane; curvature = -0.0029979246*Bz*q/pT.
 *   - Covariances are the 15-element lower triangle, row-major: (0,0),(1,0),(1,1),(2,0),...,(4,4).
 */
#ifndef TPCTRACK_H
#define TPCTRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPC_OK 0
#define TPC_E_INVAL -1    /* malformed argument, handle or cluster data */
#define TPC_E_NOMEM -2    /* device or host allocation failed */
#define TPC_E_BUDGET -3   /* a frame larger than the whole HBM budget */
#define TPC_E_CAPACITY -4 /* an internal capacity overflowed and could not be grown */
#define TPC_E_TIMEOUT -5  /* a bounded device wait or tpc_poll timeout expired */
#define TPC_E_CUDA -6     /* a CUDA runtime call failed */
#define TPC_E_STATE -7    /* call not valid in the frame's current state */

#define TPC_NSECTORS 36
#define TPC_NROWS 152

typedef struct tpc_ctx tpc_ctx;
typedef uint64_t tpc_frame_t; /* frame handle / serving ticket; 0 is never a valid handle */

/* Method and runtime parameters. Obtain defaults with tpc_default_params(), then edit. */
typedef struct {
  uint32_t struct_size;   /* = sizeof(tpc_params) */
  /* method parameters (the tracker's readings of the HLT-derived algorithm). They are given in
   * double and rounded once to float on the device, as derived constants are: kq = (float)(
   * -0.0029979246*bz), sigma^2 = (float)(sigma*sigma), Highland constant from x0_per_row. */
  double bz;              /* solenoid field, T (0.5) */
  double ky, kw, eps;     /* neighbour windows |dy| <= ky*dx + eps, |dw| <= kw*dx + eps (cm) */
  double chi_n_max;       /* neighbour mid-point deviation cut dy^2 + dw^2 (cm^2) */
  int32_t lmin;           /* minimum cleaned-chain length of a start hit (6) */
  double sigma_y, sigma_w;/* cluster errors (cm) */
  double chi2_hit_max;    /* Kalman hit acceptance, 2 dof (16) */
  int32_t n_miss_max;     /* consecutive empty rows ending an extension (5) */
  double win_nsig, win_add; /* extension search window nsig*sqrt(C) + add (cm) */
  double x0_per_row;      /* X/X0 per row for scattering noise (0.03/152); 0 = none */
  double max_sin;         /* |sin(phi)| limit of propagation (0.999) */
  double y_margin;        /* stop extending when |y| > x*tan(10 deg) + y_margin (cm) */
  int32_t nmin;           /* minimum hits of a voting tracklet and of a track (10) */
  double cov0[5];         /* seed covariance diagonal */
  int32_t ext_stop;       /* 1: a tracklet's outward extension ends once it accepts the start hit of
                             another tracklet, whose tracklet covers the rows beyond (1) */
  double drift_length;    /* drift length L, cm: a cluster of a collision at time t_c has
                             w = v_d t_c + L - |z| (250) */
  double drift_velocity;  /* v_d, cm per microsecond (250/90) */
  double keep_vy, keep_vw;/* compression, strategy B (Sec. 4): clusters within +-keep_vy in y and
                             +-keep_vw in w of a good track's predicted position are kept (1, 1 cm) */
  double keep_qpt_max;    /* a good track has |q/pT| <= keep_qpt_max, i.e. pT >= 50 MeV/c (20) */
  /* storage / runtime */
  int32_t packed;         /* 1: store cluster coordinates as 16-bit offsets in their grid bin */
  float bin_occupancy;    /* target clusters per bin of the search grid (1); a launch-shape knob */
  float tracklet_capacity;/* tracklet slots per cluster reserved in a workspace (0.08) */
  int64_t hbm_budget;     /* serving admission budget in bytes (80 GB) */
  int32_t max_batch_frames; /* frames per batched launch (16) */
  int32_t use_graphs;     /* 1: replay the kernel sequence as a CUDA graph */
  int32_t compress;       /* 1: also compute the compression inputs (track-model residuals, strategy-B
                             keep mask; tpc_tracks.residual, tpc_get_keep_mask) (0) */
  /* launch shapes: no result depends on them; tpc_autotune() picks them by timing */
  int32_t k2_warps;       /* neighbour search: warps per block, each on 32 hits of one row at a
                             time (4 or 8) */
  int32_t k2_tma;         /* neighbour search reads of the adjacent rows: 0 through L1, each lane
                             walking its window's bins; 1 staged in shared memory by bulk TMA
                             copies, each lane walking its bins; 2 staged, and scanned once by the
                             whole warp with per-lane candidate lists */
  int32_t k5_block;       /* tracklet construction: threads per block, one tracklet per thread at
                             a time (64, 128 or 256) */
  int32_t k5_regs;        /* registers per tracklet thread the kernel is compiled for (64, 72, 80;
                             see k5_ilp for 2 tracklets per thread) */
  int32_t k5_blocks_per_sm; /* tracklet blocks launched per SM (0 = all that fit); with k5_block
                             it sets how many tracklets each warp builds */
  int32_t k5_order;       /* tracklet processing order: 0 canonical, 1 longest chain first,
                             2 innermost start row first, 3 outermost start row first */
  int32_t sel_lanes;      /* tracklet selection: lanes per tracklet, 32 (a warp takes its rows 32
                             at a time) or 1 (a warp takes a tile of 32 tracklets row by row) */
  int32_t autotune;       /* 1: the first tpc_track_batch / tpc_track_sectors call runs
                             tpc_autotune() on its batch first (0) */
  /* merging across sector boundaries and the global refit (Sec. 6: the tracks are refit after the
   * sector tracking; Table 1 of Sec. 7.2: "Track Fit"); results from tpc_get_merged_tracks() */
  int32_t merge;          /* 1: also merge and refit the frame's sector tracks (0) */
  int32_t merge_gap_rows; /* the outer segment's reference row lies 1 .. this many rows above the
                             inner segment's last hit row (10) */
  double merge_dw;        /* |w(outer segment at x_ref) - w(inner segment at its last row)| <= this,
                             cm (5) */
  double merge_chi2_max;  /* 5-parameter chi2 cut of a merge (50) */
  int32_t refit_passes;   /* Kalman passes of the refit, alternately inward and outward, odd (3) */
  double refit_scale;     /* a refit pass starts from the previous pass's covariance times this (100) */
  int32_t k5_ilp;         /* launch shape: tracklets each tracklet thread keeps in flight, 1 or 2; with
                             2 a thread advances both by one row step per iteration, phase by
                             phase, with k5_block 64 or 128 and k5_regs 128 (1) */
  int32_t wide_votes;     /* tracklet selection: 0 votes with 32-bit keys (hit count, start-hit
                             rank) while every rank of the batch is below 2^24, else 64-bit keys;
                             1 always 64-bit keys. The selection is the same either way (0) */
} tpc_params;

/* Clusters of one time frame, structure of arrays in the caller's order (n entries each).
 * on_device = 0: host pointers, copied before tpc_load_clusters/tpc_submit_frame returns.
 * on_device = 1: device pointers borrowed until the frame's tracking has completed.
 * on_device = 2: host pointers (page-locked for an asynchronous copy) borrowed by tpc_submit_frame
 *                until the frame's tracks are read: the frame is uploaded when it is admitted, on
 *                the stream of the slot that tracks it, and waits in the queue without a host copy
 *                or device memory; the caller keeps the arrays unchanged until tpc_get_tracks() of
 *                the frame. tpc_load_clusters() copies such input before return, as for 0. */
typedef struct {
  const uint8_t* sector;
  const uint8_t* row;
  const float* y;
  const float* w;
  int64_t n;
  int32_t on_device;
} tpc_clusters;

/* Host views of a frame's sector tracks, owned by the context until tpc_release_frame().
 * Tracks are in canonical order: sector, then the row-rank of the tracklet's start hit (its
 * position among the sector's clusters ordered by row, w, y, input index). Hit lists run in
 * ascending row order and hold indices into the caller's cluster arrays. */
typedef struct {
  int64_t n_tracks;
  const int32_t* sector;      /* [n] */
  const float* x_ref;         /* [n] x of the innermost fitted hit */
  const float* param;         /* [n][5] y, w, sin(phi), dw/ds, q/pT at x_ref */
  const float* cov;           /* [n][15] lower triangle */
  const float* chi2;          /* [n] */
  const int32_t* ndf;         /* [n] 2*(fitted hits) - 5 */
  const int64_t* hit_offset;  /* [n+1] */
  const uint32_t* hit_index;  /* [hit_offset[n]] */
  const float* beam;          /* [n][5] the fit transported to the beam line x = 0 without material
                                 (Sec. 6): y0, w0, var(w0), then for a primary from z = 0 its
                                 collision time t0 = (w0 - L)/v_d (us) and its z at x_ref,
                                 +-(w0 - w_ref) (+ on side A); all NaN where the transport fails
                                 (|sin(phi)| reaches max_sin before x = 0) */
  /* compression inputs (Sec. 4), NULL unless tpc_params.compress: each track's fit is transported
   * (state only, no scattering) from x_ref directly to each row it spans; hit i of the track is stored as
   * q(hit) - q(prediction) at its row, q(v) = rint(512 v) in units of 2^-9 cm, for i < n_pred, and
   * as q(hit) beyond (the transport failed there). A decoder with the same arithmetic restores q(hit). */
  const int32_t* residual;    /* [hit_offset[n]][2] (y, w) */
  const int32_t* n_pred;      /* [n] */
} tpc_tracks;

/* Merged tracks of a frame (tpc_params.merge = 1), owned by the context until tpc_release_frame().
 * Each is a chain of sector tracks (segments) in phi-neighbouring sectors of one drift side, inner to
 * outer, refit over all its hits; a sector track without partners is a chain of one. Order: the
 * canonical index of the innermost segment. */
typedef struct {
  int64_t n_merged;
  const int32_t* sector;      /* [n] sector whose frame holds the refit result (the innermost segment's) */
  const int32_t* n_seg;       /* [n] segments */
  const int32_t* head;        /* [n] index of the innermost segment among the frame's sector tracks */
  const float* x_ref;         /* [n] x of the innermost refit hit */
  const float* param;         /* [n][5] y, w, sin(phi), dw/ds, q/pT at x_ref */
  const float* cov;           /* [n][15] lower triangle */
  const float* chi2;          /* [n] chi2 of the last refit pass */
  const int32_t* ndf;         /* [n] 2 * n_fit - 5 */
  const int32_t* n_fit;       /* [n] hits of the last refit pass (all of them unless a step failed) */
  const int64_t* hit_offset;  /* [n+1] */
  const uint32_t* hit_index;  /* the segments' hits, inner segment first, each in ascending row */
  int64_t n_tracks;           /* the frame's sector tracks */
  const int32_t* track_next;  /* [n_tracks] each sector track's outer partner, -1 if none */
  const float* track_merge_chi2; /* [n_tracks] chi2 of that merge, NaN if none */
} tpc_merged_tracks;

/* Per-kernel device time of the last tpc_track_* call on a frame or batch (CUDA events on the
 * launching stream; filled when timing is enabled with tpc_set_timing). */
typedef struct {
  int32_t n_kernels;
  const char* const* names;
  const float* ms;            /* [n_kernels] device time of each stage */
  const int64_t* launches;    /* [n_kernels] kernel launches of each stage */
} tpc_kernel_times;

/* Defaults of every parameter: the method's readings of Sec. 6 (the paper gives no values) and the
 * runtime's sizes. */
void tpc_default_params(tpc_params* p);

/* Create a context on the current CUDA device. It owns the device memory and streams of the
 * tracking steps of Sec. 6 (the paper's one GPU per time frame, Sec. 7.1). */
int tpc_create(const tpc_params* p, tpc_ctx** out);
/* Free the context and all its device and host memory (no counterpart in the paper). */
void tpc_destroy(tpc_ctx* ctx);
/* One-line description of the context's last failure (no counterpart in the paper). */
const char* tpc_last_error(const tpc_ctx* ctx);
/* Library name and version (no counterpart in the paper). */
const char* tpc_version(void);

/* Load one frame's clusters (Sec. 2: a time frame of continuous readout in native row and time
 * coordinates; frames are reconstructed independently). Validated on the device during tracking:
 * sector < 36, row < 152, finite y and w. Returns a frame handle in *out. */
int tpc_load_clusters(tpc_ctx* ctx, const tpc_clusters* clusters, tpc_frame_t* out);

/* Enqueue the standalone sector tracking of one loaded frame (Sec. 6: tracking without corrections,
 * derived from the Run-2 HLT tracker) on `cuda_stream` (a cudaStream_t; NULL = the context's
 * stream). Asynchronous: results are available from tpc_get_tracks(). */
int tpc_track_sectors(tpc_ctx* ctx, tpc_frame_t frame, void* cuda_stream);

/* Enqueue tracking of several loaded frames in one batched launch sequence (all their sectors
 * together; Sec. 7.1: enough parallelism comes from processing many collisions in one go). Each
 * frame's tracks are identical to tracking it alone. */
int tpc_track_batch(tpc_ctx* ctx, const tpc_frame_t* frames, int32_t n_frames, void* cuda_stream);

/* Wait (bounded) for the frame's tracking and return host views of its sector tracks (Sec. 6:
 * tracks with parameters, covariances and their clusters). */
int tpc_get_tracks(tpc_ctx* ctx, tpc_frame_t frame, tpc_tracks* out);

/* Merged and refit tracks of a tracked frame (tpc_params.merge = 1; else TPC_E_STATE): the step
 * after the sector tracking (Sec. 6: the tracks are refit; Table 1 of Sec. 7.2 times it as "Track
 * Fit", with its sorts). The paper gives no rule; the library computes:
 *   outer state  each sector track's fit transported row by row, with the scattering noise of each
 *                row, from its reference row to the row of its last hit;
 *   candidates   a sector track B of a phi-neighbouring sector of the same frame and drift side whose
 *                reference row lies 1 .. merge_gap_rows above A's last hit row, with
 *                |w_B(x_ref) - w_A(outer)| <= merge_dw;
 *   chi2         A's outer state rotated into B's frame (the point kept, the direction angle less
 *                20 degrees, the covariance carried at fixed x to first order) and carried by one
 *                helix step with one row of scattering noise to B's x_ref; chi2 = d^T (C_A + C_B)^-1 d
 *                over the 5 parameters (Cholesky), at most merge_chi2_max;
 *   matching     A's best candidate and B's best candidate (smallest chi2, tie: smaller index); the
 *                two merge when each is the other's best; merged pairs chain inner to outer;
 *   refit        every chain refit over all its hits by the Kalman filter of the tracklets (no hit
 *                rejected) in refit_passes passes, inward, outward, inward, each from the previous
 *                pass's end state with its covariance times refit_scale (the first from the
 *                outermost segment's outer state), row by row within a segment, rotated into the next
 *                hit's frame at a segment change and carried by one step to its row; a failed step
 *                ends the refit at the last updated hit (NaN fit if no hit was updated).
 * No pair across the central membrane (opposite drift sides) is formed: there the drift coordinate
 * of the outer segment mirrors about the unknown collision time (primaries from z = 0 never cross it).
 * Host views, valid until tpc_release_frame(). */
int tpc_get_merged_tracks(tpc_ctx* ctx, tpc_frame_t frame, tpc_merged_tracks* out);

/* Free the frame's device and host memory (Sec. 7.1: memory is reused for consecutive steps and
 * frames rather than held per collision). */
int tpc_release_frame(tpc_ctx* ctx, tpc_frame_t frame);

/* Serving: admit a frame (copied/borrowed as for tpc_load_clusters) into the request queue. The
 * paper has no serving loop; this follows the continuous-batching pattern of this library (frames of
 * uneven size admitted by HBM budget, their work overlapped on the device).
 * Never blocks on the HBM budget: frames wait host-side until memory frees up. A frame larger
 * than the whole budget is refused with TPC_E_BUDGET. */
int tpc_submit_frame(tpc_ctx* ctx, const tpc_clusters* clusters, tpc_frame_t* ticket);

/* Serving (no counterpart in the paper; the continuous-batching pattern of tpc_submit_frame):
 * advance the scheduler (retire finished batches, queueing their results' copies; admit
 * queued frames into free slots, a batch growing only while it holds at most 2^21 clusters, and
 * launch it) and return up to max_done finished tickets in done[] (frames whose results are on the
 * host); waits at most timeout_us for at least one.
 * Returns the number of tickets written (>= 0) or a negative error. Finished frames are read
 * with tpc_get_tracks() and freed with tpc_release_frame(). */
int tpc_poll(tpc_ctx* ctx, tpc_frame_t* done, int32_t max_done, int32_t timeout_us);

/* Diagnostics for parity tests (the cellular-automaton links of the HLT-derived tracker, Sec. 6):
 * copy a per-cluster array of a tracked frame into host memory
 * (caller-owned, n = number of clusters), indexed by the caller's cluster order.
 * what: 0 = raw up link, 1 = raw down link, 2 = cleaned up link, 3 = cleaned down link
 * (each the input index of the linked cluster or -1). */
int tpc_get_links(tpc_ctx* ctx, tpc_frame_t frame, int32_t what, int32_t* host_out, int64_t n);

/* Compression, strategy B (Sec. 4: every hit not in the vicinity of a good track is removed): copy
 * the keep mask of a tracked frame into host memory (caller-owned, n = number of clusters), indexed
 * by the caller's cluster order: 1 = kept (a hit of a good track, or within +-(keep_vy, keep_vw) of a
 * good track's predicted position at its row), 0 = removed. Needs tpc_params.compress = 1 (else
 * TPC_E_STATE). */
int tpc_get_keep_mask(tpc_ctx* ctx, tpc_frame_t frame, uint8_t* host_out, int64_t n);

/* Number of start hits and of tracks of a tracked frame (diagnostic; Sec. 6 steps). */
int tpc_get_counts(tpc_ctx* ctx, tpc_frame_t frame, int64_t* n_start, int64_t* n_tracks);

/* Device counters of the batch a frame was tracked in, for diagnostics and roofline accounting
 * (no counterpart in the paper):
 * out[0..n) = clusters, clusters in the grid, grid bins, start hits, tracklets, tracklet row steps,
 * hits fitted by tracklets, tracks, track hits, device error bits. Returns the number of counters
 * available (>= 0) or a negative error. */
int tpc_get_stats(tpc_ctx* ctx, tpc_frame_t frame, int64_t* out, int32_t n);

/* ---- autotuning of the launch shapes (the batched persistent path's rows-per-block and
 * tracklets-per-warp choices; the paper has no tuner: its one common source runs on CUDA,
 * OpenCL, HIP and the CPU, abstract). One timed configuration: */
typedef struct {
  float bin_occupancy;
  int32_t k2_warps, k2_tma, k5_block, k5_regs, k5_blocks_per_sm, k5_order, sel_lanes;
  float ms;        /* median device time of the stages the knob being tuned acts on */
  float total_ms;  /* median device time of the whole sequence */
  int32_t stage;   /* what ms measures: 0 all stages, 1 neighbour search, 2 chains + tracklets,
                      3 votes + kept + write_tracks */
  int32_t k5_ilp;
} tpc_tune_entry;
typedef struct {
  int32_t n_entries;               /* configurations timed, in the order they were timed */
  const tpc_tune_entry* entries;   /* owned by the context until the next tpc_autotune call */
  int32_t best;                    /* index of the chosen configuration (now the context's) */
} tpc_tune_report;
/* Times launch shapes on the given frames (a batch, as tpc_track_batch runs it) and keeps the
 * fastest for the context's later runs. Coordinate descent, each candidate run reps + 1 times (the
 * first discarded, median of the rest) with events between stages on the context's stream:
 * bin_occupancy in {0.35, 0.5, 0.7, 1, 2} on the whole sequence; then k2_warps in {4, 8} x k2_tma in {0, 1, 2}
 * on the neighbour search; then (k5_block, k5_regs, k5_ilp), k5_order and k5_blocks_per_sm on
 * chains + tracklets; then sel_lanes in {1, 32} on the selection. Results of the frames are those of any
 * shape. Blocks until done. Errors: TPC_E_INVAL
 * (bad list, reps < 1), TPC_E_STATE (a frame queued for serving), or any error tpc_track_batch
 * returns. */
int tpc_autotune(tpc_ctx* ctx, const tpc_frame_t* frames, int32_t n_frames, int32_t reps, tpc_tune_report* out);

/* Enable (1) or disable (0) per-kernel CUDA-event timing; read the last call's times (Sec. 7.2 times
 * the steps per GPU; these are the per-kernel times of this library's steps). */
int tpc_set_timing(tpc_ctx* ctx, int32_t enable);
int tpc_get_kernel_times(tpc_ctx* ctx, tpc_kernel_times* out);

/* ---- cluster finding from digits (Table 1 of Sec. 7.2 times it as the first GPU step of the
 * synchronous reconstruction; Sec. 2: the TPC records, per pad, the charge of every time bin, and a
 * pad row's clusters are reconstructed from these zero-suppressed digits). The paper names the step
 * but not its rules; the library computes:
 *   cells     row r has n_pads(r) = 2 ceil(x_r tan(10 deg) / pad_pitch) pads; pad k spans
 *             y in [(k - n_pads/2) pad_pitch, (k + 1 - n_pads/2) pad_pitch); time bin j spans
 *             w in [j time_bin_w, (j + 1) time_bin_w). q(s, r, k, j) = the charge of the digit in
 *             that cell, 0 where there is none or outside the row.
 *   peak      a digit c with q_c >= q_peak_min that beats each of its 8 neighbours n in the 3x3
 *             window: q_n < q_c, or q_n = q_c and n comes later in (time, pad) order (dj > 0, or
 *             dj = 0 and dk > 0); a plateau of equal charges has one peak, its first cell.
 *   cluster   the 3x3 window around a peak plus each cell of the surrounding 5x5 ring whose charge
 *             does not exceed that of the window cell next to it on the way to the peak (the +-2
 *             coordinates stepped one cell inwards); kept if Q = sum of charges >= q_total_min.
 *   values    from the integer sums Q, Sk = sum q dk, Sj = sum q dj, Skk = sum q dk^2,
 *             Sjj = sum q dj^2 (dk, dj relative to the peak), in FP32 with IEEE operations in this
 *             order: mk = Sk/Q, mj = Sj/Q; y = ((k + mk) - (n_pads/2 - 0.5)) * pad_pitch;
 *             w = ((j + mj) + 0.5) * time_bin_w; sigma_pad = sqrt(Skk/Q - mk*mk) (0 if not > 0),
 *             sigma_time likewise (in pads and time bins). */
typedef struct {
  double pad_pitch;     /* cm (default 0.4) */
  double time_bin_w;    /* cm of drift coordinate per time bin (default (250/90) * 0.2: 0.2 us) */
  int32_t q_peak_min;   /* default 3 */
  int32_t q_total_min;  /* default 10 */
} tpc_cf_params;

/* Digits of one time frame, structure of arrays in the caller's order (n entries each): at most one
 * digit per (sector, row, pad, time) cell, sector < 36, row < 152, pad < n_pads(row),
 * time < n_time, adc >= 1; anything else makes tpc_find_clusters return TPC_E_INVAL. */
typedef struct {
  const uint8_t* sector;
  const uint8_t* row;
  const uint16_t* pad;
  const uint16_t* time;
  const uint16_t* adc;
  int64_t n;            /* < 2^31 */
  int32_t n_time;       /* time bins of the frame, <= 65535 */
  int32_t on_device;    /* 1: device pointers (read during the call), 0: host memory */
} tpc_digits;

/* Clusters found in a frame's digits, in the input order of their peak digits. The arrays belong
 * to the context and stay valid until its next tpc_find_clusters() call or tpc_destroy(). With
 * on_device = 1 they are device arrays: (sector, row, y, w) can be passed as a tpc_clusters with
 * on_device = 1 to tpc_load_clusters(), which borrows them until the frame's tracking completes,
 * so track it before the next tpc_find_clusters() call. */
typedef struct {
  int64_t n_clusters;
  int32_t on_device;
  const uint8_t* sector;
  const uint8_t* row;
  const float* y;
  const float* w;
  const uint32_t* q_tot;
  const uint16_t* q_max;      /* the peak digit's charge */
  const float* sigma_pad;
  const float* sigma_time;
  const uint32_t* digit;      /* input index of the peak digit */
} tpc_cluster_list;

void tpc_cf_default_params(tpc_cf_params* p);

/* Find the clusters of one frame's digits (the kernels run on cuda_stream, NULL = the context's
 * stream; the call waits, bounded, for them). to_host = 1 returns page-locked host copies, 0 the
 * device arrays. The context keeps a charge map of 36 * 152 * (lines) * stride 16-bit cells
 * (stride = n_pads of the widest row + 4, rounded up to 16) in device memory between calls, within
 * half of the context's hbm_budget: lines = n_time + 4 when the whole frame fits, else the frame is
 * processed in time windows of as many bins as fit (lines = window + 4, two passes over the windows,
 * each window's map also holding the 2 time bins beyond each of its edges); the clusters are the
 * same, in the same order. TPC_E_BUDGET if not even a window of 16 time bins fits. Returns TPC_OK,
 * TPC_E_INVAL (bad parameters or digits, nothing written), TPC_E_BUDGET, TPC_E_NOMEM, TPC_E_TIMEOUT
 * or TPC_E_CUDA. */
int tpc_find_clusters(tpc_ctx* ctx, const tpc_cf_params* params, const tpc_digits* digits, int32_t to_host,
                      tpc_cluster_list* out, void* cuda_stream);

/* Per-kernel device time of the last tpc_find_clusters() call (with tpc_set_timing(ctx, 1)); in
 * time windows cf_fill holds the lists of each window's digit groups and the first pass (fill, peak
 * flags, clear), cf_copy the second (fill, clusters written to their slots, clear), and the launch
 * counts are 3 per window for each of them, 6 for cf_scan (the count scan and the three list
 * kernels) and 0 for cf_peaks and cf_clear. */
int tpc_get_cf_kernel_times(tpc_ctx* ctx, tpc_kernel_times* out);

/* Diagnostic of the kernels' bounded waits (no counterpart in the paper). Every device-side wait of
 * the library (the neighbour search waits on shared-memory barriers for its staging copies) gives
 * up after a time limit, records a timeout in a device status word and returns, so a lost copy
 * becomes TPC_E_TIMEOUT on the host instead of a hang. This call exercises that path: one warp
 * waits on a barrier whose announced transfer is never issued, with a limit of limit_us
 * microseconds of device time (1 .. 10^6). Returns TPC_E_TIMEOUT when the wait ran out (the
 * expected outcome), TPC_OK if it completed, TPC_E_INVAL for a limit out of range, TPC_E_CUDA on a
 * CUDA error. Nothing is left in flight; the device and every context stay usable. Runs on
 * cuda_stream (NULL: the legacy default stream) and waits for it. */
int tpc_check_wait_timeout(int32_t limit_us, void* cuda_stream);

/* Largest frame (clusters) that tpc_links_static() accepts. */
#define TPC_STATIC_MAX_CLUSTERS 262144

/* Cleaned neighbour links of one frame, computed without allocating any device memory. The paper
 * has no counterpart to this call; it exists for callers that cannot allocate device memory at the
 * moment they call: code running while another allocator (e.g. a framework's caching allocator)
 * owns the device's memory, code under a real-time or allocation-free rule (cudaMalloc/cudaFree
 * synchronise the device and may fail), or code that must not enter the allocator from where it
 * runs. It runs the search-grid, neighbour and cleaning kernels of tpc_track_sectors() on one frame,
 * with all of their scratch in one fixed-size array that is part of the library's device image
 * (about 17.9 MiB, held on every GPU that loads the library until the process exits), and writes the
 * same cleaned links that tpc_get_links(what = 2 / 3) returns after tracking the frame.
 *   p         method parameters (NULL: defaults); bin_occupancy below 1 is refused (TPC_E_CAPACITY)
 *   clusters  one frame, on_device = 1 (device pointers, caller-owned, read during the call)
 *   up, down  caller-owned device arrays of clusters->n int32: the input index of the linked
 *             cluster in the next / previous row, or -1
 *   cuda_stream  stream to run on (NULL: the legacy default stream)
 * Returns TPC_OK once the links are written (the call waits, at most two minutes, for its kernels),
 * TPC_E_CAPACITY if clusters->n > TPC_STATIC_MAX_CLUSTERS, TPC_E_INVAL for bad arguments or
 * malformed clusters, TPC_E_TIMEOUT, or TPC_E_CUDA. After TPC_E_TIMEOUT the call's kernels may still
 * be running and writing the scratch array and up/down: synchronise cuda_stream before freeing up or
 * down or making the next call. All calls share the one scratch array, which
 * keeps the previous call's contents (each call clears what must start at zero); calls that overlap
 * on the GPU, from two host threads or on two streams, race on it and must be serialised by the
 * caller. The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * creates its completion event; make that first call before any stream capture. */
int tpc_links_static(const tpc_params* p, const tpc_clusters* clusters, int32_t* up, int32_t* down,
                     void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TPCTRACK_H */
