// tpc_dev.cuh — device-side definitions shared by the tracking kernels (sm_103a).
//
// Layout of one batch in HBM (all frames of a batch share one workspace; every array is indexed by
// a batch-global "sorted position" p of a cluster after the grid build):
//   hyw[p]      float2 (y, w) of the cluster at sorted position p (FP32 storage), or
//   hq[p]       uint32 (qy | qw << 16) in the 16-bit storage: y = qy/512 - 64 and w = (column base +
//               qw)/512, qw the offset in 2^-9 cm from the lower edge of the cluster's grid column;
//               hcol[p] (uint16) that column, for reads by position
//   horig[p]    uint32 index of the cluster in its frame's input arrays
//   segments    g = frame*5472 + sector*152 + row; seg_bb[g] = first bin, seg_dim[g] = (nw, ny,
//               iw0, k + 9), seg_geo[g] = (w_lo, w-bins per cm, y_lo, y-bins per cm) of the
//               segment's 2-D grid over the drift coordinate w and the pad-row coordinate y;
//               bin = iw * ny + iy; w-columns have width 2^k cm (-3 <= k <= 7) and are aligned to
//               multiples of it (column iw starts at (iw0 + iw) * 2^k cm)
//   bin_start[b] sorted position of the first cluster of bin b (exclusive prefix over all bins), so
//               a w-column (all y of one w bin) is one contiguous position range, and a window is
//               one contiguous range per w-column it touches
//   links[p]    int2 (down, up) raw neighbour links; clinks[p] the cleaned (reciprocal) links
//   starts[t]   start hits in canonical order (frame, sector, row-rank)
//   slab        sorted position of tracklet t's hit in row r (0xFFFFFFFF: none), written for rows
//               [ref_row, top_row]; tracklet-major (slab_at): a lane's stores over successive row
//               steps fill consecutive words, so a 32-byte sector is completed by one lane rather
//               than by partial writes of eight tracklets, and a warp reads a tracklet's rows
//               coalesced
//
// The Kalman arithmetic below is written so that every float result is the same sequence of
// correctly rounded operations as the method's plain definition (compiled with -fmad=false, IEEE
// division and square root, explicit fused multiply-adds where the definition accumulates a sum of
// products): products with exact zeros and ones of the Jacobian and of I - KH are skipped, the
// remaining terms are accumulated in the same order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tpc {

constexpr int kNSec = 36;
constexpr int kNRow = 152;
constexpr int kSegPerFrame = kNSec * kNRow;  // 5472
constexpr int kMaxFrames = 64;               // frames per batched launch
constexpr int kHistThreads = 1024;           // threads per block of the segment histogram
constexpr uint32_t kNoHit = 0xFFFFFFFFu;
constexpr int kMergeBins = 2048;             // w bins per (frame, sector) of the merge step's search
// batches of more clusters than this are placed into grid order in two passes per segment (their
// grid and cluster arrays outgrow the L2); smaller ones in one pass
constexpr long long kTwoPassMin = 1LL << 23;
constexpr int kScatterParts = 4;             // blocks that share one segment in the second pass
constexpr int kSegUnroll = 4;                // records a thread has in flight in the per-segment passes

// error bits (device error word)
constexpr uint32_t kErrInput = 1u;      // malformed cluster (sector/row range, non-finite)
constexpr uint32_t kErrTracklets = 2u;  // tracklet capacity exceeded
constexpr uint32_t kErrBins = 4u;       // bin capacity exceeded
constexpr uint32_t kErrTimeout = 8u;    // bounded mbarrier wait expired
constexpr uint32_t kErrTracks = 16u;    // output hit capacity exceeded

struct DevParams {
  float kq;                      // d(curvature)/d(q/pT)
  float chi_n_max;
  int lmin;
  float r00, r11;                // measurement variances
  float chi2_max;
  int n_miss_max;
  float win_nsig, win_add;
  int ms_on;
  float x0_row, ms_c, mass2;
  float max_sin, y_margin, tan10;
  int nmin;
  int ext_stop;
  float drift_len, vdrift;       // L (cm) and v_d (cm/us) of the continuous-readout drift coordinate
  float keep_vy, keep_vw;        // strategy-B vicinity of a good track's prediction (cm)
  float keep_qpt_max;            // good track: |q/pT| <= this
  float cov0[5];
  // K12 merging and refit
  int merge_gap_rows;            // the outer segment starts 1 .. this many rows above the inner one
  float merge_dw;                // |w difference| of a candidate pair (cm)
  float merge_chi2_max;          // 5-parameter chi2 cut of a merge
  float rot_c, rot_s;            // cos and sin of the 20-degree angle between neighbouring sectors
  float refit_scale;             // a refit pass starts from the previous covariance times this
  int refit_passes;              // refit passes, alternately inward and outward
  float occ;                     // target clusters per grid bin
  float aspect;                  // w/y extent of a grid bin (the neighbour window's aspect)
  float x[kNRow];                // row radii
  float pitch;                   // row pitch (float)160 / (float)151
  // neighbour windows per row r (valid for 1 <= r <= 150)
  float wy_dn[kNRow], ww_dn[kNRow], wy_up[kNRow], ww_up[kNRow], f_mid[kNRow];
  float yext[kNRow];             // half extent of the grid in y: x * tan(10 deg) + 1 cm
};

struct FrameIn {
  const uint8_t* sector;
  const uint8_t* row;
  const float* y;
  const float* w;
  long long n;
  long long off;  // first batch-global input index of this frame
};

struct BatchDesc {
  int nf;
  int pad_;
  long long ntot;
  FrameIn f[kMaxFrames];
};

// Counters and per-batch scalars in device memory (zeroed at the start of each run).
struct DevCounters {
  uint32_t nseg;          // frames * 5472 (from the batch descriptor)
  uint32_t ntot;          // clusters of the batch
  uint32_t err;
  uint32_t n_starts;      // start hits found (may exceed tcap: overflow)
  uint32_t n_tracklets;   // min(n_starts, tcap)
  uint32_t k5_next;       // work counter of the tracklet kernel
  uint32_t wide_keys;     // non-zero: a start-hit rank of the batch is >= 2^24 (64-bit vote keys)
  uint32_t seg_next[3];   // segment work counters of the neighbour, cleaning and start kernels
  uint32_t n_chunks;      // 32-hit chunks of the neighbour kernel
  uint32_t k2_next;       // chunk work counter of the neighbour kernel
  uint32_t n_bins;        // total bins of the batch
  uint32_t n_bins_1p;     // bins the one-pass placement zeroes and scans: n_bins, or 0 when the
                          // per-segment passes place the batch (they zero and scan each segment's bins)
  uint32_t scan_sink;     // total of a scan whose total is already known
  uint32_t n_sorted;      // clusters placed in the grid
  uint32_t n_tracks;
  uint32_t n_track_hits;
  unsigned long long n_steps;         // tracklet row steps (propagations + candidate checks)
  unsigned long long n_tracklet_hits; // hits fitted by all tracklets
  uint32_t wrange[2 * kMaxFrames];  // per frame (min, max) of w, order-preserving encoding
  uint32_t frame_start0[kMaxFrames + 1];  // first start index of each frame
  uint32_t frame_track0[kMaxFrames + 1];  // first track index of each frame
  uint32_t frame_hit0[kMaxFrames + 1];    // first output hit of each frame
  uint32_t n_merged;                      // K12: merged tracks (chains) of the batch
  uint32_t n_merged_hits;
  uint32_t n_merge_bins;                  // K12: tracks placed in the search bins
  uint32_t frame_merged0[kMaxFrames + 1]; // first merged track of each frame
  uint32_t frame_mhit0[kMaxFrames + 1];   // first merged hit of each frame
};

// Workspace pointers (device arrays), sized by capacities.
struct Work {
  DevCounters* cnt;
  const BatchDesc* batch;
  // grid
  uint32_t* seg_cnt;     // [scap]
  uint32_t* seg_nb;      // [scap]  bins of the segment (nw * ny), scanned into seg_bb
  uint32_t* seg_bb;      // [scap + 1]
  int4* seg_dim;         // [scap] (nw, ny, iw0, k + 9)
  float4* seg_geo;       // [scap] (w_lo, w-bins per cm, y_lo, y-bins per cm)
  uint32_t* bin_start;   // [bcap + 1]
  uint32_t* rank;        // [ncap] rank of each record in its bin (two-pass placement)
  uint32_t* seg_start;   // [scap + 1] exclusive scan of seg_cnt: first record of each segment
  uint32_t* seg_cur;     // [scap] append cursor of each segment
  uint4* rec;            // [ncap] (y, w, batch index, segment) in segment order
  float2* hyw;           // [ncap + 2] FP32 storage
  uint32_t* hq;          // [ncap + 4] 16-bit storage
  uint16_t* hcol;        // [ncap]     16-bit storage: grid column of each position
  uint32_t* horig;       // [ncap]
  // links
  uint32_t* k2_off;      // [scap + 1] 32-hit chunks of every segment work item, scanned
  uint2* k2_tab;         // [k2cap] (segment, first position) of every chunk, in work-item order
  int2* links;           // [ncap]
  int2* clinks;          // [ncap]
  uint8_t* is_start;     // [ncap] 1 at the start hit of a tracklet
  uint32_t* seg_nstart;  // [scap + 1] -> scanned
  uint4* starts_raw;     // [tcap] (hit, seg, first bin of its w-column, -)
  uint4* starts;         // [tcap] (hit, seg, rank-in-sector, -)
  int4* chains;          // [tcap] (middle hit, last hit, chain length, -)
  uint32_t* order;       // [tcap] processing order of the tracklet kernel (longest chain first)
  uint32_t* len_cnt;     // [kNRow + 1] chain-length histogram, then bucket cursors
  // tracklets
  float* tl_state;       // [tcap][24]: P[5], C[15], chi2, x_ref, -, -
  uint32_t* tl_info;     // [tcap]: nhits | ref_row << 8 | top_row << 16 | ok << 24
  uint32_t* slab;        // [tcap][kNRow] (slab_at)
  unsigned long long* hit_w;  // [ncap]
  uint32_t* tl_kept;     // [tcap + 1] -> scanned (track index)
  uint32_t* tl_nkept;    // [tcap + 1] -> scanned (hit offset)
  // tracks, in the layout of the host's output arrays (each copied to the host as one block)
  float* tr_param;       // [tcap][5] fit state at x_ref
  float* tr_cov;         // [tcap][15] its covariance (lower triangle)
  float* tr_chi2;        // [tcap]
  float* tr_xref;        // [tcap]
  int32_t* tr_sector;    // [tcap]
  int32_t* tr_ndf;       // [tcap]
  long long* tr_hoff;    // [tcap] first output hit of the track in the batch's hit list
  float* tr_beam;        // [tcap][5] beam-line extrapolation (K9)
  int32_t* tr_res;       // [ncap][2] compression residuals of the output hits (K10; null: off)
  int32_t* tr_npred;     // [tcap] output hits stored as residuals (K10)
  uint8_t* keep;         // [ncap] strategy-B protection per batch input index (K10)
  uint32_t* tr_hits;     // [ncap] output hits (frame-local input indices)
  // K12 merging and refit (null when off)
  float* m_state;        // [tcap][20] outer state: P[5], C[15] at the last hit's row
  uint32_t* m_info;      // [tcap] last_row | ref_row << 8 | outer state ok << 16 | frame << 17
  uint32_t* m_bin;       // [mbcap + 1] tracks per (frame, sector, w bin) -> scanned -> bin ends
  uint32_t* m_list;      // [tcap] tracks in bin order
  unsigned long long* m_bestA;  // [tcap] best inner partner of each track: chi2 bits << 32 | index
  unsigned long long* m_bestB;  // [tcap] best outer partner of each track: chi2 bits << 32 | index
  float* m_chi;          // [tcap] its chi2
  int32_t* m_next;       // [tcap] linked outer partner, -1 if none
  uint32_t* m_prev;      // [tcap] 1 if linked from an inner partner
  uint32_t* m_hidx;      // [tcap + 1] chain head flags -> scanned -> merged index
  uint32_t* m_hoff;      // [tcap + 1] chain hit counts -> scanned -> first merged hit
  float* mt_param;       // [tcap][5] refit state at x_ref
  float* mt_cov;         // [tcap][15]
  float* mt_chi2;        // [tcap]
  float* mt_xref;        // [tcap]
  int32_t* mt_sector;    // [tcap] frame of the refit result
  int32_t* mt_ndf;       // [tcap]
  int32_t* mt_nfit;      // [tcap]
  int32_t* mt_nseg;      // [tcap]
  int32_t* mt_head;      // [tcap] frame-local sector-track index of the innermost segment
  long long* mt_hoff;    // [tcap] first merged hit
  uint32_t* mt_hits;     // [ncap] frame-local input indices, inner segment first
  int32_t* tr_next;      // [tcap] frame-local outer partner of each sector track, -1 if none
  float* tr_mchi2;       // [tcap] chi2 of that merge, NaN if none
  long long mbcap;       // search bins (frames x sectors x kMergeBins)
  // scan scratch
  uint32_t* scan_tmp;    // [scan_tmp_cap]
  long long ncap, scap, bcap, tcap, scan_tmp_cap, k2cap;
  int packed;            // 1: 16-bit cluster storage (hq, hcol), 0: FP32 (hyw)
  int wide_votes;        // 1: 64-bit vote keys whatever the ranks (tpc_params.wide_votes)
};

// ------------------------------------------------------------------------------------ helpers
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// bin of v along one grid axis with nb bins starting at lo, inv bins per cm (monotone in v)
__device__ __forceinline__ int bin_of(float v, float lo, float inv, int nb) {
  float t = (v - lo) * inv;
  if (!(t > 0.f)) return 0;
  if (t >= (float)nb) return nb - 1;
  return (int)t;
}

// Window of a segment grid: w-columns [iw0, iw1], y-bins [iy0, iy1], for |w - wc| <= Ww and
// |y - yc| <= Wy (widened by a hair: the exact window test is done on the coordinates).
struct GridWin {
  int iw0, iw1, iy0, iy1, ny, cw0, cshift;  // cw0, cshift: column base of iw = (cw0 + iw) << cshift
  uint32_t bb;
};
__device__ __forceinline__ float win_pad(float c, float W);
__device__ __forceinline__ GridWin grid_window_from(const int4 dim, const float4 geo, uint32_t bb, float yc, float wc,
                                                    float Wy, float Ww) {
  GridWin q;
  q.bb = bb;
  q.ny = dim.y;
  q.cw0 = dim.z;
  q.cshift = dim.w;
  const float pw = win_pad(wc, Ww), py = win_pad(yc, Wy);
  q.iw0 = bin_of((wc - Ww) - pw, geo.x, geo.y, (int)dim.x);
  q.iw1 = bin_of((wc + Ww) + pw, geo.x, geo.y, (int)dim.x);
  q.iy0 = bin_of((yc - Wy) - py, geo.z, geo.w, (int)dim.y);
  q.iy1 = bin_of((yc + Wy) + py, geo.z, geo.w, (int)dim.y);
  return q;
}
__device__ __forceinline__ GridWin grid_window(const uint32_t* seg_bb, const int4* seg_dim, const float4* seg_geo,
                                               int g, float yc, float wc, float Wy, float Ww) {
  return grid_window_from(seg_dim[g], seg_geo[g], seg_bb[g], yc, wc, Wy, Ww);
}

// conservative widening of a window for the bin lookup (rounding of w +- W)
__device__ __forceinline__ float win_pad(float wc, float W) {
  return fabsf(wc) * 1.0e-6f + W * 1.0e-6f + 1.0e-6f;
}

// ---- 16-bit storage. Column base in units of 2^-9 cm; y = qy/512 - 64, w = (base + qw)/512: both
// exact floats for |w| < 32768 cm, equal to rint(512 w)/512 whatever the column.
__device__ __forceinline__ int col_base(int cw0, int cshift, int iw) { return (cw0 + iw) * (1 << cshift); }
__device__ __forceinline__ float2 unpack_hit(uint32_t q, int base) {
  return make_float2((float)(q & 0xFFFFu) * (1.0f / 512.0f) - 64.0f, (float)(base + (int)(q >> 16)) * (1.0f / 512.0f));
}
// (y, w) of position p whose column base is known
template <bool kPacked>
__device__ __forceinline__ float2 hit_in_col(const float2* hyw, const uint32_t* hq, int p, int base) {
  if (kPacked) return unpack_hit(hq[p], base);
  return hyw[p];
}
// (y, w) of position p of segment g (reads the column of p in the 16-bit storage)
template <bool kPacked>
__device__ __forceinline__ float2 hit_by_index(const float2* hyw, const uint32_t* hq, const uint16_t* hcol,
                                               const int4* seg_dim, int g, int p) {
  if (kPacked) {
    const int4 d = seg_dim[g];
    return unpack_hit(hq[p], col_base(d.z, d.w, (int)hcol[p]));
  }
  return hyw[p];
}

// row-order key comparison: (w, y, input index) lexicographic
__device__ __forceinline__ bool key_less(float wa, float ya, uint32_t oa, float wb, float yb, uint32_t ob) {
  if (wa < wb) return true;
  if (wa > wb) return false;
  if (ya < yb) return true;
  if (ya > yb) return false;
  return oa < ob;
}

// Segment work item k -> segment: rows 1..150 first, inner (denser) rows first, all sectors and
// frames of a row together; the boundary rows 0 and 151 last.
__device__ __forceinline__ int segment_of_item(int k, int nf) {
  const int per_row = nf * kNSec;
  int ri = k / per_row;
  const int rest = k - ri * per_row;
  const int f = rest / kNSec, sec = rest - f * kNSec;
  const int r = ri < kNRow - 2 ? ri + 1 : (ri == kNRow - 2 ? 0 : kNRow - 1);
  return f * kSegPerFrame + sec * kNRow + r;
}

// Dynamic segment assignment: thread 0 of the block takes the next work item.
__device__ __forceinline__ int next_segment(uint32_t* counter, int nf, int* s_item) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  const int k = *s_item;
  return k < nf * kSegPerFrame ? segment_of_item(k, nf) : -1;
}

__device__ __forceinline__ int frame_of(const BatchDesc* B, long long i) {
  int lo = 0, hi = B->nf - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (B->f[mid].off <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------------------ KF math
// asin(t): half-angle reduction t -> t / sqrt(2 (1 + sqrt(1 - t^2))) until |t| < 0.1, then the
// Maclaurin series of asin(t)/t to t^10 (only correctly rounded operations, no library call)
__device__ __forceinline__ float asin_series_ratio(float t) {  // Horner with fused multiply-adds
  const float t2 = t * t;
  float p = (float)0.022372159090909092;
  p = __fmaf_rn(t2, p, (float)0.030381944444444444);
  p = __fmaf_rn(t2, p, (float)0.044642857142857144);
  p = __fmaf_rn(t2, p, (float)0.075);
  p = __fmaf_rn(t2, p, (float)0.16666666666666666);
  return __fmaf_rn(t2, p, 1.0f);
}
__device__ __forceinline__ float asin_hr(float t) {
  float scale = 1.0f;
  for (int it = 0; it < 40 && fabsf(t) >= (float)0.1; ++it) {
    t = t / sqrtf(2.0f * (1.0f + sqrtf(1.0f - t * t)));
    scale = scale * 2.0f;
  }
  return scale * t * asin_series_ratio(t);
}
__device__ __forceinline__ float arc_ratio(float t) {
  if (fabsf(t) < (float)0.1) return asin_series_ratio(t);
  return asin_hr(t) / t;
}
__device__ __forceinline__ float arc_ratio_deriv(float t) {
  if (fabsf(t) < (float)0.1) {
    const float t2 = t * t;
    float p = (float)0.22372159090909091;
    p = __fmaf_rn(t2, p, (float)0.24305555555555555);
    p = __fmaf_rn(t2, p, (float)0.26785714285714285);
    p = __fmaf_rn(t2, p, (float)0.3);
    p = __fmaf_rn(t2, p, (float)0.3333333333333333);
    return t * p;
  }
  return (1.0f / sqrtf(1.0f - t * t) - arc_ratio(t)) / t;
}

// slab index of tracklet t, row r: kNRow consecutive words per tracklet
__host__ __device__ __forceinline__ long long slab_at(uint32_t t, int r) {
  return (long long)t * kNRow + r;
}

// lower-triangular packed covariance index
__host__ __device__ constexpr int lt(int i, int k) { return i >= k ? i * (i + 1) / 2 + k : k * (k + 1) / 2 + i; }

// Exact helix transport with scattering noise. Returns false if |sin(phi)| would reach max_sin.
__device__ __forceinline__ bool kf_propagate(const DevParams& Q, float* P, float* C, float x0, float x1,
                                             bool scatter = true) {
  const float dx = x1 - x0;
  const float k = Q.kq * P[4];
  const float s0 = P[2];
  const float s1 = s0 + k * dx;
  if (!(fabsf(s1) < Q.max_sin)) return false;
  const float c0 = sqrtf(1.0f - s0 * s0);
  const float c1 = sqrtf(1.0f - s1 * s1);
  const float N = s0 + s1, D = c0 + c1;
  const float iD = 1.0f / D;
  const float dy = dx * (N * iD);
  const float l = sqrtf(dx * dx + dy * dy);
  const float t = l * k * 0.5f;
  float a = l * arc_ratio(t);
  if (dx < 0.f) a = -a;
  const float tw = P[3];
  const float ic0 = 1.0f / c0, ic1 = 1.0f / c1, il = 1.0f / l;
  const float iDD = iD * iD;
  const float dy_ds0 = dx * (2.0f * iD + N * (s0 * ic0 + s1 * ic1) * iDD);
  const float dy_dk = dx * dx * (iD + N * s1 * ic1 * iDD);
  float da_dl = 1.0f / sqrtf(1.0f - t * t);
  float da_dk = l * l * 0.5f * arc_ratio_deriv(t);
  if (dx < 0.f) { da_dl = -da_dl; da_dk = -da_dk; }
  const float dl_ds0 = dy * dy_ds0 * il;
  const float dl_dk = dy * dy_dk * il;
  const float J02 = dy_ds0;
  const float J04 = dy_dk * Q.kq;
  const float J12 = tw * (da_dl * dl_ds0);
  const float J13 = a;
  const float J14 = tw * (da_dl * dl_dk + da_dk) * Q.kq;
  const float J24 = dx * Q.kq;
  P[0] = P[0] + dy;
  P[1] = P[1] + tw * a;
  P[2] = s1;
  // T = J C: the nonzero terms of the index-ordered fused multiply-add sums of the dense product
  float T[5][5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    T[0][c] = __fmaf_rn(J04, C[lt(4, c)], __fmaf_rn(J02, C[lt(2, c)], C[lt(0, c)]));
    T[1][c] = __fmaf_rn(J14, C[lt(4, c)], __fmaf_rn(J13, C[lt(3, c)], __fmaf_rn(J12, C[lt(2, c)], C[lt(1, c)])));
    T[2][c] = __fmaf_rn(J24, C[lt(4, c)], C[lt(2, c)]);
    T[3][c] = C[lt(3, c)];
    T[4][c] = C[lt(4, c)];
  }
  // O = T J^T (lower triangle)
  float O[15];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    O[lt(i, 0)] = __fmaf_rn(T[i][4], J04, __fmaf_rn(T[i][2], J02, T[i][0]));
    if (i >= 1) O[lt(i, 1)] = __fmaf_rn(T[i][4], J14, __fmaf_rn(T[i][3], J13, __fmaf_rn(T[i][2], J12, T[i][1])));
    if (i >= 2) O[lt(i, 2)] = __fmaf_rn(T[i][4], J24, T[i][2]);
    if (i >= 3) O[lt(i, 3)] = T[i][3];
    if (i >= 4) O[lt(i, 4)] = T[i][4];
  }
  if (scatter && Q.ms_on && P[4] != 0.f) {
    const float one_tw2 = 1.0f + tw * tw;
    const float pathf = sqrtf(one_tw2) * ic1;
    const float xx0 = Q.x0_row * pathf;
    const float q2 = P[4] * P[4] / one_tw2;
    const float th2 = Q.ms_c * xx0 * q2 * (1.0f + Q.mass2 * q2);
    O[lt(2, 2)] = O[lt(2, 2)] + th2 * (c1 * c1) * one_tw2;
    O[lt(3, 3)] = O[lt(3, 3)] + th2 * one_tw2 * one_tw2;
  }
#pragma unroll
  for (int i = 0; i < 15; ++i) C[i] = O[i];
  return true;
}

// row radius x_r = 85 + r * (160/151) cm, evaluated with the same two rounded float operations as
// the host table (a per-lane row index into a parameter table would serialise the warp's loads)
__device__ __forceinline__ float row_x(const DevParams& Q, int r) {
  return __fadd_rn(85.0f, __fmul_rn((float)r, Q.pitch));
}

// The state part of kf_propagate alone, the same operations (the compression step's predictions).
__device__ __forceinline__ bool kf_propagate_state(const DevParams& Q, float* P, float x0, float x1) {
  const float dx = x1 - x0;
  const float k = Q.kq * P[4];
  const float s0 = P[2];
  const float s1 = s0 + k * dx;
  if (!(fabsf(s1) < Q.max_sin)) return false;
  const float c0 = sqrtf(1.0f - s0 * s0);
  const float c1 = sqrtf(1.0f - s1 * s1);
  const float N = s0 + s1, D = c0 + c1;
  const float iD = 1.0f / D;
  const float dy = dx * (N * iD);
  const float l = sqrtf(dx * dx + dy * dy);
  const float t = l * k * 0.5f;
  float a = l * arc_ratio(t);
  if (dx < 0.f) a = -a;
  P[0] = P[0] + dy;
  P[1] = P[1] + P[3] * a;
  P[2] = s1;
  return true;
}

// Inverse of the residual covariance S = H C H^T + R of the current state; pd: det S > 0. The chi2
// of every candidate of a row and the update use the same inverse (the same operations as
// computing it for each of them).
struct SInv {
  float i00, i01, i10, i11;
  bool pd;
};
__device__ __forceinline__ SInv kf_sinv(const DevParams& Q, const float* C) {
  const float S00 = C[0] + Q.r00, S01 = C[1], S10 = C[1], S11 = C[2] + Q.r11;
  const float det = S00 * S11 - S01 * S10;
  const float idet = 1.0f / det;
  return SInv{S11 * idet, -S01 * idet, -S10 * idet, S00 * idet, det > 0.f};
}
// chi2 of a measurement (ym, wm): +inf when S is not positive definite
__device__ __forceinline__ float kf_chi2(const SInv& V, const float* P, float ym, float wm) {
  if (!V.pd) return __int_as_float(0x7f800000);
  const float r0 = ym - P[0], r1 = wm - P[1];
  const float u0 = __fmaf_rn(V.i01, r1, V.i00 * r0), u1 = __fmaf_rn(V.i11, r1, V.i10 * r0);
  return __fmaf_rn(r1, u1, r0 * u0);
}

__device__ __forceinline__ void kf_update(const DevParams& Q, const SInv& V, float* P, float* C, float ym, float wm) {
  const float i00 = V.i00, i01 = V.i01, i10 = V.i10, i11 = V.i11;
  float K[5][2];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float ci0 = C[lt(i, 0)], ci1 = C[lt(i, 1)];
    K[i][0] = __fmaf_rn(ci1, i10, ci0 * i00);
    K[i][1] = __fmaf_rn(ci1, i11, ci0 * i01);
  }
  const float r0 = ym - P[0], r1 = wm - P[1];
#pragma unroll
  for (int i = 0; i < 5; ++i) P[i] = P[i] + __fmaf_rn(K[i][1], r1, K[i][0] * r0);
  // A = I - K H: only the first two columns differ from the identity
  float A[5][2];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    A[i][0] = (i == 0 ? 1.0f : 0.0f) - K[i][0];
    A[i][1] = (i == 1 ? 1.0f : 0.0f) - K[i][1];
  }
  // T = A C: rows i, columns 0, 1 and (for i >= 2) the diagonal-block column k <= i
  float T0[5], T1[5], Tk[15];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    T0[i] = __fmaf_rn(A[i][1], C[lt(1, 0)], A[i][0] * C[lt(0, 0)]);
    T1[i] = __fmaf_rn(A[i][1], C[lt(1, 1)], A[i][0] * C[lt(0, 1)]);
    if (i >= 2) {
      T0[i] = T0[i] + C[lt(i, 0)];
      T1[i] = T1[i] + C[lt(i, 1)];
    }
  }
#pragma unroll
  for (int i = 2; i < 5; ++i)
#pragma unroll
    for (int k = 2; k <= i; ++k) Tk[lt(i, k)] = __fmaf_rn(A[i][1], C[lt(1, k)], A[i][0] * C[lt(0, k)]) + C[lt(i, k)];
  float KR[5][2];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    KR[i][0] = K[i][0] * Q.r00;
    KR[i][1] = K[i][1] * Q.r11;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int k = 0; k <= i; ++k) {
      float o = __fmaf_rn(T1[i], A[k][1], T0[i] * A[k][0]);
      if (k >= 2) o = o + Tk[lt(i, k)];
      C[lt(i, k)] = o + __fmaf_rn(KR[i][1], K[k][1], KR[i][0] * K[k][0]);
    }
}

// Seed from the first, middle and last chain hits (x, y, w): circle through them in (x, y), state
// at the first hit, dw/ds from the end points over the arc.
__device__ __forceinline__ bool kf_seed(const DevParams& Q, const float h[3][3], float* P) {
  const float ax = h[1][0] - h[0][0], ay = h[1][1] - h[0][1];
  const float bx = h[2][0] - h[0][0], by = h[2][1] - h[0][1];
  const float cx = h[2][0] - h[1][0], cy = h[2][1] - h[1][1];
  const float cross = ax * by - ay * bx;
  const float d01 = sqrtf(ax * ax + ay * ay);
  const float d02 = sqrtf(bx * bx + by * by);
  const float d12 = sqrtf(cx * cx + cy * cy);
  const float k = 2.0f * cross / (d01 * d02 * d12);
  const float sg = k * d02 * 0.5f;
  if (!(fabsf(sg) < 1.0f)) return false;
  const float cg = sqrtf(1.0f - sg * sg);
  const float sphi = (by * cg - bx * sg) / d02;
  if (!(fabsf(sphi) < Q.max_sin)) return false;
  const float arc = d02 * arc_ratio(sg);
  P[0] = h[0][1];
  P[1] = h[0][2];
  P[2] = sphi;
  P[3] = (h[2][2] - h[0][2]) / arc;
  P[4] = Q.kq != 0.f ? k / Q.kq : 0.0f;
  return true;
}

}  // namespace tpc
