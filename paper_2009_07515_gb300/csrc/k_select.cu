// k_select.cu — K6/K7 tracklet selection and K8 canonical output.
//
// Every hit goes to the tracklet with the largest key (nhits, then the smaller rank of the start
// hit) among the tracklets with >= nmin hits that contain it (atomicMax on a 32- or 64-bit word per
// hit, see Votes; keys are unique within a sector, so the outcome does not depend on atomic order). A
// tracklet becomes a track if it keeps >= nmin hits and at least half of its hits. Tracks are
// compacted by prefix sums in tracklet order, which is already canonical (frame, sector, rank of
// the start hit); each track's kept hits are written in ascending row order as input indices
// (k_kept clears the slab entries of the hits a tracklet lost, so the writer reads no vote words).
#include "tpc_dev.cuh"

namespace tpc {

__device__ __forceinline__ unsigned long long tl_key(uint32_t nh, uint32_t rank) {
  return ((unsigned long long)nh << 32) | (unsigned long long)(0xFFFFFFFFu - rank);
}

// The vote words of the hits: 32-bit keys nhits << 24 | (2^24 - 1 - rank) when every start-hit rank
// of the batch is below 2^24 (k_start_order sets cnt->wide_keys otherwise; nhits <= kNRow < 2^8),
// else the 64-bit keys of tl_key. Both order a sector's tracklets the same way (nhits, then the
// smaller rank), so they give the same selection; the 32-bit words halve the array the selection
// kernels gather from.
struct Votes {
  unsigned long long* w64;
  uint32_t* w32;
  bool narrow;
  __device__ explicit Votes(const Work& W)
      : w64(W.hit_w), w32(reinterpret_cast<uint32_t*>(W.hit_w)), narrow(W.cnt->wide_keys == 0u) {}
  __device__ __forceinline__ unsigned long long key(uint32_t nh, uint32_t rank) const {
    return narrow ? (unsigned long long)((nh << 24) | (0xFFFFFFu - rank)) : tl_key(nh, rank);
  }
  __device__ __forceinline__ void cast(uint32_t h, unsigned long long k) const {
    if (narrow) atomicMax(w32 + h, (uint32_t)k);
    else atomicMax(w64 + h, k);
  }
  __device__ __forceinline__ unsigned long long of(uint32_t h) const { return narrow ? (unsigned long long)w32[h] : w64[h]; }
};

// One warp per tracklet (grid-stride over tracklets): the lanes take the tracklet's rows 32 at a
// time, so the row loop's dependent loads (slab entry, then the hit's word) overlap across lanes;
// a tracklet's rows are consecutive slab words, so each pass reads one or two 128-byte lines. The
// selection kernels read (and k_kept clears) the slab with streaming cache hints: each slab line is
// used once per kernel, and evicting it first keeps the L2 for the vote and cluster words that the
// tracklets in flight share.
__device__ __forceinline__ uint32_t warp_global(int& lane) {
  lane = threadIdx.x & 31;
  return (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

__global__ void __launch_bounds__(256) k_votes_warp(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const Votes votes(W);
  int lane;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = warp_global(lane); t < ntl; t += nw) {
    const uint32_t info = W.tl_info[t];
    const uint32_t nh = info & 255u;
    if (!(info >> 24) || (int)nh < Q.nmin) continue;
    const unsigned long long key = votes.key(nh, W.starts[t].z);
    const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
    for (int r = ref + lane; r <= top; r += 32) {
      const uint32_t h = __ldcs(&W.slab[slab_at(t, r)]);
      if (h != kNoHit) votes.cast(h, key);
    }
  }
}

__global__ void __launch_bounds__(256) k_kept_warp(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const Votes votes(W);
  int lane;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = warp_global(lane); t < ntl; t += nw) {
    const uint32_t info = W.tl_info[t];
    const uint32_t nh = info & 255u;
    uint32_t acc = 0, kept = 0;
    if ((info >> 24) && (int)nh >= Q.nmin) {
      const unsigned long long key = votes.key(nh, W.starts[t].z);
      const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
      for (int r0 = ref; r0 <= top; r0 += 32) {
        const int r = r0 + lane;
        bool mine = false;
        if (r <= top) {
          const uint32_t h = __ldcs(&W.slab[slab_at(t, r)]);
          mine = h != kNoHit && votes.of(h) == key;
          if (h != kNoHit && !mine) __stcs(&W.slab[slab_at(t, r)], kNoHit);  // a hit the tracklet lost
        }
        kept += (uint32_t)__popc(__ballot_sync(0xffffffffu, mine));
      }
      acc = ((int)kept >= Q.nmin && 2u * kept >= nh) ? 1u : 0u;
    }
    if (lane == 0) {
      W.tl_kept[t] = acc;
      W.tl_nkept[t] = acc ? kept : 0u;
    }
  }
}

__global__ void __launch_bounds__(256) k_write_tracks_warp(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  int lane;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = warp_global(lane); t < ntl; t += nw) {
    const uint32_t k = W.tl_kept[t];
    if (W.tl_kept[t + 1] == k) continue;
    const uint32_t info = W.tl_info[t];
    const uint32_t nh = info & 255u;
    const uint4 st = W.starts[t];
    if (lane < 22) {
      const float v = W.tl_state[(long long)t * 24 + lane];
      if (lane < 5) W.tr_param[(long long)k * 5 + lane] = v;
      else if (lane < 20) W.tr_cov[(long long)k * 15 + (lane - 5)] = v;
      else if (lane == 20) W.tr_chi2[k] = v;
      else W.tr_xref[k] = v;
    }
    uint32_t off = W.tl_nkept[t];
    if (lane == 0) {
      W.tr_sector[k] = (int)((st.y % kSegPerFrame) / kNRow);
      W.tr_ndf[k] = 2 * (int)nh - 5;
      W.tr_hoff[k] = (long long)off;
    }
    // kept hits in ascending row order (k_kept left only them in the slab): ballot over each group
    // of 32 rows
    const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
    for (int r0 = ref; r0 <= top; r0 += 32) {
      const int r = r0 + lane;
      uint32_t h = kNoHit;
      if (r <= top) h = __ldcs(&W.slab[slab_at(t, r)]);
      const bool mine = h != kNoHit;
      const uint32_t m = __ballot_sync(0xffffffffu, mine);
      if (mine) W.tr_hits[off + (uint32_t)__popc(m & ((1u << lane) - 1u))] = W.horig[h];
      off += (uint32_t)__popc(m);
    }
  }
}

// One thread per tracklet, 32 consecutive tracklets per warp: the lanes walk the union of their
// row ranges together (a slab read of the warp touches one line per lane; the autotuner keeps
// this variant for frames where it measures faster).
struct RowRange {
  int lo, hi;  // warp-wide union of the lanes' [ref, top] (empty: lo > hi)
};
__device__ __forceinline__ RowRange warp_rows(bool on, int ref, int top) {
  int lo = on ? ref : kNRow, hi = on ? top : -1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  return RowRange{lo, hi};
}

__global__ void __launch_bounds__(256) k_votes_thread(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const Votes votes(W);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < ntl; t0 += stride) {
    const uint32_t t = t0 + (threadIdx.x & 31u);
    const uint32_t info = t < ntl ? W.tl_info[t] : 0u;
    const uint32_t nh = info & 255u;
    const bool on = (info >> 24) && (int)nh >= Q.nmin;
    const unsigned long long key = on ? votes.key(nh, W.starts[t].z) : 0ull;
    const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
    const RowRange rr = warp_rows(on, ref, top);
    for (int r = rr.lo; r <= rr.hi; ++r) {
      if (!on || r < ref || r > top) continue;
      const uint32_t h = __ldcs(&W.slab[slab_at(t, r)]);
      if (h != kNoHit) votes.cast(h, key);
    }
  }
}

__global__ void __launch_bounds__(256) k_kept_thread(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const Votes votes(W);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < ntl; t0 += stride) {
    const uint32_t t = t0 + (threadIdx.x & 31u);
    const uint32_t info = t < ntl ? W.tl_info[t] : 0u;
    const uint32_t nh = info & 255u;
    const bool on = (info >> 24) && (int)nh >= Q.nmin;
    const unsigned long long key = on ? votes.key(nh, W.starts[t].z) : 0ull;
    const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
    const RowRange rr = warp_rows(on, ref, top);
    uint32_t kept = 0;
    for (int r = rr.lo; r <= rr.hi; ++r) {
      if (!on || r < ref || r > top) continue;
      const uint32_t h = __ldcs(&W.slab[slab_at(t, r)]);
      if (h == kNoHit) continue;
      if (votes.of(h) == key) ++kept;
      else __stcs(&W.slab[slab_at(t, r)], kNoHit);  // a hit the tracklet lost
    }
    const uint32_t acc = (on && (int)kept >= Q.nmin && 2u * kept >= nh) ? 1u : 0u;
    if (t < ntl) {
      W.tl_kept[t] = acc;
      W.tl_nkept[t] = acc ? kept : 0u;
    }
  }
}

__global__ void __launch_bounds__(256) k_write_tracks_thread(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < ntl; t0 += stride) {
    const uint32_t t = t0 + (threadIdx.x & 31u);
    bool on = false;
    uint32_t k = 0;
    if (t < ntl) {
      k = W.tl_kept[t];
      on = W.tl_kept[t + 1] != k;
    }
    uint32_t info = 0, off = 0;
    if (on) {
      info = W.tl_info[t];
      const uint32_t nh = info & 255u;
      const uint4 st = W.starts[t];
      const float* src = W.tl_state + (long long)t * 24;
#pragma unroll
      for (int i = 0; i < 5; ++i) W.tr_param[(long long)k * 5 + i] = src[i];
#pragma unroll
      for (int i = 0; i < 15; ++i) W.tr_cov[(long long)k * 15 + i] = src[5 + i];
      W.tr_chi2[k] = src[20];
      W.tr_xref[k] = src[21];
      off = W.tl_nkept[t];
      W.tr_sector[k] = (int)((st.y % kSegPerFrame) / kNRow);
      W.tr_ndf[k] = 2 * (int)nh - 5;
      W.tr_hoff[k] = (long long)off;
    }
    const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
    const RowRange rr = warp_rows(on, ref, top);
    for (int r = rr.lo; r <= rr.hi; ++r) {
      if (!on || r < ref || r > top) continue;
      const uint32_t h = __ldcs(&W.slab[slab_at(t, r)]);  // k_kept left only the track's own hits
      if (h != kNoHit) W.tr_hits[off++] = W.horig[h];
    }
  }
}

// selection kernels of the chosen mode (lanes per tracklet: 32 or 1)
void launch_votes(int lanes, int grid, cudaStream_t s, const Work& W, const DevParams& Q) {
  if (lanes == 1) k_votes_thread<<<grid, 256, 0, s>>>(W, Q);
  else k_votes_warp<<<grid, 256, 0, s>>>(W, Q);
}
void launch_kept(int lanes, int grid, cudaStream_t s, const Work& W, const DevParams& Q) {
  if (lanes == 1) k_kept_thread<<<grid, 256, 0, s>>>(W, Q);
  else k_kept_warp<<<grid, 256, 0, s>>>(W, Q);
}
void launch_write_tracks(int lanes, int grid, cudaStream_t s, const Work& W, const DevParams& Q) {
  if (lanes == 1) k_write_tracks_thread<<<grid, 256, 0, s>>>(W, Q);
  else k_write_tracks_warp<<<grid, 256, 0, s>>>(W, Q);
}

// K10 compression inputs (Sec. 4: hits of good tracks are stored as residuals to the extrapolated
// track position; strategy B removes every hit not in the vicinity of a good track). One warp per
// track, its lanes on 32 rows at a time: the fit is transported (state only, no scattering) from
// x_ref directly to each row up to the last hit's row. At every row a good track (|q/pT| <=
// keep_qpt_max) protects the row's clusters within +-(keep_vy, keep_vw) of its prediction; each of
// its hits is stored as q(hit) - q(prediction), q(v) = rint(512 v), or as q(hit) from the first row
// whose transport fails on (n_pred counts the predicted hits).
__device__ __forceinline__ int32_t quant512(float v) { return (int32_t)rintf(v * 512.0f); }
template <bool kPacked>
__device__ __forceinline__ void mark_vicinity(const Work& W, const DevParams& Q, int g, float yp, float wp,
                                              long long off) {
  const GridWin q = grid_window(W.seg_bb, W.seg_dim, W.seg_geo, g, yp, wp, Q.keep_vy, Q.keep_vw);
  for (int cw = q.iw0; cw <= q.iw1; ++cw) {
    const uint32_t col = q.bb + (uint32_t)(cw * q.ny);
    const int base = col_base(q.cw0, q.cshift, cw);
    const int p1 = (int)W.bin_start[col + q.iy1 + 1];
    for (int p = (int)W.bin_start[col + q.iy0]; p < p1; ++p) {
      const float2 c = hit_in_col<kPacked>(W.hyw, W.hq, p, base);
      if (fabsf(c.y - wp) <= Q.keep_vw && fabsf(c.x - yp) <= Q.keep_vy) W.keep[off + W.horig[p]] = 1;
    }
  }
}
template <bool kPacked>
__global__ void __launch_bounds__(256) k_compress(Work W, DevParams Q) {
  const uint32_t ntl = W.cnt->n_tracklets;
  int lane;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = warp_global(lane); t < ntl; t += nw) {
    const uint32_t k = W.tl_kept[t];
    if (W.tl_kept[t + 1] == k) continue;
    const uint32_t info = W.tl_info[t];
    const uint4 st = W.starts[t];
    const int ref = (info >> 8) & 255, top = (info >> 16) & 255;
    const int g0 = (int)st.y, gb = g0 - (g0 % kSegPerFrame) % kNRow;
    const long long off = W.batch->f[g0 / kSegPerFrame].off;
    float P0[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) P0[i] = W.tl_state[(long long)t * 24 + i];
    const bool good = fabsf(P0[4]) <= Q.keep_qpt_max;
    const float x0 = row_x(Q, ref);
    // the last row with a hit of the track
    int last = -1;
    for (int c0 = ref; c0 <= top; c0 += 32) {
      const int r = c0 + lane;
      bool mine = false;
      if (r <= top) {
        const uint32_t h = W.slab[slab_at(t, r)];
        mine = h != kNoHit;  // k_kept left only the track's own hits
      }
      const uint32_t m = __ballot_sync(0xffffffffu, mine);
      if (m) last = c0 + 31 - __clz((int)m);
    }
    int32_t* res = W.tr_res + 2 * (long long)W.tl_nkept[t];
    uint32_t n = 0, np = 0;
    bool failed = false;  // a transport failed at an earlier row
    for (int c0 = ref; c0 <= last; c0 += 32) {
      const int r = c0 + lane;
      const bool in = r <= last;
      float P[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) P[i] = P0[i];
      bool ok = in && (r == ref || kf_propagate_state(Q, P, x0, row_x(Q, r)));
      // from the first failing row on, no row is predicted
      const uint32_t fail = __ballot_sync(0xffffffffu, in && !ok);
      if (failed || (fail & ((2u << lane) - 1u))) ok = false;
      if (ok && good) mark_vicinity<kPacked>(W, Q, gb + r, P[0], P[1], off);
      bool mine = false;
      uint32_t h = kNoHit;
      if (in) {
        h = W.slab[slab_at(t, r)];
        mine = h != kNoHit;  // k_kept left only the track's own hits
      }
      const uint32_t m = __ballot_sync(0xffffffffu, mine);
      if (mine) {
        if (good) W.keep[off + W.horig[h]] = 1;
        const float2 c = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, gb + r, (int)h);
        const uint32_t o = n + (uint32_t)__popc(m & ((1u << lane) - 1u));
        res[2 * o] = ok ? quant512(c.x) - quant512(P[0]) : quant512(c.x);
        res[2 * o + 1] = ok ? quant512(c.y) - quant512(P[1]) : quant512(c.y);
      }
      n += (uint32_t)__popc(m);
      np += (uint32_t)__popc(__ballot_sync(0xffffffffu, mine && ok));
      failed = failed || fail != 0u;
    }
    if (lane == 0) W.tr_npred[k] = (int32_t)np;
  }
}
void launch_compress(int packed, int grid, cudaStream_t s, const Work& W, const DevParams& Q) {
  if (packed) k_compress<true><<<grid, 256, 0, s>>>(W, Q);
  else k_compress<false><<<grid, 256, 0, s>>>(W, Q);
}

// K9 beam line (Sec. 6: track seeds are extrapolated to the beam line, and the most likely z is
// computed assuming a primary from a vertex at the origin). One thread per track: its fit at
// x_ref is transported by the exact helix step, without scattering noise, to the plane x = 0
// through the beam axis. Out: y0, w0, var(w0) there; for a primary from z = 0 (continuous
// readout: w = v_d t_c + L - |z|, so w0 = v_d t_c + L) the collision time t0 = (w0 - L) / v_d and
// the track's z at x_ref, +-(w0 - w_ref) by drift side (+ on side A); NaN where the transport
// fails.
__global__ void __launch_bounds__(256) k_beamline(Work W, DevParams Q) {
  const uint32_t ntr = W.cnt->n_tracks;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ntr; k += gridDim.x * blockDim.x) {
    float P[5], C[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) P[i] = W.tr_param[(long long)k * 5 + i];
#pragma unroll
    for (int i = 0; i < 15; ++i) C[i] = W.tr_cov[(long long)k * 15 + i];
    const float w_ref = P[1];
    float* o = W.tr_beam + (long long)k * 5;
    if (!kf_propagate(Q, P, C, W.tr_xref[k], 0.0f, false)) {
      const float nan = __int_as_float(0x7fc00000);
#pragma unroll
      for (int i = 0; i < 5; ++i) o[i] = nan;
      continue;
    }
    const float w0 = P[1];
    const float dz = w0 - w_ref;
    o[0] = P[0];
    o[1] = w0;
    o[2] = C[lt(1, 1)];
    o[3] = (w0 - Q.drift_len) / Q.vdrift;
    o[4] = W.tr_sector[k] < kNSec / 2 ? dz : -dz;
  }
}

// per frame: first tracklet, track and output hit of the frame
__global__ void k_frame_offsets(Work W) {
  const int nf = W.batch->nf;
  const uint32_t ntl = W.cnt->n_tracklets;
  for (int f = threadIdx.x; f <= nf; f += blockDim.x) {
    const uint32_t s = min(W.seg_nstart[f * kSegPerFrame], ntl);
    W.cnt->frame_start0[f] = s;
    W.cnt->frame_track0[f] = W.tl_kept[s];
    W.cnt->frame_hit0[f] = W.tl_nkept[s];
  }
}

// ------------------------------------------------------------------------------------ utilities
__global__ void k_reset_counters(Work W) {
  DevCounters* c = W.cnt;
  if (threadIdx.x == 0) {
    c->nseg = (uint32_t)(W.batch->nf * kSegPerFrame);
    c->ntot = (uint32_t)W.batch->ntot;
  }
  for (int i = threadIdx.x; i < kMaxFrames; i += blockDim.x) {
    c->wrange[2 * i] = 0xFFFFFFFFu;
    c->wrange[2 * i + 1] = 0u;
  }
  if (threadIdx.x == 0) {
    c->err = 0; c->n_starts = 0; c->n_tracklets = 0; c->k5_next = 0; c->n_bins = 0;
    c->seg_next[0] = 0; c->seg_next[1] = 0; c->seg_next[2] = 0; c->n_chunks = 0; c->k2_next = 0;
    c->n_sorted = 0; c->n_tracks = 0; c->n_track_hits = 0; c->n_steps = 0; c->n_tracklet_hits = 0;
    c->wide_keys = W.wide_votes ? 1u : 0u;
  }
}

// zero (*n_dev + add) * mul 32-bit words, at most n_cap (or n_cap words when n_dev is null)
__global__ void k_zero_u32(uint32_t* p, const uint32_t* n_dev, long long n_cap, int add, int mul) {
  long long n = n_dev ? ((long long)*n_dev + add) * mul : n_cap;
  if (n > n_cap) n = n_cap;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = 0u;
}

__global__ void k_set_ntracklets(Work W) {
  if (threadIdx.x == 0) W.cnt->n_tracklets = min(W.cnt->n_starts, (uint32_t)W.tcap);
}

// per-cluster link arrays of frame f in the caller's index order (debug / parity)
__global__ void k_links_to_input(Work W, int f, int what, int32_t* out) {
  const uint32_t p0 = W.bin_start[W.seg_bb[f * kSegPerFrame]];
  const uint32_t p1 = W.bin_start[W.seg_bb[(f + 1) * kSegPerFrame]];
  const int2* L = what < 2 ? W.links : W.clinks;
  for (uint32_t p = p0 + blockIdx.x * blockDim.x + threadIdx.x; p < p1; p += gridDim.x * blockDim.x) {
    const int2 l = L[p];
    const int v = (what & 1) ? l.x : l.y;
    out[W.horig[p]] = v >= 0 ? (int32_t)W.horig[v] : -1;
  }
}

}  // namespace tpc
