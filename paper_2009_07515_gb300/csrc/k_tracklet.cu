// k_tracklet.cu — K5 tracklet construction (helix Kalman filter in the solenoid field).
//
// k_chains walks each start hit's cleaned chain once (length, middle and last hit) and writes the
// chain's hits into the tracklet's slab rows, so the tracklet kernel seeds and follows the chain
// without pointer chasing (the outward chain steps read slab rows at known addresses, like the
// inward refit).
//
// k_tracklets: one lane builds one tracklet at a time (or two, interleaved); a lane that finishes one takes the next start
// hit from a device work counter (persistent kernel, grid = SMs x resident blocks). The loop body
// has one propagation and one update shared by both directions, so lanes of a warp that are in
// different phases still execute the same Kalman instructions together. Steps of one tracklet:
//   seed    circle through the first, middle and last chain hits, covariance diag(cov0);
//   out     outward, one row per step: the candidate is the chain hit (from the slab) while the
//           chain lasts, then the hit of smallest chi2 in the row's grid window
//           nsig*sqrt(C)+add; Joseph-form update when chi2 <= chi2_max; stop after n_miss_max
//           empty rows past the chain, on |sin(phi)| >= max_sin, when |y| leaves the row by more
//           than y_margin, or (ext_stop) right after accepting the start hit of another tracklet;
//   in      inward from the outermost hit with the covariance reset: refit the outward hits row
//           by row, then search below the chain start the same way; the state at the last
//           accepted hit is the tracklet's fit at x_ref.
// Output per tracklet: fit (P, C, chi2, x_ref), counts, and its hit in every row of
// [ref_row, top_row] in the tracklet-major slab.
#include "tpc_dev.cuh"

namespace tpc {


// Processing-order key of a tracklet (a counting sort over kNRow + 1 buckets): order 1 takes the
// longest chains first, order 2 the innermost start rows first, order 3 the outermost start rows
// first (the outermost chain of a track runs to its end and back over the whole track when an
// extension stops at the next tracklet's start hit).
__device__ __forceinline__ int order_key(const Work& W, int order, uint32_t t, int m) {
  if (order == 1) return kNRow - m;
  const int r0 = ((int)W.starts[t].y % kSegPerFrame) % kNRow;
  return order == 3 ? kNRow - 1 - r0 : r0;
}

// Adds n to counter[key] once per group of lanes of the warp with the same key; returns the value
// before this lane's share (lanes of a group take consecutive values in lane order). All 32 lanes
// call it; lanes with take = false add nothing.
__device__ __forceinline__ uint32_t warp_add(uint32_t* counter, int key, bool take) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, take ? key : -1);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (take && lane == leader) base = atomicAdd(&counter[key], (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// (middle hit, last hit, chain length) of every start hit; the chain hits go to slab rows r0 .. r0+m-1
__global__ void __launch_bounds__(256) k_chains(Work W, int order) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const uint32_t stride = gridDim.x * blockDim.x;
  // warp-uniform trip count: every lane takes part in the aggregated count
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < ntl; t0 += stride) {
    const uint32_t t = t0 + (threadIdx.x & 31u);
    int m = 0;
    if (t < ntl) {
      const uint4 st = W.starts[t];
      const int r0 = ((int)st.y % kSegPerFrame) % kNRow;
      int head = (int)st.x, mid = head;
      m = 1;
      W.slab[slab_at(t, r0)] = (uint32_t)head;
      for (;;) {
        const int nx = W.clinks[head].y;
        if (nx < 0 || m >= kNRow) break;
        head = nx;
        W.slab[slab_at(t, r0 + m)] = (uint32_t)head;
        ++m;
        if ((m & 1) == 0) mid = W.clinks[mid].y;
      }
      W.chains[t] = make_int4(mid, head, m, 0);
    }
    if (order) (void)warp_add(W.len_cnt, t < ntl ? order_key(W, order, t, m) : 0, t < ntl);
  }
}

// Processing order of the tracklet kernel (order_key; the order inside a bucket is arbitrary, and
// no result depends on it: every tracklet reads only the grid and the links and writes only its
// own outputs). Long tracklets first shorten the tail where few lanes still run.
// One warp: exclusive scan of the kNRow + 1 bucket counts.
__global__ void __launch_bounds__(32) k_length_offsets(Work W) {
  constexpr int kPer = (kNRow + 1 + 31) / 32;
  const int lane = threadIdx.x;
  uint32_t c[kPer], s = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = lane * kPer + j;
    c[j] = k <= kNRow ? W.len_cnt[k] : 0u;
    s += c[j];
  }
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  uint32_t run = x - s;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = lane * kPer + j;
    if (k <= kNRow) W.len_cnt[k] = run;
    run += c[j];
  }
}
__global__ void __launch_bounds__(256) k_length_scatter(Work W, int order) {
  const uint32_t ntl = W.cnt->n_tracklets;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < ntl; t0 += stride) {
    const uint32_t t = t0 + (threadIdx.x & 31u);
    const bool ok = t < ntl;
    const uint32_t slot = warp_add(W.len_cnt, ok ? order_key(W, order, t, W.chains[t].z) : 0, ok);
    if (ok) W.order[slot] = t;
  }
}

__device__ __forceinline__ void reset_cov(const DevParams& Q, float* C) {
#pragma unroll
  for (int i = 0; i < 15; ++i) C[i] = 0.f;
  C[lt(0, 0)] = Q.cov0[0];
  C[lt(1, 1)] = Q.cov0[1];
  C[lt(2, 2)] = Q.cov0[2];
  C[lt(3, 3)] = Q.cov0[3];
  C[lt(4, 4)] = Q.cov0[4];
}

// smallest-chi2 hit of segment g inside the window around the predicted (y, w); -1 if none
template <bool kPacked>
__device__ __forceinline__ int search_row(const Work& W, const DevParams& Q, const int4 sdim, const float4 sgeo,
                                          uint32_t sbb, const float* P, const float* C, const SInv& V, float& chi_out,
                                          float2& hit_out) {
  const float wy = Q.win_nsig * sqrtf(C[lt(0, 0)]) + Q.win_add;
  const float ww = Q.win_nsig * sqrtf(C[lt(1, 1)]) + Q.win_add;
  const GridWin q = grid_window_from(sdim, sgeo, sbb, P[0], P[1], wy, ww);
  int best = -1;
  float bchi = __int_as_float(0x7f800000);
  float2 bc = make_float2(0.f, 0.f);
  for (int cw = q.iw0; cw <= q.iw1; ++cw) {
    const uint32_t col = q.bb + (uint32_t)(cw * q.ny);
    const int base = col_base(q.cw0, q.cshift, cw);
    const int p1 = (int)W.bin_start[col + q.iy1 + 1];
    for (int h0 = (int)W.bin_start[col + q.iy0]; h0 < p1; h0 += 4) {
      // up to four candidates per memory round trip: the coordinates are loaded together, then
      // tested in position order
      float2 cb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        cb[u] = h0 + u < p1 ? hit_in_col<kPacked>(W.hyw, W.hq, h0 + u, base) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int h = h0 + u;
        const float2 c = cb[u];
        if (h >= p1 || !(fabsf(c.x - P[0]) <= wy && fabsf(c.y - P[1]) <= ww)) continue;
        const float chi = kf_chi2(V, P, c.x, c.y);
        bool better;
        if (best < 0 || chi < bchi) better = true;
        else if (chi > bchi) better = false;
        else better = key_less(c.y, c.x, W.horig[h], bc.y, bc.x, W.horig[best]);
        if (better) { best = h; bchi = chi; bc = c; }
      }
    }
  }
  chi_out = bchi;
  hit_out = bc;
  return best;
}

// kThreads threads per block, compiled for kRegs registers per thread (the resident blocks per SM
// follow: 65536 / (kThreads * kRegs))
template <int kThreads, int kRegs, bool kPacked>
__global__ void __launch_bounds__(kThreads, 65536 / (kThreads * kRegs)) k_tracklets(Work W, DevParams Q, int ordered) {
  const uint32_t ntl = W.cnt->n_tracklets;
  float P[5], C[15];
  // state at the last accepted hit, kept in shared memory (one column per thread) to save registers
  __shared__ float sv[20][kThreads];
  const int tid = threadIdx.x;
  float chi2sum = 0.f;
  int t = -1, r = 0, r0 = 0, top = -1, ref = -1, nmiss = 0, nh = 0, mlen = 0, gb = 0;
  uint32_t steps = 0;
  unsigned long long all_steps = 0, all_hits = 0;
  bool inward = false, active = false;
  for (;;) {
    if (!active) {
      // next tracklet: seed from the precomputed chain
      const uint32_t tn = atomicAdd(&W.cnt->k5_next, 1u);
      if (tn >= ntl) {
        if (all_steps) {
          atomicAdd(&W.cnt->n_steps, all_steps);
          atomicAdd(&W.cnt->n_tracklet_hits, all_hits);
        }
        break;
      }
      t = ordered ? (int)W.order[tn] : (int)tn;
      const uint4 st = W.starts[t];
      const int4 ch = W.chains[t];
      const int g = (int)st.y;
      r0 = (g % kSegPerFrame) % kNRow;
      gb = g - r0;
      const float2 a = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, g, (int)st.x);
      const float2 b = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, gb + r0 + ch.z / 2, ch.x);
      const float2 c = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, gb + r0 + ch.z - 1, ch.y);
      float hh[3][3];
      hh[0][0] = Q.x[r0];                hh[0][1] = a.x; hh[0][2] = a.y;
      hh[1][0] = Q.x[r0 + ch.z / 2];     hh[1][1] = b.x; hh[1][2] = b.y;
      hh[2][0] = Q.x[r0 + ch.z - 1];     hh[2][1] = c.x; hh[2][2] = c.y;
      if (!kf_seed(Q, hh, P)) {
        W.tl_info[t] = 0u;
        continue;
      }
      reset_cov(Q, C);
      r = r0;
      top = -1;
      nmiss = 0;
      mlen = ch.z;
      inward = false;
      active = true;
    }
    // ---- one row step (both directions)
    ++steps;
    bool stop = false;
    // loads whose addresses are known before the propagation are issued first, so its arithmetic
    // covers their latency: a known candidate (chain hit outward, outward result inward), or the
    // grid geometry of the row to search
    const bool known = inward ? r >= r0 : r < r0 + mlen;
    int khit = -1;
    float2 kc = make_float2(0.f, 0.f);
    int4 sdim = make_int4(0, 0, 0, 0);
    float4 sgeo = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t sbb = 0;
    if (known) {
      const uint32_t s = W.slab[slab_at((uint32_t)t, r)];
      if (s != kNoHit) {
        khit = (int)s;
        kc = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, gb + r, khit);
      }
    } else {
      sdim = W.seg_dim[gb + r];
      sgeo = W.seg_geo[gb + r];
      sbb = W.seg_bb[gb + r];
    }
    const bool prop = inward ? (r < top) : (r > r0);
    if (prop) {
      const float xf = row_x(Q, inward ? r + 1 : r - 1);
      if (!kf_propagate(Q, P, C, xf, row_x(Q, r))) stop = true;
      else if (fabsf(P[0]) > row_x(Q, r) * Q.tan10 + Q.y_margin) stop = true;
    }
    if (!stop) {
      int hit = -1;
      float chi = __int_as_float(0x7f800000);
      float2 c = make_float2(0.f, 0.f);
      bool searched = false;
      const SInv V = kf_sinv(Q, C);
      if (known) {
        hit = khit;
        c = kc;
        if (hit >= 0) chi = kf_chi2(V, P, c.x, c.y);
      } else {
        searched = true;
        hit = search_row<kPacked>(W, Q, sdim, sgeo, sbb, P, C, V, chi, c);
      }
      const bool acc = hit >= 0 && chi <= Q.chi2_max;
      if (acc) {
        kf_update(Q, V, P, C, c.x, c.y);
#pragma unroll
        for (int i = 0; i < 5; ++i) sv[i][tid] = P[i];
        // the saved covariance is read only at the end of the inward pass (the tracklet's fit); the
        // inward restart after the outward pass takes the parameters alone
        if (inward) {
#pragma unroll
          for (int i = 0; i < 15; ++i) sv[5 + i][tid] = C[i];
        }
        nmiss = 0;
        if (inward) {
          nh += 1;
          chi2sum = chi2sum + chi;
          ref = r;
        } else {
          top = r;
          // the extension reached another tracklet's start hit: that tracklet covers the rows beyond
          if (searched && Q.ext_stop && W.is_start[hit]) stop = true;
        }
      } else {
        nmiss += 1;
        if (searched && nmiss >= Q.n_miss_max) stop = true;
      }
      W.slab[slab_at((uint32_t)t, r)] = acc ? (uint32_t)hit : kNoHit;
      r += inward ? -1 : 1;
      if (r < 0 || r >= kNRow) stop = true;
    }
    if (stop) {
      if (!inward) {
        if (top < 0) {
          W.tl_info[t] = 0u;
          all_steps += steps;
          steps = 0;
          active = false;
          continue;
        }
        // inward: start again from the outermost hit with the covariance reset
#pragma unroll
        for (int i = 0; i < 5; ++i) P[i] = sv[i][tid];
        reset_cov(Q, C);
        inward = true;
        r = top;
        nmiss = 0;
        nh = 0;
        ref = -1;
        chi2sum = 0.f;
      } else {
        if (ref >= 0) {
          float* o = W.tl_state + (long long)t * 24;
#pragma unroll
          for (int i = 0; i < 5; ++i) o[i] = sv[i][tid];
#pragma unroll
          for (int i = 0; i < 15; ++i) o[5 + i] = sv[5 + i][tid];
          o[20] = chi2sum;
          o[21] = Q.x[ref];
          W.tl_info[t] = (uint32_t)nh | ((uint32_t)ref << 8) | ((uint32_t)top << 16) | (1u << 24);
          all_hits += (unsigned long long)nh;
        } else {
          W.tl_info[t] = 0u;
        }
        all_steps += steps;
        steps = 0;
        active = false;
      }
    }
  }
}

// One tracklet in flight in a lane: its state between row steps.
struct Tl {
  float P[5], C[15];
  float chi2sum;
  int t, r, r0, top, ref, nmiss, nh, mlen, gb;
  uint32_t steps;
  bool inward, active, done;
};
// The loads of one row step whose addresses are known before the propagation: a known candidate
// (chain hit outward, outward result inward), or the grid geometry of the row to search.
struct TlLoads {
  bool known;
  int khit;
  float2 kc;
  int4 sdim;
  float4 sgeo;
  uint32_t sbb;
};

// Takes start hits from the work counter until one seeds (T.active) or the counter is exhausted
// (T.done).
template <bool kPacked>
__device__ __forceinline__ void tl_take(const Work& W, const DevParams& Q, Tl& T, uint32_t ntl, int ordered) {
  while (!T.active) {
    const uint32_t tn = atomicAdd(&W.cnt->k5_next, 1u);
    if (tn >= ntl) {
      T.done = true;
      return;
    }
    const int t = ordered ? (int)W.order[tn] : (int)tn;
    const uint4 st = W.starts[t];
    const int4 ch = W.chains[t];
    const int g = (int)st.y;
    const int r0 = (g % kSegPerFrame) % kNRow;
    const int gb = g - r0;
    T.t = t;
    T.r0 = r0;
    T.gb = gb;
    // seed from the precomputed chain
    const float2 a = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, g, (int)st.x);
    const float2 b = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, gb + r0 + ch.z / 2, ch.x);
    const float2 c = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, gb + r0 + ch.z - 1, ch.y);
    float hh[3][3];
    hh[0][0] = Q.x[r0];                hh[0][1] = a.x; hh[0][2] = a.y;
    hh[1][0] = Q.x[r0 + ch.z / 2];     hh[1][1] = b.x; hh[1][2] = b.y;
    hh[2][0] = Q.x[r0 + ch.z - 1];     hh[2][1] = c.x; hh[2][2] = c.y;
    if (!kf_seed(Q, hh, T.P)) {
      W.tl_info[t] = 0u;
      continue;
    }
    reset_cov(Q, T.C);
    T.r = r0;
    T.top = -1;
    T.nmiss = 0;
    T.mlen = ch.z;
    T.inward = false;
    T.active = true;
  }
}

template <bool kPacked>
__device__ __forceinline__ TlLoads tl_loads(const Work& W, const Tl& T) {
  TlLoads L;
  L.known = T.inward ? T.r >= T.r0 : T.r < T.r0 + T.mlen;
  L.khit = -1;
  L.kc = make_float2(0.f, 0.f);
  L.sdim = make_int4(0, 0, 0, 0);
  L.sgeo = make_float4(0.f, 0.f, 0.f, 0.f);
  L.sbb = 0;
  if (L.known) {
    const uint32_t s = W.slab[slab_at((uint32_t)T.t, T.r)];
    if (s != kNoHit) {
      L.khit = (int)s;
      L.kc = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, T.gb + T.r, L.khit);
    }
  } else {
    L.sdim = W.seg_dim[T.gb + T.r];
    L.sgeo = W.seg_geo[T.gb + T.r];
    L.sbb = W.seg_bb[T.gb + T.r];
  }
  return L;
}

// The propagation to the step's row (none on the first row of a direction); true: stop.
__device__ __forceinline__ bool tl_propagate(const DevParams& Q, Tl& T) {
  const bool prop = T.inward ? (T.r < T.top) : (T.r > T.r0);
  if (!prop) return false;
  const float xf = row_x(Q, T.inward ? T.r + 1 : T.r - 1);
  if (!kf_propagate(Q, T.P, T.C, xf, row_x(Q, T.r))) return true;
  return fabsf(T.P[0]) > row_x(Q, T.r) * Q.tan10 + Q.y_margin;
}

// The measurement of the step's row: the known hit or the window search, the update, the slab
// entry; sv = the lane's column of the saved state (stride kStride). True: stop.
template <bool kPacked, int kStride>
__device__ __forceinline__ bool tl_measure(const Work& W, const DevParams& Q, Tl& T, const TlLoads& L, float* sv) {
  bool stop = false;
  int hit = -1;
  float chi = __int_as_float(0x7f800000);
  float2 c = make_float2(0.f, 0.f);
  bool searched = false;
  const SInv V = kf_sinv(Q, T.C);
  if (L.known) {
    hit = L.khit;
    c = L.kc;
    if (hit >= 0) chi = kf_chi2(V, T.P, c.x, c.y);
  } else {
    searched = true;
    hit = search_row<kPacked>(W, Q, L.sdim, L.sgeo, L.sbb, T.P, T.C, V, chi, c);
  }
  const bool acc = hit >= 0 && chi <= Q.chi2_max;
  if (acc) {
    kf_update(Q, V, T.P, T.C, c.x, c.y);
#pragma unroll
    for (int i = 0; i < 5; ++i) sv[i * kStride] = T.P[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) sv[(5 + i) * kStride] = T.C[i];
    T.nmiss = 0;
    if (T.inward) {
      T.nh += 1;
      T.chi2sum = T.chi2sum + chi;
      T.ref = T.r;
    } else {
      T.top = T.r;
      // the extension reached another tracklet's start hit: that tracklet covers the rows beyond
      if (searched && Q.ext_stop && W.is_start[hit]) stop = true;
    }
  } else {
    T.nmiss += 1;
    if (searched && T.nmiss >= Q.n_miss_max) stop = true;
  }
  W.slab[slab_at((uint32_t)T.t, T.r)] = acc ? (uint32_t)hit : kNoHit;
  T.r += T.inward ? -1 : 1;
  if (T.r < 0 || T.r >= kNRow) stop = true;
  return stop;
}

// The end of a direction: the outward pass turns inward from the outermost hit with the covariance
// reset; the inward pass writes the tracklet's fit and frees the lane's slot.
template <int kStride>
__device__ __forceinline__ void tl_stop(const Work& W, const DevParams& Q, Tl& T, const float* sv,
                                        unsigned long long& all_steps, unsigned long long& all_hits) {
  if (!T.inward) {
    if (T.top < 0) {
      W.tl_info[T.t] = 0u;
      all_steps += T.steps;
      T.steps = 0;
      T.active = false;
      return;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) T.P[i] = sv[i * kStride];
    reset_cov(Q, T.C);
    T.inward = true;
    T.r = T.top;
    T.nmiss = 0;
    T.nh = 0;
    T.ref = -1;
    T.chi2sum = 0.f;
    return;
  }
  if (T.ref >= 0) {
    float* o = W.tl_state + (long long)T.t * 24;
#pragma unroll
    for (int i = 0; i < 20; ++i) o[i] = sv[i * kStride];
    o[20] = T.chi2sum;
    o[21] = Q.x[T.ref];
    W.tl_info[T.t] = (uint32_t)T.nh | ((uint32_t)T.ref << 8) | ((uint32_t)T.top << 16) | (1u << 24);
    all_hits += (unsigned long long)T.nh;
  } else {
    W.tl_info[T.t] = 0u;
  }
  all_steps += T.steps;
  T.steps = 0;
  T.active = false;
}

// The same construction with kIlp tracklets in flight per lane: each loop iteration advances every
// one of them by one row step, phase by phase (loads, propagations, measurements, ends), so their
// independent chains of dependent arithmetic and loads can overlap within one thread.
template <int kThreads, int kRegs, bool kPacked, int kIlp>
__global__ void __launch_bounds__(kThreads, 65536 / (kThreads * kRegs))
    k_tracklets_ilp(Work W, DevParams Q, int ordered) {
  const uint32_t ntl = W.cnt->n_tracklets;
  // state at the last accepted hit, kept in shared memory (one column per thread) to save registers
  __shared__ float sv[kIlp][20][kThreads];
  const int tid = threadIdx.x;
  Tl T[kIlp];
#pragma unroll
  for (int k = 0; k < kIlp; ++k) {
    T[k].chi2sum = 0.f;
    T[k].t = -1; T[k].r = 0; T[k].r0 = 0; T[k].top = -1; T[k].ref = -1;
    T[k].nmiss = 0; T[k].nh = 0; T[k].mlen = 0; T[k].gb = 0;
    T[k].steps = 0;
    T[k].inward = false; T[k].active = false; T[k].done = false;
  }
  unsigned long long all_steps = 0, all_hits = 0;
  for (;;) {
    bool any = false;
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
      if (!T[k].active && !T[k].done) tl_take<kPacked>(W, Q, T[k], ntl, ordered);
      any = any || T[k].active;
    }
    if (!any) break;
    // ---- one row step of every tracklet in flight (both directions)
    TlLoads L[kIlp];
    bool stop[kIlp];
#pragma unroll
    for (int k = 0; k < kIlp; ++k)
      if (T[k].active) {
        ++T[k].steps;
        L[k] = tl_loads<kPacked>(W, T[k]);
      }
#pragma unroll
    for (int k = 0; k < kIlp; ++k) stop[k] = T[k].active && tl_propagate(Q, T[k]);
#pragma unroll
    for (int k = 0; k < kIlp; ++k)
      if (T[k].active && !stop[k]) stop[k] = tl_measure<kPacked, kThreads>(W, Q, T[k], L[k], &sv[k][0][tid]);
#pragma unroll
    for (int k = 0; k < kIlp; ++k)
      if (T[k].active && stop[k]) tl_stop<kThreads>(W, Q, T[k], &sv[k][0][tid], all_steps, all_hits);
  }
  if (all_steps) {
    atomicAdd(&W.cnt->n_steps, all_steps);
    atomicAdd(&W.cnt->n_tracklet_hits, all_hits);
  }
}

// host-side launchers (the kernel templates stay in this translation unit). Shapes: one tracklet
// per lane at 64, 128 or 256 threads per block, each compiled for 64, 72 or 80 registers per
// thread; two tracklets per lane at 64 or 128 threads, compiled for 128 registers (fewer spill).
template <int kT, int kR, bool kP, int kI>
static auto k5_kernel() {
  if constexpr (kI == 1) return k_tracklets<kT, kR, kP>;
  else return k_tracklets_ilp<kT, kR, kP, kI>;
}
template <int kT, int kR, int kI>
static void launch_shape(int packed, int grid, cudaStream_t s, const Work& W, const DevParams& Q, int ordered) {
  if (packed) k5_kernel<kT, kR, true, kI>()<<<grid, kT, 0, s>>>(W, Q, ordered);
  else k5_kernel<kT, kR, false, kI>()<<<grid, kT, 0, s>>>(W, Q, ordered);
}
template <int kT, int kR, int kI>
static int shape_blocks(int packed) {
  int nb = 0;
  if (packed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k5_kernel<kT, kR, true, kI>(), kT, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k5_kernel<kT, kR, false, kI>(), kT, 0);
  return nb;
}
#define TPC_K5_SHAPES                                                                              \
  TPC_K5_SHAPE(64, 64, 1) TPC_K5_SHAPE(64, 72, 1) TPC_K5_SHAPE(64, 80, 1)                          \
  TPC_K5_SHAPE(128, 64, 1) TPC_K5_SHAPE(128, 72, 1) TPC_K5_SHAPE(128, 80, 1)                       \
  TPC_K5_SHAPE(256, 64, 1) TPC_K5_SHAPE(256, 72, 1) TPC_K5_SHAPE(256, 80, 1)                       \
  TPC_K5_SHAPE(64, 128, 2) TPC_K5_SHAPE(128, 128, 2)
// false for a shape that is not compiled
bool launch_tracklets(int threads, int regs, int ilp, int packed, int grid, cudaStream_t s, const Work& W,
                      const DevParams& Q, int ordered) {
#define TPC_K5_SHAPE(T, R, I)                                  \
  if (threads == T && regs == R && ilp == I) {                 \
    launch_shape<T, R, I>(packed, grid, s, W, Q, ordered);     \
    return true;                                               \
  }
  TPC_K5_SHAPES
#undef TPC_K5_SHAPE
  return false;
}
int tracklets_blocks_per_sm(int threads, int regs, int ilp, int packed) {
#define TPC_K5_SHAPE(T, R, I) \
  if (threads == T && regs == R && ilp == I) return shape_blocks<T, R, I>(packed);
  TPC_K5_SHAPES
#undef TPC_K5_SHAPE
  return 0;
}
#undef TPC_K5_SHAPES

}  // namespace tpc
