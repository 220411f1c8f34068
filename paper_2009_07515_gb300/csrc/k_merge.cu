// k_merge.cu — K12: merging of sector tracks across sector boundaries and the global refit
// (Sec. 6: after the standalone sector tracking the tracks are refit; Table 1 of Sec. 7.2 times the
// refit with its sorts as "Track Fit").
//
// Method (the full statement is at tpc_get_merged_tracks in tpctrack.h):
//   outer state  each sector track's fit transported row by row, with scattering noise, from its
//                reference row to the row of its last hit;
//   candidates   a track B of a phi-neighbouring sector of the same frame and drift side whose
//                reference row lies 1 .. merge_gap_rows rows above A's last hit row, with
//                |w_B(x_ref) - w_A(outer)| <= merge_dw;
//   chi2         A's outer state rotated into B's frame and carried by one helix step to B's x_ref;
//                5-parameter chi2 with C_A + C_B (Cholesky); <= merge_chi2_max;
//   matching     mutual best partners (smallest chi2, tie: smaller index), chained inner to outer;
//   refit        every chain refit over all its hits in refit_passes Kalman passes (inward, outward,
//                inward), each from the previous state with the covariance times refit_scale.
//
// Layout and kernels (one thread per track or chain; the candidate search uses a counting sort of
// the tracks by (frame, sector, w bin), kMergeBins bins spanning each frame's w range):
//   k_merge_outer   frame, reference and last row of each track, its outer state, bin counts
//   (exclusive scan of the bin counts)
//   k_merge_fill    each track into its bin's list
//   k_merge_match   candidates of each track in the neighbouring sectors' bins around its outer w,
//                   queued per warp and evaluated 32 at a time: an atomic minimum of (chi2, index)
//                   on each track's best inner and best outer partner
//   k_merge_link    mutual best partners linked; chain heads and their hit counts
//   (exclusive scans: merged index and first hit of each chain head)
//   k_merge_refit   each chain's hits copied in order, the refit, the merged track written
//   k_merge_frames  first merged track and hit of each frame
// Every float result is the oracle's sequence of IEEE operations (fused multiply-adds where it
// accumulates a sum of products, reciprocals formed once and multiplied).
#include "tpc_dev.cuh"

namespace tpc {

// The state at x in the frame of angle alpha, expressed in the frame of angle alpha + d (cd, sd):
// x' = x cd + y sd, y' = y cd - x sd, sin(phi') = sin(phi) cd - cos(phi) sd; the covariance carried
// at fixed x' to first order (J: dy'/dy = c/c1, dw'/dy = -t sd / c1, dsin'/dy = -k sd,
// dsin'/dsin = c1/c). False if cos(phi') <= 0 or |sin(phi')| >= max_sin.
__device__ __forceinline__ bool rotate_state(const DevParams& Q, float* P, float* C, float& x, float cd, float sd) {
  const float s = P[2];
  const float c = sqrtf(1.0f - s * s);
  const float s1 = s * cd - c * sd;
  const float c1 = c * cd + s * sd;
  if (!(c1 > 0.f) || !(fabsf(s1) < Q.max_sin)) return false;
  const float x1 = x * cd + P[0] * sd;
  const float y1 = P[0] * cd - x * sd;
  const float k = Q.kq * P[4];
  const float ic = 1.0f / c, ic1 = 1.0f / c1;
  const float J00 = c * ic1;
  const float J10 = -((P[3] * sd) * ic1);
  const float J20 = -(k * sd);
  const float J22 = c1 * ic;
  // T = J C (rows of the dense index-ordered sums that are not exact copies)
  float T[5][5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    T[0][q] = J00 * C[lt(0, q)];
    T[1][q] = J10 * C[lt(0, q)] + C[lt(1, q)];
    T[2][q] = __fmaf_rn(J22, C[lt(2, q)], J20 * C[lt(0, q)]);
    T[3][q] = C[lt(3, q)];
    T[4][q] = C[lt(4, q)];
  }
  // O = T J^T, lower triangle
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    C[lt(i, 0)] = T[i][0] * J00;
    if (i >= 1) C[lt(i, 1)] = T[i][0] * J10 + T[i][1];
    if (i >= 2) C[lt(i, 2)] = __fmaf_rn(T[i][2], J22, T[i][0] * J20);
    if (i >= 3) C[lt(i, 3)] = T[i][3];
    if (i >= 4) C[lt(i, 4)] = T[i][4];
  }
  P[0] = y1;
  P[2] = s1;
  x = x1;
  return true;
}

// d^T S^-1 d for a symmetric positive definite S (lower triangle), Cholesky and forward
// substitution; +inf when S is not positive definite.
__device__ __forceinline__ float chi2_5(const float* S, const float* d) {
  float L[15], z[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    float acc = S[lt(j, j)];
#pragma unroll
    for (int q = 0; q < j; ++q) acc = __fmaf_rn(-L[lt(j, q)], L[lt(j, q)], acc);
    if (!(acc > 0.f)) return __int_as_float(0x7f800000);
    L[lt(j, j)] = sqrtf(acc);
    const float il = 1.0f / L[lt(j, j)];
#pragma unroll
    for (int i = j + 1; i < 5; ++i) {
      float a = S[lt(i, j)];
#pragma unroll
      for (int q = 0; q < j; ++q) a = __fmaf_rn(-L[lt(i, q)], L[lt(j, q)], a);
      L[lt(i, j)] = a * il;
    }
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float acc = d[i];
#pragma unroll
    for (int q = 0; q < i; ++q) acc = __fmaf_rn(-L[lt(i, q)], z[q], acc);
    z[i] = acc * (1.0f / L[lt(i, i)]);
  }
  float qs = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) qs = __fmaf_rn(z[i], z[i], qs);
  return qs;
}

// the rotation from sector a's frame to the frame of its phi neighbour b: +20 degrees if b follows a
__device__ __forceinline__ float rot_sign(int sa, int sb) { return ((sa % 18) + 1) % 18 == sb % 18 ? 1.0f : -1.0f; }

// frame of batch-global track k (frame_track0 is the first track of each frame)
__device__ __forceinline__ int track_frame(const DevCounters* c, int nf, uint32_t k) {
  int lo = 0, hi = nf - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (c->frame_track0[mid] <= k) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// row index of a track's reference x (x_ref is a row radius, row_x of its row)
__device__ __forceinline__ int ref_row_of(const DevParams& Q, float xref) {
  int r = (int)rintf((xref - 85.0f) / Q.pitch);
  r = min(max(r, 0), kNRow - 1);
  if (row_x(Q, r) != xref) r += row_x(Q, r) < xref ? 1 : -1;
  return min(max(r, 0), kNRow - 1);
}

// the tracker's view (y, w) of input cluster i of frame F: the input, or its 16-bit read-back
__device__ __forceinline__ float2 cluster_yw(const FrameIn& F, uint32_t i, int packed) {
  float y = F.y[i], w = F.w[i];
  if (packed) {
    float qy = rintf((y + 64.0f) * 512.0f);
    qy = fminf(fmaxf(qy, 0.0f), 65535.0f);
    y = qy * (1.0f / 512.0f) - 64.0f;
    w = rintf(w * 512.0f) * (1.0f / 512.0f);
  }
  return make_float2(y, w);
}

// bin of a w in the frame's (sector) bin range
struct MergeBins {
  float lo, inv;
};
__device__ __forceinline__ MergeBins merge_bins(const DevCounters* c, int f) {
  const float lo = ord2f(c->wrange[2 * f]), hi = ord2f(c->wrange[2 * f + 1]);
  return MergeBins{lo, (float)kMergeBins / fmaxf(hi - lo, 1.0f)};
}
__device__ __forceinline__ long long merge_bin(int f, int sector, const MergeBins& b, float w) {
  return ((long long)f * kNSec + sector) * kMergeBins + bin_of(w, b.lo, b.inv, kMergeBins);
}

__device__ __forceinline__ uint32_t track_nhits(const Work& W, uint32_t k, uint32_t ntr) {
  const long long h1 = k + 1 < ntr ? W.tr_hoff[k + 1] : (long long)W.cnt->n_track_hits;
  return (uint32_t)(h1 - W.tr_hoff[k]);
}

__global__ void __launch_bounds__(256) k_merge_outer(Work W, DevParams Q) {
  const uint32_t ntr = W.cnt->n_tracks;
  const int nf = W.batch->nf;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ntr; k += gridDim.x * blockDim.x) {
    const int fr = track_frame(W.cnt, nf, k);
    const uint8_t* row = W.batch->f[fr].row;
    const long long h0 = W.tr_hoff[k];
    const uint32_t nh = track_nhits(W, k, ntr);
    const int last = row[W.tr_hits[h0 + nh - 1]];
    const int ref = ref_row_of(Q, W.tr_xref[k]);
    float P[5], C[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) P[i] = W.tr_param[(long long)k * 5 + i];
#pragma unroll
    for (int i = 0; i < 15; ++i) C[i] = W.tr_cov[(long long)k * 15 + i];
    bool ok = true;
    for (int r = ref + 1; r <= last && ok; ++r) ok = kf_propagate(Q, P, C, row_x(Q, r - 1), row_x(Q, r));
    float* o = W.m_state + (long long)k * 20;
#pragma unroll
    for (int i = 0; i < 5; ++i) o[i] = P[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) o[5 + i] = C[i];
    W.m_info[k] = (uint32_t)last | (uint32_t)ref << 8 | (ok ? 1u : 0u) << 16 | (uint32_t)fr << 17;
    W.m_bestA[k] = ~0ull;
    W.m_bestB[k] = ~0ull;
    W.m_prev[k] = 0u;
    const int sec = W.tr_sector[k];
    atomicAdd(W.m_bin + merge_bin(fr, sec, merge_bins(W.cnt, fr), W.tr_param[(long long)k * 5 + 1]), 1u);
  }
}

__global__ void __launch_bounds__(256) k_merge_fill(Work W) {
  const uint32_t ntr = W.cnt->n_tracks;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ntr; k += gridDim.x * blockDim.x) {
    const int fr = (int)(W.m_info[k] >> 17);
    const long long b = merge_bin(fr, W.tr_sector[k], merge_bins(W.cnt, fr), W.tr_param[(long long)k * 5 + 1]);
    // after this kernel W.m_bin[b] is the end of bin b (its start was the scanned offset)
    W.m_list[atomicAdd(W.m_bin + b, 1u)] = k;
  }
}

// The chi2 of a candidate pair (A, B): A's outer state rotated into B's frame and carried to B's
// reference row, against B's fit; an atomic minimum of (chi2 bits, index) on both tracks' best
// partner words when it passes the cut (chi2 >= 0, so its bits order like its value).
__device__ __forceinline__ void merge_pair(const Work& W, const DevParams& Q, uint32_t a, uint32_t b) {
  const int last = (int)(W.m_info[a] & 255u);
  const int ref_b = (int)((W.m_info[b] >> 8) & 255u);
  const float* oa = W.m_state + (long long)a * 20;
  const float* pb = W.tr_param + (long long)b * 5;
  const float* cb = W.tr_cov + (long long)b * 15;
  float P[5], C[15], x = row_x(Q, last);
#pragma unroll
  for (int q = 0; q < 5; ++q) P[q] = oa[q];
#pragma unroll
  for (int q = 0; q < 15; ++q) C[q] = oa[5 + q];
  if (!rotate_state(Q, P, C, x, Q.rot_c, rot_sign(W.tr_sector[a], W.tr_sector[b]) * Q.rot_s)) return;
  if (!kf_propagate(Q, P, C, x, row_x(Q, ref_b))) return;
  float S[15], d[5];
#pragma unroll
  for (int q = 0; q < 15; ++q) S[q] = C[q] + cb[q];
#pragma unroll
  for (int q = 0; q < 5; ++q) d[q] = P[q] - pb[q];
  const float chi = chi2_5(S, d);
  if (!(chi <= Q.merge_chi2_max)) return;
  const unsigned long long cbits = (unsigned long long)__float_as_uint(chi) << 32;
  atomicMin(W.m_bestA + b, cbits | a);
  atomicMin(W.m_bestB + a, cbits | b);
}

// One lane per track A walks A's candidate range in each phi-neighbouring sector's w bins, one
// candidate per iteration, and applies the cheap cuts (B's reference row 1 .. merge_gap_rows rows
// above A's last row, |w_B(x_ref) - w_A(outer)| <= merge_dw). The pairs that pass go to the warp's
// queue in shared memory; whenever it holds 32 pairs, the 32 lanes compute their chi2 together
// (rotation, one helix step, Cholesky), so the expensive arithmetic runs on full warps although
// only a few tracks of a warp have candidates at a time.
constexpr int kMatchQ = 64;
__global__ void __launch_bounds__(256) k_merge_match(Work W, DevParams Q) {
  __shared__ uint2 queue[256 / 32][kMatchQ];
  const int lane = threadIdx.x & 31;
  uint2* q = queue[threadIdx.x >> 5];
  const unsigned below = (1u << lane) - 1u;
  const uint32_t ntr = W.cnt->n_tracks;
  const uint32_t stride = gridDim.x * blockDim.x;
  int qn = 0;  // pairs in the warp's queue (warp-uniform)
  for (uint32_t a0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); a0 < ntr; a0 += stride) {
    const uint32_t a = a0 + (uint32_t)lane;
    // the lane's two candidate ranges [i, e) and [i2, e2) of the list of bin members
    uint32_t i = 0, e = 0, i2 = 0, e2 = 0;
    int last = 0;
    float wa = 0.f;
    if (a < ntr) {
      const uint32_t ia = W.m_info[a];
      if (ia >> 16 & 1u) {
        const int fr = (int)(ia >> 17);
        last = (int)(ia & 255u);
        const int sa = W.tr_sector[a], side = sa / 18, ka = sa % 18;
        wa = W.m_state[(long long)a * 20 + 1];
        const MergeBins mb = merge_bins(W.cnt, fr);
        const float pad = fabsf(wa) * 1.0e-6f + 1.0e-6f;
        for (int dir = -1; dir <= 1; dir += 2) {
          const int sb = side * 18 + (ka + dir + 18) % 18;
          const long long b0 = merge_bin(fr, sb, mb, (wa - Q.merge_dw) - pad);
          const long long b1 = merge_bin(fr, sb, mb, (wa + Q.merge_dw) + pad);
          const uint32_t lo = b0 > 0 ? W.m_bin[b0 - 1] : 0u, hi = W.m_bin[b1];
          if (dir < 0) { i = lo; e = hi; } else { i2 = lo; e2 = hi; }
        }
      }
    }
    for (;;) {
      if (i >= e && i2 < e2) { i = i2; e = e2; i2 = e2; }
      const bool more = i < e;
      if (!__any_sync(0xffffffffu, more)) break;
      bool pass = false;
      uint32_t b = 0;
      if (more) {
        b = W.m_list[i++];
        const int g = (int)((W.m_info[b] >> 8) & 255u) - last;
        pass = g >= 1 && g <= Q.merge_gap_rows && fabsf(W.tr_param[(long long)b * 5 + 1] - wa) <= Q.merge_dw;
      }
      const unsigned pm = __ballot_sync(0xffffffffu, pass);
      if (pass) q[qn + __popc(pm & below)] = make_uint2(a, b);
      qn += __popc(pm);
      __syncwarp();
      if (qn >= 32) {
        const uint2 pr = q[lane];
        merge_pair(W, Q, pr.x, pr.y);
        __syncwarp();
        if (lane < qn - 32) q[lane] = q[32 + lane];
        qn -= 32;
        __syncwarp();
      }
    }
  }
  if (lane < qn) {
    const uint2 pr = q[lane];
    merge_pair(W, Q, pr.x, pr.y);
  }
}

// mutual best partners linked; chain heads flagged with their hit counts (for the scans)
__global__ void __launch_bounds__(256) k_merge_link(Work W) {
  const uint32_t ntr = W.cnt->n_tracks;
  for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < ntr; a += gridDim.x * blockDim.x) {
    // A's best outer partner and its chi2 (+inf and -1 when A has none)
    const unsigned long long kb = W.m_bestB[a];
    const int b = kb == ~0ull ? -1 : (int)(uint32_t)(kb & 0xFFFFFFFFull);
    W.m_chi[a] = kb == ~0ull ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(kb >> 32));
    const bool link = b >= 0 && (uint32_t)(W.m_bestA[b] & 0xFFFFFFFFull) == a;
    W.m_next[a] = link ? b : -1;
    if (link) W.m_prev[b] = 1u;
  }
}
__global__ void __launch_bounds__(256) k_merge_heads(Work W) {
  const uint32_t ntr = W.cnt->n_tracks;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntr; t += gridDim.x * blockDim.x) {
    const bool head = W.m_prev[t] == 0u;
    uint32_t nh = 0;
    if (head)
      for (int s = (int)t; s >= 0; s = W.m_next[s]) nh += track_nhits(W, (uint32_t)s, ntr);
    W.m_hidx[t] = head ? 1u : 0u;
    W.m_hoff[t] = nh;
  }
}

constexpr int kMaxSeg = 18;  // segments of a chain: at most the sectors of one drift side

__global__ void __launch_bounds__(128, 5) k_merge_refit(Work W, DevParams Q) {
  const uint32_t ntr = W.cnt->n_tracks;
  const int packed = W.packed;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntr; t += gridDim.x * blockDim.x) {
    const uint32_t it = W.m_info[t];
    const int fr = (int)(it >> 17);
    const uint32_t f_t0 = W.cnt->frame_track0[fr];
    // per sector track: its outer partner (frame-local) and the merge chi2
    {
      const int nx = W.m_next[t];
      W.tr_next[t] = nx >= 0 ? nx - (int)f_t0 : -1;
      W.tr_mchi2[t] = nx >= 0 ? W.m_chi[t] : __int_as_float(0x7fc00000);
    }
    if (W.m_prev[t] != 0u) continue;
    const uint32_t m = W.m_hidx[t];
    const FrameIn F = W.batch->f[fr];
    // the chain's hits copied in order, inner segment first; per segment its end in that order and
    // its sector, packed as end | sector << 16 (a chain holds at most kMaxSeg * kNRow hits), read
    // only where a pass crosses from one segment into the next
    uint32_t seg_es[kMaxSeg];
    const uint32_t h_out = W.m_hoff[t];
    uint32_t nh = 0;
    int nseg = 0, tm = (int)t;
    for (int s = (int)t; s >= 0 && nseg < kMaxSeg; s = W.m_next[s]) {
      const uint32_t n = track_nhits(W, (uint32_t)s, ntr);
      const long long h0 = W.tr_hoff[s];
      for (uint32_t i = 0; i < n; ++i) W.mt_hits[h_out + nh + i] = W.tr_hits[h0 + i];
      nh += n;
      seg_es[nseg] = nh | (uint32_t)W.tr_sector[s] << 16;
      tm = s;
      ++nseg;
    }
    float Pr[5], Cr[15], xr = 0.f, chi_last = 0.f;
    int sr = W.tr_sector[t], nfit = 0;
    if (W.m_info[tm] >> 16 & 1u) {
      float P[5], Cs[15];
      const float* om = W.m_state + (long long)tm * 20;
#pragma unroll
      for (int i = 0; i < 5; ++i) P[i] = om[i];
#pragma unroll
      for (int i = 0; i < 15; ++i) Cs[i] = om[5 + i];
      const uint32_t* mh = W.mt_hits + h_out;
      bool ok = true;
      for (int pass = 0; pass < Q.refit_passes && ok; ++pass) {
        const bool inward = pass != 1;
        float C[15];
#pragma unroll
        for (int i = 0; i < 15; ++i) C[i] = Cs[i] * Q.refit_scale;
        // the current segment j spans hits [lo, hi) of the chain; the next hit's row and (y, w)
        // are loaded one hit ahead, so their latency is not on the chain of dependent Kalman
        // operations
        int j = inward ? nseg - 1 : 0;
        uint32_t hi = seg_es[j] & 0xffffu, lo = j > 0 ? seg_es[j - 1] & 0xffffu : 0u;
        int hsec = (int)(seg_es[j] >> 16);
        int cur_sec = hsec, cur_row = -2;
        float cur_x = 0.f, chi_pass = 0.f;
        int n_pass = 0;
        uint32_t k = inward ? nh - 1 : 0;
        uint32_t hc = mh[k];
        int nrow = F.row[hc];
        float2 nc = cluster_yw(F, hc, packed);
        for (uint32_t k2 = 0; k2 < nh; ++k2) {
          if (k < lo || k >= hi) {
            j += inward ? -1 : 1;
            hi = seg_es[j] & 0xffffu;
            lo = j > 0 ? seg_es[j - 1] & 0xffffu : 0u;
            hsec = (int)(seg_es[j] >> 16);
          }
          const int r = nrow;
          const float2 c = nc;
          // advance the cursor and prefetch the next hit
          if (k2 + 1 < nh) {
            k = inward ? k - 1 : k + 1;
            const uint32_t hn = mh[k];
            nrow = F.row[hn];
            nc = cluster_yw(F, hn, packed);
          }
          if (hsec != cur_sec) {
            if (!rotate_state(Q, P, C, cur_x, Q.rot_c, rot_sign(cur_sec, hsec) * Q.rot_s)) { ok = false; break; }
            cur_sec = hsec;
            cur_row = -1;
          }
          if (cur_row == -1) {
            if (!kf_propagate(Q, P, C, cur_x, row_x(Q, r))) { ok = false; break; }
          } else if (cur_row >= 0) {
            bool bad = false;
            if (inward) {
              for (int rr = cur_row - 1; rr >= r && !bad; --rr) bad = !kf_propagate(Q, P, C, row_x(Q, rr + 1), row_x(Q, rr));
            } else {
              for (int rr = cur_row + 1; rr <= r && !bad; ++rr) bad = !kf_propagate(Q, P, C, row_x(Q, rr - 1), row_x(Q, rr));
            }
            if (bad) { ok = false; break; }
          }
          cur_row = r;
          cur_x = row_x(Q, r);
          const SInv V = kf_sinv(Q, C);
          const float chi = kf_chi2(V, P, c.x, c.y);
          kf_update(Q, V, P, C, c.x, c.y);
          chi_pass = chi_pass + chi;
          ++n_pass;
#pragma unroll
          for (int q = 0; q < 5; ++q) Pr[q] = P[q];
#pragma unroll
          for (int q = 0; q < 15; ++q) Cr[q] = C[q];
          xr = cur_x;
          sr = cur_sec;
        }
        nfit = n_pass;
        chi_last = chi_pass;
#pragma unroll
        for (int q = 0; q < 15; ++q) Cs[q] = Cr[q];
      }
    }
    const float nan = __int_as_float(0x7fc00000);
#pragma unroll
    for (int q = 0; q < 5; ++q) W.mt_param[(long long)m * 5 + q] = nfit ? Pr[q] : nan;
#pragma unroll
    for (int q = 0; q < 15; ++q) W.mt_cov[(long long)m * 15 + q] = nfit ? Cr[q] : nan;
    W.mt_chi2[m] = nfit ? chi_last : nan;
    W.mt_xref[m] = nfit ? xr : nan;
    W.mt_sector[m] = sr;
    W.mt_ndf[m] = 2 * nfit - 5;
    W.mt_nfit[m] = nfit;
    W.mt_nseg[m] = nseg;
    W.mt_head[m] = (int)(t - f_t0);
    W.mt_hoff[m] = (long long)h_out;
  }
}

// per frame: first merged track and merged hit
__global__ void k_merge_frames(Work W) {
  const int nf = W.batch->nf;
  const uint32_t ntr = W.cnt->n_tracks;
  for (int f = threadIdx.x; f <= nf; f += blockDim.x) {
    const uint32_t t0 = W.cnt->frame_track0[f];
    W.cnt->frame_merged0[f] = t0 < ntr ? W.m_hidx[t0] : W.cnt->n_merged;
    W.cnt->frame_mhit0[f] = t0 < ntr ? W.m_hoff[t0] : W.cnt->n_merged_hits;
  }
}

}  // namespace tpc
