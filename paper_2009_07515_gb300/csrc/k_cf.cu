// k_cf.cu — cluster finding from digits: the first GPU step of the synchronous reconstruction
// (Table 1 of Sec. 7.2; Sec. 2: the TPC records, per pad, the charge of every time bin, and a pad
// row's clusters are reconstructed from these zero-suppressed digits).
//
// Rules (the full statement is at tpc_find_clusters in tpctrack.h):
//   peak     a digit c with q_c >= q_peak_min that beats each neighbour n of its 3x3 window:
//            q_n < q_c, or q_n = q_c and n comes later in (time, pad) order;
//   cluster  the 3x3 window plus each cell of the 5x5 ring whose charge does not exceed that of
//            the window cell next to it on the way to the peak; kept if its charge Q >= q_total_min;
//   values   integer moment sums, then FP32 IEEE operations in a fixed order (mean pad and time,
//            y and w of the centroid, widths in pads and time bins);
//   order    the input order of the peak digits.
//
// The charge map is dense per (sector, row) and lives in HBM across calls, zero between them:
// only the cells of the frame's digits are written, read and cleared, so a frame costs traffic in
// proportion to its digits, not to the map. Kernels (persistent, tiles of 256 digits):
//   k_cf_fill   validate each digit and add its charge into its cell (a 32-bit atomic add on the
//               cell's word; a cell that was not zero before the add holds a second digit)
//   k_cf_peaks  each digit checks that its cell holds its own charge (else a second digit shares
//               the cell), the peak test, the cluster of a kept peak; each warp writes its kept
//               clusters compacted in digit order into its block's region of a temporary array
//               (slots taken from a shared-memory counter), their first slot and their count
//   (exclusive scan of the per-warp counts: each warp's first output slot)
//   k_cf_copy   the clusters of each 32 digits move to their output slots (coalesced stores)
//   k_cf_clear  zero the cells of the valid digits, leaving the map clean for the next call
#include "cf_dev.cuh"

namespace tpc {

__device__ __forceinline__ bool cf_digit(const CfArgs& A, long long i, int& s, int& r, int& k, int& j, int& q) {
  s = A.sector[i];
  r = A.row[i];
  k = A.pad[i];
  j = A.time[i];
  q = A.adc[i];
  return s < kNSec && r < kNRow && k < (int)__ldg(A.npads + r) && j < A.n_time && q > 0;
}

__device__ __forceinline__ size_t cf_cell(const CfArgs& A, int s, int r, int k, int j) {
  return ((size_t)(s * kNRow + r) * (size_t)A.lines + (size_t)(j - A.t_lo + kCfGuard)) * (size_t)A.stride +
         (size_t)(k + kCfGuard);
}
// the digit's cell is in this pass's map: its window or the two halo lines on each side
__device__ __forceinline__ bool cf_in_map(const CfArgs& A, int j) { return j >= A.t_lo - kCfGuard && j < A.t_hi + kCfGuard; }
__device__ __forceinline__ bool cf_in_window(const CfArgs& A, int j) { return j >= A.t_lo && j < A.t_hi; }

// the 3x3 window around a cell, w[dj + 1][dk + 1]
__device__ __forceinline__ void cf_window3(const uint16_t* m, int stride, int w[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) w[a][b] = __ldg(m + (a - 1) * stride + (b - 1));
}

// the centre beats its 3x3 neighbours: earlier ones (in (time, pad) order) strictly, later ones or ties
__device__ __forceinline__ bool cf_is_peak3(const int w[3][3]) {
  const int q = w[1][1];
  bool peak = true;
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      if (dk == 0 && dj == 0) continue;
      const int qn = w[dj + 1][dk + 1];
      const bool later = dj > 0 || (dj == 0 && dk > 0);
      peak &= later ? qn <= q : qn < q;
    }
  return peak;
}

struct CfSums {
  int Q, Sk, Sj, Skk, Sjj;
};

// moment sums over the 3x3 window (given) and the 5x5 ring cells that do not rise away from the peak
__device__ __forceinline__ CfSums cf_sums3(const uint16_t* m, int stride, const int w[3][3]) {
  CfSums S{0, 0, 0, 0, 0};
#pragma unroll
  for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
    for (int dk = -2; dk <= 2; ++dk) {
      const bool ring = dk == 2 || dk == -2 || dj == 2 || dj == -2;
      int q;
      if (ring) {
        const int ik = dk == 2 ? 1 : dk == -2 ? -1 : dk;
        const int ij = dj == 2 ? 1 : dj == -2 ? -1 : dj;
        q = __ldg(m + dj * stride + dk);
        if (q > w[ij + 1][ik + 1]) q = 0;
      } else {
        q = w[dj + 1][dk + 1];
      }
      S.Q += q;
      S.Sk += q * dk;
      S.Sj += q * dj;
      S.Skk += q * dk * dk;
      S.Sjj += q * dj * dj;
    }
  return S;
}

__global__ void __launch_bounds__(kCfTile, 8) k_cf_fill(CfArgs A) {
  uint32_t bad = 0;
  for (long long i = (long long)blockIdx.x * kCfTile + threadIdx.x; i < A.n; i += (long long)gridDim.x * kCfTile) {
    int s, r, k, j, q;
    if (!cf_digit(A, i, s, r, k, j, q)) {
      bad |= kCfErrDigit;
      continue;
    }
    if (!cf_in_map(A, j)) continue;
    const size_t c = cf_cell(A, s, r, k, j);
    const uint32_t sh = (uint32_t)(c & 1) * 16u;
    const uint32_t old = atomicAdd(reinterpret_cast<uint32_t*>(A.map) + (c >> 1), (uint32_t)q << sh);
    // the map is zero at the start of a call, so a non-zero cell before the add means a second
    // digit in the cell, whatever the charges add up to
    if ((old >> sh) & 0xffffu) bad |= kCfErrTwice;
  }
  if (bad) atomicOr(A.err, bad);
}

__global__ void __launch_bounds__(kCfTile) k_cf_peaks(CfArgs A) {
  __shared__ uint32_t used;  // temporary slots taken in this block's region
  const int lane = threadIdx.x & 31;
  const long long ntiles = (A.n + kCfTile - 1) / kCfTile;
  // the block's region: as many slots as the digits of its tiles (blockIdx.x + k * gridDim.x)
  const uint32_t region = (uint32_t)(blockIdx.x * ((ntiles + gridDim.x - 1) / gridDim.x) * kCfTile);
  if (threadIdx.x == 0) used = 0;
  __syncthreads();
  uint32_t bad = 0;
  // warp-uniform trip count (block-aligned bases): every lane takes part in the warp's compaction
  for (long long base = (long long)blockIdx.x * kCfTile; base < A.n; base += (long long)gridDim.x * kCfTile) {
    const long long i = base + threadIdx.x;
    bool keep = false;
    int s = 0, r = 0, k = 0, j = 0, q = 0;
    CfSums S{0, 0, 0, 0, 0};
    if (i < A.n && cf_digit(A, i, s, r, k, j, q)) {
      const uint16_t* m = A.map + cf_cell(A, s, r, k, j);
      int w[3][3];
      cf_window3(m, A.stride, w);
      if (w[1][1] != q) bad |= kCfErrTwice;
      if (q >= A.q_peak_min && cf_is_peak3(w)) {
        S = cf_sums3(m, A.stride, w);
        keep = S.Q >= A.q_total_min;
      }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    const long long wbase = i - lane;
    uint32_t first = 0;
    if (lane == 0 && b) first = region + atomicAdd(&used, (uint32_t)__popc(b));
    first = __shfl_sync(0xffffffffu, first, 0);
    if (keep) {
      const uint32_t o = first + (uint32_t)__popc(b & ((1u << lane) - 1u));
      const float Qf = (float)S.Q;
      const float mk = __fdiv_rn((float)S.Sk, Qf), mj = __fdiv_rn((float)S.Sj, Qf);
      const float pc = __fadd_rn((float)k, mk), tc = __fadd_rn((float)j, mj);
      const float centre = __fsub_rn((float)((int)__ldg(A.npads + r) / 2), 0.5f);
      const float vk = __fsub_rn(__fdiv_rn((float)S.Skk, Qf), __fmul_rn(mk, mk));
      const float vj = __fsub_rn(__fdiv_rn((float)S.Sjj, Qf), __fmul_rn(mj, mj));
      A.t_sector[o] = (uint8_t)s;
      A.t_row[o] = (uint8_t)r;
      A.t_y[o] = __fmul_rn(__fsub_rn(pc, centre), A.pitch);
      A.t_w[o] = __fmul_rn(__fadd_rn(tc, 0.5f), A.dw);
      A.t_qtot[o] = (uint32_t)S.Q;
      A.t_qmax[o] = (uint16_t)q;
      A.t_sig_pad[o] = vk > 0.f ? __fsqrt_rn(vk) : 0.f;
      A.t_sig_time[o] = vj > 0.f ? __fsqrt_rn(vj) : 0.f;
      A.t_digit[o] = (uint32_t)i;
    }
    if (lane == 0 && wbase < A.n) {
      A.wcount[wbase >> 5] = (uint32_t)__popc(b);
      A.wsrc[wbase >> 5] = first;
    }
  }
  if (bad) atomicOr(A.err, bad);
}

// The kept clusters of each 32 digits (a group), compacted from their temporary slot on, move to
// their output slots. A warp takes 32 consecutive groups, whose output slots are consecutive: each lane
// lists the source slots of its group's clusters in shared memory at their output positions, then
// the warp copies in output order, so the stores of each field are coalesced.
__global__ void __launch_bounds__(kCfTile, 8) k_cf_copy(CfArgs A) {
  __shared__ uint32_t srcs[kCfTile / 32][32 * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* sl = srcs[warp];
  const long long ng = (A.n + 31) / 32;
  const long long step = (long long)gridDim.x * kCfTile;
  // block-aligned bases: the trip count is warp-uniform
  for (long long base = (long long)blockIdx.x * kCfTile; base < ng; base += step) {
    const long long g = base + threadIdx.x;
    const long long g0 = g - lane;
    if (g0 >= ng) continue;  // warp-uniform
    const uint32_t cnt = g < ng ? A.wcount[g] : 0u, off = g < ng ? A.woff[g] : 0u;
    const uint32_t first = __shfl_sync(0xffffffffu, off, 0);
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    const uint32_t src0 = g < ng ? A.wsrc[g] : 0u;
    for (uint32_t r = 0; r < cnt; ++r) sl[off - first + r] = src0 + r;
    __syncwarp();
    for (uint32_t q = lane; q < total; q += 32) {
      const uint32_t src = sl[q], dst = first + q;
      A.o_sector[dst] = A.t_sector[src];
      A.o_row[dst] = A.t_row[src];
      A.o_y[dst] = A.t_y[src];
      A.o_w[dst] = A.t_w[src];
      A.o_qtot[dst] = A.t_qtot[src];
      A.o_qmax[dst] = A.t_qmax[src];
      A.o_sig_pad[dst] = A.t_sig_pad[src];
      A.o_sig_time[dst] = A.t_sig_time[src];
      A.o_digit[dst] = A.t_digit[src];
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kCfTile) k_cf_clear(CfArgs A) {
  const long long step = (long long)gridDim.x * kCfTile;
  for (long long i = (long long)blockIdx.x * kCfTile + threadIdx.x; i < A.n; i += 2 * step) {
    int s0, r0, k0, j0, q0, s1 = 0, r1 = 0, k1 = 0, j1 = 0, q1 = 0;
    const bool v0 = cf_digit(A, i, s0, r0, k0, j0, q0) && cf_in_map(A, j0);
    const bool v1 = i + step < A.n && cf_digit(A, i + step, s1, r1, k1, j1, q1) && cf_in_map(A, j1);
    if (v0) A.map[cf_cell(A, s0, r0, k0, j0)] = 0;
    if (v1) A.map[cf_cell(A, s1, r1, k1, j1)] = 0;
  }
}

// ---- time windows (a frame whose map exceeds the budget). First the group lists: each group of 32
// consecutive digits is listed under the windows whose maps its valid digits reach (window w's map
// holds bins [w tw - 2, (w + 1) tw + 2)); a group reaching more than two windows (digits far apart in
// time, e.g. a shuffled frame) goes to a wide list that every window visits. Then pass 1, per window:
// fill, flag, clear over the window's groups; the flags of each 32 digits accumulate over the
// windows (each digit lies in one window), and so do their counts. After the scan of the counts,
// pass 2, per window: fill, emit, clear; each kept peak computes its cluster again and writes it to
// its output slot (the group's first slot plus its rank among the group's flagged digits), so the
// output is in the input order of the peaks, as in one pass over the whole frame. A window's passes
// read only its groups' digits, not the whole frame's.

// windows [wlo, whi] whose maps the group's digits reach; false when it has none (all lanes take
// part). Only the sector, row and time are read: a digit with a bad sector, row or time sets
// kCfErrDigit in bad here, one with a bad pad or charge is found by k_cf_wfill (its group is
// listed).
__device__ __forceinline__ bool cf_group_windows(const CfArgs& A, long long g, int lane, int& wlo, int& whi,
                                                 uint32_t& bad) {
  const long long i = g * 32 + lane;
  int tmin = 0x7fffffff, tmax = -1;
  if (i < A.n) {
    const int j = A.time[i];
    if (A.sector[i] < kNSec && A.row[i] < kNRow && j < A.n_time) {
      tmin = j;
      tmax = j;
    } else {
      bad |= kCfErrDigit;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
  }
  if (tmax < 0) return false;
  wlo = max(0, tmin - kCfGuard) / A.tw;
  whi = min(A.nwin - 1, (tmax + kCfGuard) / A.tw);
  return true;
}

// a group's windows as one word: wlo | whi << 16, kCfNoWindow for a group without valid digits
constexpr uint32_t kCfNoWindow = 0xFFFFFFFFu;

// per group, one warp: its windows into gwin; per block: the groups of each window (shared
// counters, then one global add per window)
__global__ void __launch_bounds__(kCfTile) k_cf_gcount(CfArgs A) {
  extern __shared__ uint32_t sc[];  // [nwin + 1]
  for (int w = threadIdx.x; w <= A.nwin; w += blockDim.x) sc[w] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long ng = (A.n + 31) / 32, nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  uint32_t bad = 0;
  for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += nwarp) {
    int wlo = 0, whi = 0;
    const bool any = cf_group_windows(A, g, lane, wlo, whi, bad);
    if (lane != 0) continue;
    A.gwin[g] = any ? (uint32_t)wlo | ((uint32_t)whi << 16) : kCfNoWindow;
    if (!any) continue;
    if (whi - wlo <= 1) {
      atomicAdd(&sc[wlo], 1u);
      if (whi != wlo) atomicAdd(&sc[whi], 1u);
    } else {
      atomicAdd(&sc[A.nwin], 1u);
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < A.nwin; w += blockDim.x)
    if (sc[w]) atomicAdd(&A.gcnt[w], sc[w]);
  if (threadIdx.x == 0 && sc[A.nwin]) atomicAdd(&A.gcnt[kCfMaxWindows], sc[A.nwin]);
  if (bad) atomicOr(A.err, bad);
}

// one block: exclusive scan of the windows' group counts into the list starts and cursors
__global__ void __launch_bounds__(1024) k_cf_gscan(CfArgs A) {
  constexpr int kPer = (kCfMaxWindows + 1 + 1023) / 1024;
  __shared__ uint32_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t v[kPer], s = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int w = t * kPer + k;
    v[k] = w < A.nwin ? A.gcnt[w] : 0u;
    s += v[k];
  }
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w0 = wsum[lane];
    uint32_t z = w0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    wsum[lane] = z - w0;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + x - s;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int w = t * kPer + k;
    if (w <= A.nwin) {
      A.gbeg[w] = run;
      A.gcur[w] = run;
    }
    run += v[k];
  }
  if (t == 0) A.gcur[kCfMaxWindows] = 0u;
}

// per block, one thread per group (from gwin): the groups counted again, a base per window taken
// from the cursors, then each group written to its windows' lists (or the wide list)
__global__ void __launch_bounds__(kCfTile) k_cf_gplace(CfArgs A) {
  extern __shared__ uint32_t sc[];  // [2 (nwin + 1)]: counts, then local cursors; block bases
  uint32_t* sb = sc + A.nwin + 1;
  for (int w = threadIdx.x; w <= A.nwin; w += blockDim.x) sc[w] = 0u;
  __syncthreads();
  const long long ng = (A.n + 31) / 32, nthr = (long long)gridDim.x * blockDim.x;
  const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long g = g0; g < ng; g += nthr) {
    const uint32_t e = A.gwin[g];
    if (e == kCfNoWindow) continue;
    const int wlo = (int)(e & 0xFFFFu), whi = (int)(e >> 16);
    if (whi - wlo <= 1) {
      atomicAdd(&sc[wlo], 1u);
      if (whi != wlo) atomicAdd(&sc[whi], 1u);
    } else {
      atomicAdd(&sc[A.nwin], 1u);
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w <= A.nwin; w += blockDim.x) {
    sb[w] = sc[w] ? atomicAdd(w < A.nwin ? &A.gcur[w] : &A.gcur[kCfMaxWindows], sc[w]) : 0u;
    sc[w] = 0u;
  }
  __syncthreads();
  for (long long g = g0; g < ng; g += nthr) {
    const uint32_t e = A.gwin[g];
    if (e == kCfNoWindow) continue;
    const int wlo = (int)(e & 0xFFFFu), whi = (int)(e >> 16);
    if (whi - wlo <= 1) {
      A.glist[sb[wlo] + atomicAdd(&sc[wlo], 1u)] = (uint32_t)g;
      if (whi != wlo) A.glist[sb[whi] + atomicAdd(&sc[whi], 1u)] = (uint32_t)g;
    } else {
      A.gwide[sb[A.nwin] + atomicAdd(&sc[A.nwin], 1u)] = (uint32_t)g;
    }
  }
}

// the groups of window A.win, one warp per group: its list, then the wide list
template <typename F>
__device__ __forceinline__ void cf_visit_groups(const CfArgs& A, F&& f) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long b = A.gbeg[A.win], nl = (long long)A.gbeg[A.win + 1] - b, nw = A.gcnt[kCfMaxWindows];
  for (long long x = wid; x < nl + nw; x += nwarp) f(x < nl ? (long long)A.glist[b + x] : (long long)A.gwide[x - nl]);
}

__global__ void __launch_bounds__(kCfTile) k_cf_wfill(CfArgs A) {
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0;
  cf_visit_groups(A, [&](long long g) {
    const long long i = g * 32 + lane;
    int s, r, k, j, q;
    if (i >= A.n) return;
    if (!cf_digit(A, i, s, r, k, j, q)) {
      bad |= kCfErrDigit;
      return;
    }
    if (!cf_in_map(A, j)) return;
    const size_t c = cf_cell(A, s, r, k, j);
    const uint32_t sh = (uint32_t)(c & 1) * 16u;
    const uint32_t old = atomicAdd(reinterpret_cast<uint32_t*>(A.map) + (c >> 1), (uint32_t)q << sh);
    if ((old >> sh) & 0xffffu) bad |= kCfErrTwice;
  });
  if (bad) atomicOr(A.err, bad);
}

__global__ void __launch_bounds__(kCfTile) k_cf_wclear(CfArgs A) {
  const int lane = threadIdx.x & 31;
  cf_visit_groups(A, [&](long long g) {
    const long long i = g * 32 + lane;
    int s, r, k, j, q;
    if (i < A.n && cf_digit(A, i, s, r, k, j, q) && cf_in_map(A, j)) A.map[cf_cell(A, s, r, k, j)] = 0;
  });
}

__global__ void __launch_bounds__(kCfTile) k_cf_flag(CfArgs A) {
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0;
  cf_visit_groups(A, [&](long long g) {
    const long long i = g * 32 + lane;
    bool keep = false;
    int s = 0, r = 0, k = 0, j = 0, q = 0;
    if (i < A.n && cf_digit(A, i, s, r, k, j, q) && cf_in_window(A, j)) {
      const uint16_t* m = A.map + cf_cell(A, s, r, k, j);
      int w[3][3];
      cf_window3(m, A.stride, w);
      if (w[1][1] != q) bad |= kCfErrTwice;
      if (q >= A.q_peak_min && cf_is_peak3(w)) keep = cf_sums3(m, A.stride, w).Q >= A.q_total_min;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    if (lane == 0 && b) {
      A.wflag[g] |= b;
      A.wcount[g] += (uint32_t)__popc(b);
    }
  });
  if (bad) atomicOr(A.err, bad);
}

// the groups of window A.win, one lane per group (for kernels whose work per group is sparse)
template <typename F>
__device__ __forceinline__ void cf_visit_groups_lane(const CfArgs& A, F&& f) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const long long b = A.gbeg[A.win], nl = (long long)A.gbeg[A.win + 1] - b, nw = A.gcnt[kCfMaxWindows];
  for (long long x = tid; x < nl + nw; x += nthr) f(x < nl ? (long long)A.glist[b + x] : (long long)A.gwide[x - nl]);
}

// one lane per group: the group's flagged digits of this window, each cluster computed again and
// written to its slot (the peaks are about one digit in eight, so a warp per group would leave
// most lanes idle)
__global__ void __launch_bounds__(kCfTile) k_cf_emit(CfArgs A) {
  cf_visit_groups_lane(A, [&](long long g) {
    uint32_t fl = A.wflag[g];
    const uint32_t o0 = A.woff[g];
    for (uint32_t rest = fl; rest; rest &= rest - 1u) {
      const int l = __ffs(rest) - 1;
      const long long i = g * 32 + l;
      int s = 0, r = 0, k = 0, j = 0, q = 0;
      if (i >= A.n || !cf_digit(A, i, s, r, k, j, q) || !cf_in_window(A, j)) continue;
      const uint16_t* m = A.map + cf_cell(A, s, r, k, j);
      int w[3][3];
      cf_window3(m, A.stride, w);
      const CfSums S = cf_sums3(m, A.stride, w);
      const uint32_t o = o0 + (uint32_t)__popc(fl & ((1u << l) - 1u));
      const float Qf = (float)S.Q;
      const float mk = __fdiv_rn((float)S.Sk, Qf), mj = __fdiv_rn((float)S.Sj, Qf);
      const float pc = __fadd_rn((float)k, mk), tc = __fadd_rn((float)j, mj);
      const float centre = __fsub_rn((float)((int)__ldg(A.npads + r) / 2), 0.5f);
      const float vk = __fsub_rn(__fdiv_rn((float)S.Skk, Qf), __fmul_rn(mk, mk));
      const float vj = __fsub_rn(__fdiv_rn((float)S.Sjj, Qf), __fmul_rn(mj, mj));
      A.o_sector[o] = (uint8_t)s;
      A.o_row[o] = (uint8_t)r;
      A.o_y[o] = __fmul_rn(__fsub_rn(pc, centre), A.pitch);
      A.o_w[o] = __fmul_rn(__fadd_rn(tc, 0.5f), A.dw);
      A.o_qtot[o] = (uint32_t)S.Q;
      A.o_qmax[o] = (uint16_t)q;
      A.o_sig_pad[o] = vk > 0.f ? __fsqrt_rn(vk) : 0.f;
      A.o_sig_time[o] = vj > 0.f ? __fsqrt_rn(vj) : 0.f;
      A.o_digit[o] = (uint32_t)i;
    }
  });
}

}  // namespace tpc
