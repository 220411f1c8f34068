// k_cf.cu — cluster finding from digits: the first GPU step of the synchronous reconstruction
// (Table 1 of Sec. 6.2; Sec. 2: the TPC records, per pad, the charge of every time bin, and a pad
// row's clusters are reconstructed from these zero-suppressed digits).
//
// Rules (the full statement is at tpc_find_clusters in tpctrack.h):
//   peak     a digit c with q_c >= q_peak_min that beats each neighbour n of its 3x3 window:
//            q_n < q_c, or q_n = q_c and n comes later in (time, pad) order;
//   cluster  the 3x3 window plus each cell of the 5x5 ring whose charge does not exceed that of
//            the window cell next to it on the way to the peak; kept if its charge Q >= q_total_min;
//   values   integer moment sums, then FP32 IEEE operations in a fixed order (mean pad and time,
//            y and w of the centroid, widths in pads and time bins).
//
// The charge map is dense per (sector, row) and lives in HBM across calls, zero between them:
// only the cells of the frame's digits are written, read and cleared, so a frame costs traffic in
// proportion to its digits, not to the map. Kernels (persistent, tiles of 256 digits):
//   k_cf_fill   validate each digit and OR its charge into its cell (a 32-bit atomic on the cell's
//               word; a nonzero old half is a second digit in the same cell)
//   k_cf_peaks  peak test and cluster charge; one bit per digit, kept clusters per tile
//   (exclusive scan of the tile counts: each tile's first output slot)
//   k_cf_build  each kept peak recomputes its sums and writes its cluster at its ordered slot
//   k_cf_clear  zero the cells of the valid digits, leaving the map clean for the next call
#include "tpc_dev.cuh"

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
  return ((size_t)(s * kNRow + r) * (size_t)A.lines + (size_t)(j + kCfGuard)) * (size_t)A.stride +
         (size_t)(k + kCfGuard);
}

// c beats its 3x3 neighbours: earlier ones (in (time, pad) order) strictly, later ones or ties
__device__ __forceinline__ bool cf_is_peak(const uint16_t* m, int stride, int q) {
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      if (dk == 0 && dj == 0) continue;
      const int qn = __ldg(m + dj * stride + dk);
      const bool later = dj > 0 || (dj == 0 && dk > 0);
      if (later ? qn > q : qn >= q) return false;
    }
  return true;
}

struct CfSums {
  int Q, Sk, Sj, Skk, Sjj;
};

// moment sums over the 3x3 window and the 5x5 ring cells that do not rise away from the peak
__device__ __forceinline__ CfSums cf_sums(const uint16_t* m, int stride) {
  int v[5][5];  // v[dj + 2][dk + 2]
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) v[a][b] = __ldg(m + (a - 2) * stride + (b - 2));
  CfSums S{0, 0, 0, 0, 0};
#pragma unroll
  for (int dj = -2; dj <= 2; ++dj)
#pragma unroll
    for (int dk = -2; dk <= 2; ++dk) {
      int q = v[dj + 2][dk + 2];
      const bool ring = dk == 2 || dk == -2 || dj == 2 || dj == -2;
      if (ring) {
        const int ik = dk == 2 ? 1 : dk == -2 ? -1 : dk;
        const int ij = dj == 2 ? 1 : dj == -2 ? -1 : dj;
        if (q > v[ij + 2][ik + 2]) q = 0;
      }
      S.Q += q;
      S.Sk += q * dk;
      S.Sj += q * dj;
      S.Skk += q * dk * dk;
      S.Sjj += q * dj * dj;
    }
  return S;
}

__global__ void __launch_bounds__(kCfTile) k_cf_fill(CfArgs A) {
  uint32_t bad = 0;
  for (long long i = (long long)blockIdx.x * kCfTile + threadIdx.x; i < A.n; i += (long long)gridDim.x * kCfTile) {
    int s, r, k, j, q;
    if (!cf_digit(A, i, s, r, k, j, q)) {
      bad |= kCfErrDigit;
      continue;
    }
    const size_t c = cf_cell(A, s, r, k, j);
    const uint32_t sh = (uint32_t)(c & 1) * 16u;
    const uint32_t old = atomicOr(reinterpret_cast<uint32_t*>(A.map) + (c >> 1), (uint32_t)q << sh);
    if ((old >> sh) & 0xFFFFu) bad |= kCfErrTwice;
  }
  if (bad) atomicOr(A.err, bad);
}

__global__ void __launch_bounds__(kCfTile) k_cf_peaks(CfArgs A) {
  __shared__ uint32_t wc[kCfTile / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ntiles = (A.n + kCfTile - 1) / kCfTile;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long i = t * kCfTile + threadIdx.x;
    bool keep = false;
    int s, r, k, j, q;
    if (i < A.n && cf_digit(A, i, s, r, k, j, q) && q >= A.q_peak_min) {
      const uint16_t* m = A.map + cf_cell(A, s, r, k, j);
      if (cf_is_peak(m, A.stride, q)) keep = cf_sums(m, A.stride).Q >= A.q_total_min;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    const long long wbase = t * kCfTile + warp * 32;
    if (lane == 0) {
      if (wbase < A.n) A.mask[wbase >> 5] = b;
      wc[warp] = (uint32_t)__popc(b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t c = 0;
#pragma unroll
      for (int w = 0; w < kCfTile / 32; ++w) c += wc[w];
      A.tcount[t] = c;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kCfTile) k_cf_build(CfArgs A) {
  __shared__ uint32_t wc[kCfTile / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ntiles = (A.n + kCfTile - 1) / kCfTile;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long wbase = t * kCfTile + warp * 32;
    const uint32_t b = wbase < A.n ? A.mask[wbase >> 5] : 0u;
    if (lane == 0) wc[warp] = (uint32_t)__popc(b);
    __syncthreads();
    uint32_t off = A.toff[t];
    for (int w = 0; w < warp; ++w) off += wc[w];
    __syncthreads();
    if ((b >> lane) & 1u) {
      const long long i = wbase + lane;
      const int s = A.sector[i], r = A.row[i], k = A.pad[i], j = A.time[i];
      const uint16_t* m = A.map + cf_cell(A, s, r, k, j);
      const CfSums S = cf_sums(m, A.stride);
      const uint32_t o = off + (uint32_t)__popc(b & ((1u << lane) - 1u));
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
      A.o_qmax[o] = A.adc[i];
      A.o_sig_pad[o] = vk > 0.f ? __fsqrt_rn(vk) : 0.f;
      A.o_sig_time[o] = vj > 0.f ? __fsqrt_rn(vj) : 0.f;
      A.o_digit[o] = (uint32_t)i;
    }
  }
}

__global__ void __launch_bounds__(kCfTile) k_cf_clear(CfArgs A) {
  for (long long i = (long long)blockIdx.x * kCfTile + threadIdx.x; i < A.n; i += (long long)gridDim.x * kCfTile) {
    int s, r, k, j, q;
    if (cf_digit(A, i, s, r, k, j, q)) A.map[cf_cell(A, s, r, k, j)] = 0;
  }
}

}  // namespace tpc
