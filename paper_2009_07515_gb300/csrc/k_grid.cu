// k_grid.cu — K0/K1: input validation and the per-(sector, row) search grid.
//
// The grid is a counting sort of the batch's clusters by (frame, sector, row, w-bin, y-bin): each
// segment (frame, sector, row) gets a 2-D grid over the drift coordinate w and the pad-row
// coordinate y with about `occ` clusters per bin and bins shaped like the neighbour window, so a
// window of a row is one contiguous range of sorted positions per w-column it touches. The grid
// decides no result: every window test downstream is an exact comparison on the coordinates, and
// every tie is broken by the (w, y, input index) order.
//
// Kernels (all persistent, sizes read from device memory so the sequence can be graph-captured):
//   k_seg_hist    validate, count clusters per segment, w range per frame
//   k_seg_layout  bins per segment (occupancy target), bin origins and densities in w and y
//   k_bin_rank    bin histogram; each cluster keeps its arrival rank inside its bin
//   k_scatter     sorted (y, w) and input index at bin_start[bin] + rank
//   (batches of more than kTwoPassMin clusters do these two steps per segment instead:
//   k_seg_bucket, k_bin_rank_seg, k_scatter_seg, with each segment's bins zeroed and scanned by the
//   block that ranks it; the allocation-free entry keeps the one-pass form)
//   scans         exclusive prefix sums with device-side lengths
#include "tpc_dev.cuh"

namespace tpc {

// ------------------------------------------------------------------------------------ scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// length of a scan: device-side count + add (clamped to the buffer's capacity), or a host value
__device__ __forceinline__ uint32_t scan_len(const uint32_t* n_dev, long long n_host, int add) {
  if (!n_dev) return (uint32_t)n_host;
  const long long n = (long long)*n_dev + add;
  return (uint32_t)(n < n_host ? n : n_host);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, const uint32_t* n_dev,
                                                              long long n_host, int n_add, uint32_t* __restrict__ tile_sum) {
  const uint32_t n = scan_len(n_dev, n_host, n_add);
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint32_t base = tile * kScanTile, s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      uint32_t i = base + k * kScanThreads + threadIdx.x;
      if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t v = threadIdx.x < kScanThreads / 32 ? warp_sums[threadIdx.x] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) tile_sum[tile] = v;
    }
    __syncthreads();
  }
}

// single block: exclusive scan of the tile sums in place; total written to *total (if given). Each
// thread takes kTileItems consecutive sums per pass, so a pass covers 1024 * kTileItems tiles.
constexpr int kTileItems = 8;
__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t* tile_sum, const uint32_t* n_dev, long long n_host,
                                                     int n_add, uint32_t* total) {
  const uint32_t n = scan_len(n_dev, n_host, n_add);
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < ntiles; base += blockDim.x * kTileItems) {
    const uint32_t i0 = base + threadIdx.x * kTileItems;
    uint32_t v[kTileItems], s = 0;
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) {
      v[k] = i0 + k < ntiles ? tile_sum[i0 + k] : 0u;
      s += v[k];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t w = threadIdx.x < blockDim.x / 32 ? warp_sums[threadIdx.x] : 0, z = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (threadIdx.x >= o) z += y;
      }
      warp_sums[threadIdx.x] = z - w;
    }
    __syncthreads();
    uint32_t run = carry + warp_sums[threadIdx.x >> 5] + x - s;
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) {
      if (i0 + k < ntiles) tile_sum[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// exclusive scan of each tile plus its offset; out[n] = total. in may alias out.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* in, const uint32_t* n_dev, long long n_host,
                                                             int n_add, const uint32_t* __restrict__ tile_off,
                                                             const uint32_t* total, uint32_t* out) {
  const uint32_t n = scan_len(n_dev, n_host, n_add);
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  __shared__ uint32_t buf[kScanTile];
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t base = tile * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      uint32_t i = base + k * kScanThreads + threadIdx.x;
      buf[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) { v[k] = buf[threadIdx.x * kScanItems + k]; s += v[k]; }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t w = threadIdx.x < kScanThreads / 32 ? warp_sums[threadIdx.x] : 0, z = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (threadIdx.x >= o) z += y;
      }
      if (threadIdx.x < kScanThreads / 32) warp_sums[threadIdx.x] = z - w;
    }
    __syncthreads();
    uint32_t run = tile_off[tile] + warp_sums[threadIdx.x >> 5] + x - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) { buf[threadIdx.x * kScanItems + k] = run; run += v[k]; }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      uint32_t i = base + k * kScanThreads + threadIdx.x;
      if (i < n) out[i] = buf[k * kScanThreads + threadIdx.x];
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

// Single-launch exclusive scan for arrays of a small capacity: block b scans array b of up to two
// (in[b] may alias out[b]); each thread takes 4 consecutive entries of every 4096-entry tile, and a
// running carry joins the tiles. out[n] = total, *total = total.
struct SmallScan {
  const uint32_t* in[2];
  uint32_t* out[2];
  const uint32_t* n_dev[2];
  long long n_host[2];
  uint32_t* total[2];
};
constexpr int kSmallScanThreads = 1024;
__global__ void __launch_bounds__(kSmallScanThreads) k_scan_small(SmallScan a) {
  const int b = blockIdx.x;
  const uint32_t n = scan_len(a.n_dev[b], a.n_host[b], 0);
  const uint32_t* in = a.in[b];
  uint32_t* out = a.out[b];
  __shared__ uint32_t warp_sums[kSmallScanThreads / 32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  constexpr int kItems = 4;
  constexpr uint32_t kTile = kSmallScanThreads * kItems;
  for (uint32_t base = 0; base < n; base += kTile) {
    const uint32_t i0 = base + (uint32_t)kItems * threadIdx.x;
    uint32_t v[kItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      v[k] = i0 + k < n ? in[i0 + k] : 0u;
      sum += v[k];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = warp_sums[lane];
      uint32_t z = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      warp_sums[lane] = z - w;  // exclusive prefix of the warps' sums
    }
    __syncthreads();
    uint32_t run = s_carry + warp_sums[warp] + (x - sum);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      if (i0 + k < n) out[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();  // every thread has read s_carry and warp_sums
    if (threadIdx.x == kSmallScanThreads - 1) s_carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[n] = s_carry;
    if (a.total[b]) *a.total[b] = s_carry;
  }
}

// ------------------------------------------------------------------------------------ K1
// One input cluster, validated; in the 16-bit storage its coordinates are replaced by their
// read-back values (y = rint(512 (y + 64)) / 512 - 64 clamped, w = rint(512 w) / 512), which the
// grid bins and every later kernel then use. The storage needs |w| < 32768 cm.
struct InHit {
  int g;
  float y, w;
  bool ok;
};
__device__ __forceinline__ InHit read_input(const BatchDesc* B, int packed, long long i, int& fi, long long& j) {
  fi = frame_of(B, i);
  const FrameIn& F = B->f[fi];
  j = i - F.off;
  InHit h;
  const int s = F.sector[j], r = F.row[j];
  h.y = F.y[j];
  h.w = F.w[j];
  h.ok = s < kNSec && r < kNRow && isfinite(h.y) && isfinite(h.w);
  if (h.ok && packed) {
    h.ok = fabsf(h.w) < 32767.0f;
    float qy = rintf((h.y + 64.0f) * 512.0f);
    qy = fminf(fmaxf(qy, 0.0f), 65535.0f);
    h.y = qy * (1.0f / 512.0f) - 64.0f;
    h.w = rintf(h.w * 512.0f) * (1.0f / 512.0f);
  }
  h.g = fi * kSegPerFrame + s * kNRow + r;
  return h;
}

// Clusters are processed in contiguous block chunks (one block per SM), so a block rarely spans
// two frames. Each block counts the segments of its first frame in shared memory and adds its
// nonzero counts to the global ones at the end (a few global atomics per segment instead of one
// per cluster); clusters of a later frame in its chunk are counted in global memory directly.
__global__ void __launch_bounds__(kHistThreads) k_seg_hist(Work W) {
  __shared__ uint32_t hist[kSegPerFrame];
  const BatchDesc* B = W.batch;
  const long long ntot = B->ntot;
  const long long chunk = (ntot + gridDim.x - 1) / gridDim.x;
  const long long i0 = (long long)blockIdx.x * chunk;
  const long long i1 = min(ntot, i0 + chunk);
  for (int k = threadIdx.x; k < kSegPerFrame; k += blockDim.x) hist[k] = 0u;
  const int f0 = i0 < ntot ? frame_of(B, i0) : 0;
  __syncthreads();
  int f = -1;
  uint32_t lo = 0xFFFFFFFFu, hi = 0u;
  bool bad = false;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    int fi;
    long long j;
    const InHit h = read_input(B, W.packed, i, fi, j);
    if (fi != f) {
      if (f >= 0 && lo <= hi) {
        atomicMin(&W.cnt->wrange[2 * f], lo);
        atomicMax(&W.cnt->wrange[2 * f + 1], hi);
      }
      f = fi; lo = 0xFFFFFFFFu; hi = 0u;
    }
    if (!h.ok) { bad = true; continue; }
    if (fi == f0) atomicAdd(&hist[h.g - f0 * kSegPerFrame], 1u);
    else atomicAdd(&W.seg_cnt[h.g], 1u);
    const uint32_t e = f2ord(h.w);
    lo = min(lo, e);
    hi = max(hi, e);
  }
  // lanes of a warp on the same frame combine their range first: one atomic pair per warp
  const unsigned same = __match_any_sync(0xffffffffu, f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const int f2 = __shfl_xor_sync(0xffffffffu, f, o);
    if (f2 == f) { lo = min(lo, lo2); hi = max(hi, hi2); }
  }
  const int leader = __ffs(same) - 1;
  if ((int)(threadIdx.x & 31) == leader && f >= 0 && lo <= hi) {
    atomicMin(&W.cnt->wrange[2 * f], lo);
    atomicMax(&W.cnt->wrange[2 * f + 1], hi);
  }
  if (bad) atomicOr(&W.cnt->err, kErrInput);
  __syncthreads();
  if (i0 < ntot)
    for (int k = threadIdx.x; k < kSegPerFrame; k += blockDim.x)
      if (hist[k]) atomicAdd(&W.seg_cnt[f0 * kSegPerFrame + k], hist[k]);
}

// One thread per segment: a grid of ~n/occ bins, nw x ny, bins shaped like the neighbour window
// (w/y size ratio `aspect`). The w-columns have a power-of-two width 2^k cm (-3 <= k <= 7, nearest
// to the occupancy target) and are aligned to multiples of it, so a cluster's 16-bit w offset
// from its column's lower edge always fits. A segment has at most 4 ceil(n/occ) + 260 bins, or 513
// in the 16-bit storage when a sparse segment spans the whole w range.
__global__ void __launch_bounds__(256) k_seg_layout(Work W, DevParams Q) {
  const BatchDesc* B = W.batch;
  const int nseg = B->nf * kSegPerFrame;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nseg; g += gridDim.x * blockDim.x) {
    const int f = g / kSegPerFrame, r = (g % kSegPerFrame) % kNRow;
    const uint32_t n = W.seg_cnt[g];
    float wlo = 0.f, whi = 0.f;
    if (W.cnt->wrange[2 * f] <= W.cnt->wrange[2 * f + 1]) {
      wlo = ord2f(W.cnt->wrange[2 * f]);
      whi = ord2f(W.cnt->wrange[2 * f + 1]);
    }
    const float wext = whi - wlo, yext = 2.f * Q.yext[r];
    uint32_t nbins = 1;
    if (n > 0) {
      const float want = ceilf((float)n / Q.occ);
      nbins = want < 1.f ? 1u : (want > 4194304.f ? 4194304u : (uint32_t)want);
    }
    uint32_t ny = 1;
    if (wext > 0.f && nbins > 1) {
      const float fy = sqrtf((float)nbins * (yext / wext) * Q.aspect);
      ny = fy < 1.f ? 1u : (fy > 64.f ? 64u : (uint32_t)(fy + 0.5f));
      if (ny > nbins) ny = nbins;
    }
    // column width: the power of two nearest (in log) to the occupancy's width; coarser while a
    // sparse segment would get many more columns than bins (up to 128 cm in the 16-bit storage,
    // where |w| < 32768 cm keeps it below 513 columns)
    const float bw_want = wext > 0.f ? wext / (float)((nbins + ny - 1) / ny) : 128.f;
    const int kmax = W.packed ? 7 : 30;
    int k = 7;
    while (k > -3 && ldexpf(1.41421356f, k - 1) > bw_want) --k;
    int iw0 = (int)floorf(ldexpf(wlo, -k)), iw1 = (int)floorf(ldexpf(whi, -k));
    while ((uint32_t)(iw1 - iw0 + 1) > max(4u * nbins, 64u) + 16u && k < kmax) {
      ++k;
      iw0 = (int)floorf(ldexpf(wlo, -k));
      iw1 = (int)floorf(ldexpf(whi, -k));
    }
    const uint32_t nw = (uint32_t)(iw1 - iw0 + 1);
    const uint32_t budget = 4u * nbins + 260u;
    if (nw * ny > budget) ny = max(1u, budget / nw);
    W.seg_nb[g] = nw * ny;
    W.seg_dim[g] = make_int4((int)nw, (int)ny, iw0, k + 9);
    W.seg_geo[g] = make_float4(ldexpf((float)iw0, k), ldexpf(1.0f, -k), -Q.yext[r], (float)ny / yext);
  }
}

__device__ __forceinline__ uint32_t seg_bin(const Work& W, int g, float y, float w, int& iw) {
  const int4 dim = W.seg_dim[g];
  const float4 geo = W.seg_geo[g];
  iw = bin_of(w, geo.x, geo.y, dim.x);
  const int iy = bin_of(y, geo.z, geo.w, dim.y);
  return W.seg_bb[g] + (uint32_t)(iw * dim.y + iy);
}

// one_pass_only: skip batches that the two-pass kernels place (the main path launches both forms)
__global__ void __launch_bounds__(256) k_bin_rank(Work W, int one_pass_only) {
  const BatchDesc* B = W.batch;
  const long long ntot = B->ntot;
  if (one_pass_only && ntot > kTwoPassMin) return;
  const uint32_t bcap = (uint32_t)W.bcap;
  if (W.cnt->n_bins > bcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&W.cnt->err, kErrBins);
    return;
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += (long long)gridDim.x * blockDim.x) {
    int fi, iw;
    long long j;
    const InHit h = read_input(B, W.packed, i, fi, j);
    if (!h.ok) continue;
    W.rank[i] = atomicAdd(&W.bin_start[seg_bin(W, h.g, h.y, h.w, iw)], 1u);
  }
}

__global__ void __launch_bounds__(256) k_scatter(Work W, int one_pass_only) {
  const BatchDesc* B = W.batch;
  const long long ntot = B->ntot;
  if (one_pass_only && ntot > kTwoPassMin) return;
  if (W.cnt->n_bins > (uint32_t)W.bcap) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += (long long)gridDim.x * blockDim.x) {
    int fi, iw;
    long long j;
    const InHit h = read_input(B, W.packed, i, fi, j);
    if (!h.ok) continue;
    const uint32_t p = W.bin_start[seg_bin(W, h.g, h.y, h.w, iw)] + W.rank[i];
    if (W.packed) {
      const int4 dim = W.seg_dim[h.g];
      const uint32_t qy = (uint32_t)rintf((h.y + 64.0f) * 512.0f);
      const int qw = (int)rintf(h.w * 512.0f) - col_base(dim.z, dim.w, iw);
      W.hq[p] = qy | ((uint32_t)qw << 16);
      W.hcol[p] = (uint16_t)iw;
    } else {
      W.hyw[p] = make_float2(h.y, h.w);
    }
    W.horig[p] = (uint32_t)j;
  }
}

// ---- Two-pass placement into grid order (the main path). Pass A appends each cluster, as a
// 16-byte record (y, w, batch index, segment), to its segment's contiguous range: the ranges are
// the exclusive scan of the per-segment counts, and each segment's cursor grows by warp-aggregated
// atomics, so the writes of all warps form one append stream per segment whose open 32-byte
// sectors stay in L2. Pass B takes one segment per block: its records are read in order, ranked in
// their bins (atomics on the segment's own bin counters), and after the bin scan written to their
// sorted positions, which are the same range [seg_start, seg_start + n) of the segment; the random
// accesses of a block stay inside one segment's few hundred kilobytes.
__global__ void __launch_bounds__(256) k_seg_bucket(Work W) {
  const BatchDesc* B = W.batch;
  const long long ntot = B->ntot;
  if (ntot <= kTwoPassMin) return;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // warp-uniform trip count: every lane takes part in the aggregation
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < ntot; base += stride) {
    const long long i = base + lane;
    InHit h{0, 0.f, 0.f, false};
    if (i < ntot) {
      int fi;
      long long j;
      h = read_input(B, W.packed, i, fi, j);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, h.ok ? h.g : -1 - lane);
    const int leader = __ffs(peers) - 1;
    uint32_t off = 0;
    if (h.ok && lane == leader) off = atomicAdd(&W.seg_cur[h.g], (uint32_t)__popc(peers));
    off = __shfl_sync(0xffffffffu, off, leader);
    if (h.ok) {
      const uint32_t p = W.seg_start[h.g] + off + (uint32_t)__popc(peers & ((1u << lane) - 1u));
      W.rec[p] = make_uint4(__float_as_uint(h.y), __float_as_uint(h.w), (uint32_t)i, (uint32_t)h.g);
    }
  }
}

// The bins the one-pass placement zeroes and scans (the per-segment passes do both per segment).
__global__ void k_one_pass_bins(Work W) {
  W.cnt->n_bins_1p = W.batch->ntot <= kTwoPassMin ? W.cnt->n_bins : 0u;
}

// One block per segment: its bin counters zeroed, its records ranked in their bins (atomics on the
// counters), then the counters turned in place into the bins' first sorted positions: their
// exclusive scan plus the segment's first position (a segment's bins and its positions follow the
// same segment order, so this equals the scan over all bins). Block 0 also writes the end of the
// last bin, bin_start[n_bins] = the batch's placed clusters.
constexpr int kBinItems = 4;
__global__ void __launch_bounds__(1024, 2) k_bin_rank_seg(Work W) {
  if (W.batch->ntot <= kTwoPassMin) return;
  if (W.cnt->n_bins > (uint32_t)W.bcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&W.cnt->err, kErrBins);
    return;
  }
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t block_total;
  const int nseg = (int)W.cnt->nseg;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) W.bin_start[W.cnt->n_bins] = W.seg_start[nseg];
  for (int g = blockIdx.x; g < nseg; g += gridDim.x) {
    const uint32_t bb = W.seg_bb[g], nb = W.seg_nb[g];
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) W.bin_start[bb + j] = 0u;
    __syncthreads();
    const uint32_t p1 = W.seg_start[g + 1];
    // kSegUnroll records per thread in flight: their loads, then their atomics, then the ranks
    for (uint32_t b = W.seg_start[g] + threadIdx.x; b < p1; b += blockDim.x * kSegUnroll) {
      uint4 r[kSegUnroll];
      uint32_t rk[kSegUnroll];
#pragma unroll
      for (int u = 0; u < kSegUnroll; ++u) {
        const uint32_t p = b + u * blockDim.x;
        r[u] = p < p1 ? W.rec[p] : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < kSegUnroll; ++u) {
        int iw;
        if (b + u * blockDim.x < p1)
          rk[u] = atomicAdd(&W.bin_start[seg_bin(W, g, __uint_as_float(r[u].x), __uint_as_float(r[u].y), iw)], 1u);
      }
#pragma unroll
      for (int u = 0; u < kSegUnroll; ++u)
        if (b + u * blockDim.x < p1) W.rank[b + u * blockDim.x] = rk[u];
    }
    __syncthreads();
    // exclusive scan of the segment's counters in place, kBinItems consecutive bins per thread
    uint32_t carry = W.seg_start[g];
    for (uint32_t base = 0; base < nb; base += blockDim.x * kBinItems) {
      const uint32_t i0 = base + threadIdx.x * kBinItems;
      uint32_t v[kBinItems], sum = 0;
#pragma unroll
      for (int k = 0; k < kBinItems; ++k) {
        v[k] = i0 + k < nb ? __ldcg(&W.bin_start[bb + i0 + k]) : 0u;
        sum += v[k];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) warp_sums[wid] = x;
      __syncthreads();
      if (wid == 0) {
        const uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
        uint32_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
          if (lane >= o) z += y;
        }
        warp_sums[lane] = z - w;
        if (lane == 31) block_total = z;
      }
      __syncthreads();
      uint32_t run = carry + warp_sums[wid] + (x - sum);
#pragma unroll
      for (int k = 0; k < kBinItems; ++k) {
        if (i0 + k < nb) W.bin_start[bb + i0 + k] = run;
        run += v[k];
      }
      carry += block_total;
      __syncthreads();
    }
  }
}

// kScatterParts consecutive blocks share a segment (each takes an interleaved share of its
// records), so fewer segments are in flight at once and their random-access targets (grid positions
// and bin starts) stay in L2 while the stores to a line accumulate. The grid is a multiple of it.
__global__ void __launch_bounds__(1024) k_scatter_seg(Work W) {
  if (W.batch->ntot <= kTwoPassMin || W.cnt->n_bins > (uint32_t)W.bcap) return;
  const BatchDesc* B = W.batch;
  const int nseg = (int)W.cnt->nseg;
  const int part = (int)(blockIdx.x % kScatterParts);
  const int slots = (int)(gridDim.x / kScatterParts);
  const uint32_t step = blockDim.x * kScatterParts;
  for (int g = (int)(blockIdx.x / kScatterParts); g < nseg; g += slots) {
    const uint32_t p1 = W.seg_start[g + 1];
    const long long foff = B->f[g / kSegPerFrame].off;
    // kSegUnroll records per thread in flight: their loads, then their bins' starts, then the stores
    for (uint32_t b = W.seg_start[g] + part * blockDim.x + threadIdx.x; b < p1; b += step * kSegUnroll) {
      uint4 r[kSegUnroll];
      uint32_t rk[kSegUnroll], q[kSegUnroll];
      int iw[kSegUnroll];
#pragma unroll
      for (int u = 0; u < kSegUnroll; ++u) {
        const uint32_t p = b + u * step;
        r[u] = p < p1 ? W.rec[p] : make_uint4(0u, 0u, 0u, 0u);
        rk[u] = p < p1 ? W.rank[p] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kSegUnroll; ++u)
        if (b + u * step < p1)
          q[u] = W.bin_start[seg_bin(W, g, __uint_as_float(r[u].x), __uint_as_float(r[u].y), iw[u])] + rk[u];
#pragma unroll
      for (int u = 0; u < kSegUnroll; ++u) {
        if (b + u * step >= p1) continue;
        const float y = __uint_as_float(r[u].x), w = __uint_as_float(r[u].y);
        if (W.packed) {
          const int4 dim = W.seg_dim[g];
          const uint32_t qy = (uint32_t)rintf((y + 64.0f) * 512.0f);
          const int qw = (int)rintf(w * 512.0f) - col_base(dim.z, dim.w, iw[u]);
          W.hq[q[u]] = qy | ((uint32_t)qw << 16);
          W.hcol[q[u]] = (uint16_t)iw[u];
        } else {
          W.hyw[q[u]] = make_float2(y, w);
        }
        W.horig[q[u]] = (uint32_t)((long long)r[u].z - foff);
      }
    }
  }
}

}  // namespace tpc
