// k_links.cu — K2 neighbour finding, K3 cleaning, K4 start hits and their canonical order.
//
// K2 (cellular-automaton neighbour finding): for every hit i of row r (1 <= r <= 150) the pair
// (d in row r-1, u in row r+1) inside the slope windows that minimises the mid-point deviation
// chi_n = (y_i - y_mid)^2 + (w_i - w_mid)^2, accepted if chi_n <= chi_n_max; ties go to the
// smaller (w, y, input index) of d, then of u. A CTA takes one segment (frame, sector, row) at a
// time in chunks of blockDim hits; for each chunk the windows of the two adjacent rows are one
// contiguous range each, which thread 0 stages into shared memory with 1-D bulk TMA copies
// (cp.async.bulk, completion on an mbarrier; no multicast). Each thread then scans its own
// candidate sub-ranges out of shared memory. A range too large for the stage is read from global
// memory instead (same arithmetic, same result).
//
// K3 keeps only reciprocal links and counts start hits per segment; K4 writes the start hits
// (cleaned up link, no down link, chain of >= lmin hits) by a block-wide ballot/scan compaction in
// sorted order; K4b puts the start hits into canonical order (frame, sector, row-rank) and computes
// each start hit's rank, the tie-break of the tracklet selection key.
#include "tpc_dev.cuh"

namespace tpc {

constexpr int kK2Stage = 2048;  // staged hits per adjacent row (float2)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (about a second of device time at most)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && clock64() - t0 > 2000000000LL) return false;
  }
}

// Find the best (d, u) pair of hit (yi, wi, oi); rows given as [p0, p1) position ranges, each read
// from shared memory (stage, base) when the range lies inside the stage, else from global memory.
struct RowView {
  const float2* stage;
  int base, count;  // staged positions [base, base + count)
};

__device__ __forceinline__ float2 load_hit(const Work& W, const RowView& v, int p) {
  if (p >= v.base && p < v.base + v.count) return v.stage[p - v.base];
  return W.hyw[p];
}

__device__ __forceinline__ bool pair_key_less(const Work& W, int d, int u, int bd, int bu) {
  // tie of chi_n: smaller (w, y, input index) of d, then of u
  if (d != bd) {
    const float2 a = W.hyw[d], b = W.hyw[bd];
    return key_less(a.y, a.x, W.horig[d], b.y, b.x, W.horig[bd]);
  }
  const float2 a = W.hyw[u], b = W.hyw[bu];
  return key_less(a.y, a.x, W.horig[u], b.y, b.x, W.horig[bu]);
}

__device__ __forceinline__ void row_range(const Work& W, int g, float lo, float hi, int& p0, int& p1) {
  const uint32_t bb = W.seg_bb[g];
  const int nb = (int)W.seg_nb[g];
  const float2 geo = W.seg_geo[g];
  const int b0 = bin_of(lo, geo.x, geo.y, nb), b1 = bin_of(hi, geo.x, geo.y, nb);
  p0 = (int)W.bin_start[bb + b0];
  p1 = (int)W.bin_start[bb + b1 + 1];
}

__global__ void __launch_bounds__(256) k_neighbours(Work W, DevParams Q) {
  extern __shared__ __align__(16) float2 k2_smem[];
  float2* stage_dn = k2_smem;
  float2* stage_up = k2_smem + kK2Stage + 2;
  __shared__ __align__(8) uint64_t bar;
  __shared__ float red_lo[8], red_hi[8];
  __shared__ int st_base[2], st_count[2];
  __shared__ int s_abort;
  const BatchDesc* B = W.batch;
  const int nseg = B->nf * kSegPerFrame;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
  }
  __syncthreads();
  uint32_t parity = 0;
  for (int g = blockIdx.x; g < nseg; g += gridDim.x) {
    const int r = (g % kSegPerFrame) % kNRow;
    const int a = (int)W.bin_start[W.seg_bb[g]];
    const int b = (int)W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    if (r == 0 || r == kNRow - 1) {
      for (int i = a + threadIdx.x; i < b; i += blockDim.x) W.links[i] = make_int2(-1, -1);
      continue;
    }
    const float wy_dn = Q.wy_dn[r], ww_dn = Q.ww_dn[r], wy_up = Q.wy_up[r], ww_up = Q.ww_up[r];
    const float fm = Q.f_mid[r];
    for (int c0 = a; c0 < b; c0 += blockDim.x) {
      const int i = c0 + threadIdx.x;
      const bool valid = i < b;
      float2 hi = valid ? W.hyw[i] : make_float2(0.f, 0.f);
      // chunk w range (block reduction)
      float lo_w = valid ? hi.y : 3.0e38f, hi_w = valid ? hi.y : -3.0e38f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo_w = fminf(lo_w, __shfl_xor_sync(0xffffffffu, lo_w, o));
        hi_w = fmaxf(hi_w, __shfl_xor_sync(0xffffffffu, hi_w, o));
      }
      if ((threadIdx.x & 31) == 0) { red_lo[threadIdx.x >> 5] = lo_w; red_hi[threadIdx.x >> 5] = hi_w; }
      __syncthreads();
      if (threadIdx.x == 0) {
        float l = red_lo[0], h = red_hi[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { l = fminf(l, red_lo[k]); h = fmaxf(h, red_hi[k]); }
        const float amax = fmaxf(fabsf(l), fabsf(h));
        uint32_t bytes = 0;
        for (int side = 0; side < 2; ++side) {
          const float Ww = side == 0 ? ww_dn : ww_up;
          const float pad = win_pad(amax, Ww);
          int p0, p1;
          row_range(W, g + (side == 0 ? -1 : 1), (l - Ww) - pad, (h + Ww) + pad, p0, p1);
          const int q0 = p0 & ~1, q1 = (p1 + 1) & ~1;
          if (q1 > q0 && q1 - q0 <= kK2Stage) {
            st_base[side] = q0;
            st_count[side] = q1 - q0;
            bytes += (uint32_t)(q1 - q0) * 8u;
          } else {
            st_base[side] = 0;
            st_count[side] = 0;
          }
        }
        mbar_arrive_expect_tx(&bar, bytes);
        if (st_count[0]) tma_load_1d(stage_dn, W.hyw + st_base[0], (uint32_t)st_count[0] * 8u, &bar);
        if (st_count[1]) tma_load_1d(stage_up, W.hyw + st_base[1], (uint32_t)st_count[1] * 8u, &bar);
      }
      __syncthreads();
      if (!mbar_wait_bounded(&bar, parity)) {
        if (threadIdx.x == 0) { atomicOr(&W.cnt->err, kErrTimeout); s_abort = 1; }
      }
      parity ^= 1u;
      RowView vd{stage_dn, st_base[0], st_count[0]};
      RowView vu{stage_up, st_base[1], st_count[1]};
      if (valid) {
        const float yi = hi.x, wi = hi.y;
        int dp0, dp1, up0, up1;
        row_range(W, g - 1, (wi - ww_dn) - win_pad(wi, ww_dn), (wi + ww_dn) + win_pad(wi, ww_dn), dp0, dp1);
        row_range(W, g + 1, (wi - ww_up) - win_pad(wi, ww_up), (wi + ww_up) + win_pad(wi, ww_up), up0, up1);
        float best = __int_as_float(0x7f800000);
        int bd = -1, bu = -1;
        for (int d = dp0; d < dp1; ++d) {
          const float2 hd = load_hit(W, vd, d);
          if (!(fabsf(hd.x - yi) <= wy_dn && fabsf(hd.y - wi) <= ww_dn)) continue;
          for (int u = up0; u < up1; ++u) {
            const float2 hu = load_hit(W, vu, u);
            if (!(fabsf(hu.x - yi) <= wy_up && fabsf(hu.y - wi) <= ww_up)) continue;
            const float py = hd.x + (hu.x - hd.x) * fm;
            const float pw = hd.y + (hu.y - hd.y) * fm;
            const float ey = yi - py, ew = wi - pw;
            const float chi = ey * ey + ew * ew;
            bool better;
            if (bd < 0 || chi < best) better = true;
            else if (chi > best) better = false;
            else better = pair_key_less(W, d, u, bd, bu);
            if (better) { best = chi; bd = d; bu = u; }
          }
        }
        W.links[i] = (bd >= 0 && best <= Q.chi_n_max) ? make_int2(bd, bu) : make_int2(-1, -1);
      }
      // the stage is rewritten by the async proxy next: order the generic reads before it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (s_abort) return;
    }
  }
}

// ------------------------------------------------------------------------------------ K3
__device__ __forceinline__ int clean_up(const int2* L, int j) {
  const int u = L[j].y;
  return (u >= 0 && L[u].x == j) ? u : -1;
}
__device__ __forceinline__ int clean_dn(const int2* L, int j) {
  const int d = L[j].x;
  return (d >= 0 && L[d].y == j) ? d : -1;
}

__device__ __forceinline__ int block_sum(int v, int* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int s = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(256) k_clean(Work W, DevParams Q) {
  __shared__ int red[8];
  const BatchDesc* B = W.batch;
  const int nseg = B->nf * kSegPerFrame;
  for (int g = blockIdx.x; g < nseg; g += gridDim.x) {
    const int a = (int)W.bin_start[W.seg_bb[g]];
    const int b = (int)W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    int count = 0;
    for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
      const int u = clean_up(W.links, i), d = clean_dn(W.links, i);
      W.clinks[i] = make_int2(d, u);
      if (u >= 0 && d < 0) {
        int len = 2;
        for (int h = clean_up(W.links, u); h >= 0 && len < Q.lmin; h = clean_up(W.links, h)) ++len;
        if (len >= Q.lmin) ++count;
      }
    }
    const int tot = block_sum(count, red);
    if (threadIdx.x == 0) W.seg_nstart[g] = (uint32_t)tot;
  }
}

// ------------------------------------------------------------------------------------ K4
__global__ void __launch_bounds__(256) k_starts(Work W, DevParams Q) {
  __shared__ int warp_off[8];
  __shared__ int s_total;
  const BatchDesc* B = W.batch;
  const int nseg = B->nf * kSegPerFrame;
  const uint32_t tcap = (uint32_t)W.tcap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = blockIdx.x; g < nseg; g += gridDim.x) {
    const int a = (int)W.bin_start[W.seg_bb[g]];
    const int b = (int)W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    uint32_t out = W.seg_nstart[g];
    const uint32_t bb = W.seg_bb[g];
    const int nb = (int)W.seg_nb[g];
    const float2 geo = W.seg_geo[g];
    for (int c0 = a; c0 < b; c0 += blockDim.x) {
      const int i = c0 + threadIdx.x;
      bool st = false;
      if (i < b) {
        const int2 c = W.clinks[i];
        if (c.y >= 0 && c.x < 0) {
          int len = 2;
          for (int h = W.clinks[c.y].y; h >= 0 && len < Q.lmin; h = W.clinks[h].y) ++len;
          st = len >= Q.lmin;
        }
      }
      const uint32_t m = __ballot_sync(0xffffffffu, st);
      if (lane == 0) warp_off[warp] = __popc(m);
      __syncthreads();
      if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { int v = warp_off[k]; warp_off[k] = s; s += v; }
        s_total = s;
      }
      __syncthreads();
      if (st) {
        const uint32_t pos = out + (uint32_t)warp_off[warp] + (uint32_t)__popc(m & ((1u << lane) - 1u));
        if (pos < tcap) {
          const float w = W.hyw[i].y;
          W.starts_raw[pos] = make_uint4((uint32_t)i, (uint32_t)g, bb + (uint32_t)bin_of(w, geo.x, geo.y, nb), 0u);
        }
      }
      out += (uint32_t)s_total;
      __syncthreads();
    }
  }
}

// K4b: canonical order of start hits and their rank in the sector (rows, then (w, y, input index))
__global__ void __launch_bounds__(256) k_start_order(Work W) {
  const uint32_t n = min(W.cnt->n_starts, (uint32_t)W.tcap);
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint4 e = W.starts_raw[p];
    const int i = (int)e.x, g = (int)e.y;
    const uint32_t Bn = e.z;
    const float2 hi = W.hyw[i];
    const uint32_t oi = W.horig[i];
    // run of start entries sharing the bin (contiguous in sorted order)
    uint32_t lo = p, hiq = p;
    while (lo > 0 && W.starts_raw[lo - 1].z == Bn) --lo;
    while (hiq + 1 < n && W.starts_raw[hiq + 1].z == Bn) ++hiq;
    uint32_t before = 0;
    for (uint32_t q = lo; q <= hiq; ++q) {
      if (q == p) continue;
      const int j = (int)W.starts_raw[q].x;
      const float2 hj = W.hyw[j];
      if (key_less(hj.y, hj.x, W.horig[j], hi.y, hi.x, oi)) ++before;
    }
    // rank of the hit within its bin, row and sector
    const uint32_t b0 = W.bin_start[Bn], b1 = W.bin_start[Bn + 1];
    uint32_t inbin = 0;
    for (uint32_t h = b0; h < b1; ++h) {
      if ((int)h == i) continue;
      const float2 hh = W.hyw[h];
      if (key_less(hh.y, hh.x, W.horig[h], hi.y, hi.x, oi)) ++inbin;
    }
    const int r = (g % kSegPerFrame) % kNRow;
    const uint32_t seg_first = W.bin_start[W.seg_bb[g]];
    const uint32_t sec_first = W.bin_start[W.seg_bb[g - r]];
    const uint32_t rank = (b0 - sec_first) + inbin;
    (void)seg_first;
    W.starts[lo + before] = make_uint4((uint32_t)i, (uint32_t)g, rank, 0u);
  }
}

}  // namespace tpc
