// k_links.cu — K2 neighbour finding, K3 cleaning, K4 start hits and their canonical order.
//
// K2 (cellular-automaton neighbour finding): for every hit i of row r (1 <= r <= 150) the pair
// (d in row r-1, u in row r+1) inside the slope windows that minimises the mid-point deviation
// chi_n = (y_i - y_mid)^2 + (w_i - w_mid)^2, accepted if chi_n <= chi_n_max; ties go to the
// smaller (w, y, input index) of d, then of u. Work is split into chunks of 32 consecutive hits of
// one segment (frame, sector, row), listed in segment work-item order (inner rows first) by
// k_chunk_count / scan / k_chunk_fill; each warp takes the next chunk from a device counter, so warps
// never wait for one another. The w-columns of the two adjacent rows that the 32 windows touch are
// one contiguous range each, which lane 0 stages into the warp's shared-memory slots with 1-D bulk
// TMA copies (cp.async.bulk, completion on the warp's mbarrier; no multicast).
// Each lane then scans its own candidate bins (one contiguous range per w-column) out of shared
// memory. A range too large for a slot is read from global memory instead (same arithmetic, same
// result).
//
// K3 keeps only reciprocal links, marks the start hits (cleaned up link, no down link, chain of
// >= lmin hits) and counts them per segment; K4 writes the start hits by a block-wide ballot/scan
// compaction in sorted order; K4b puts the start hits into canonical order (frame, sector, row-rank) and computes
// each start hit's rank, the tie-break of the tracklet selection key.
#include "tpc_dev.cuh"

namespace tpc {


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
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait: gives up after limit_ns of device time (the staging copies: one second)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
  }
}

// Diagnostic of the bounded wait: one warp waits on a barrier whose announced transfer is never
// issued, so the phase cannot complete; the wait gives up after limit_ns and the warp records it in
// *status (1: timed out, 0: completed) and exits. No copy is in flight at any time.
__global__ void __launch_bounds__(32) k_wait_probe(uint32_t* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_arrive_expect_tx(&bar, 16u);
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  const bool all = __all_sync(0xffffffffu, ok);
  if (threadIdx.x == 0) *status = all ? 0u : 1u;
}
void launch_wait_probe(uint32_t* status, unsigned long long limit_ns, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(status, limit_ns);
}

// A row range staged in shared memory: positions [base, base + count) (FP32 float2 records, or
// 16-bit uint32 records); positions outside it are read from global memory.
struct RowView {
  const void* stage;
  int base, count;
};


// candidate record at position p: from the stage when the side is staged (then every window of the
// chunk lies inside it), else from global memory
template <bool kPacked>
__device__ __forceinline__ float2 cand_at(const Work& W, const RowView& v, bool staged, int p, int cbase) {
  if (staged) {
    if (kPacked) return unpack_hit(reinterpret_cast<const uint32_t*>(v.stage)[p - v.base], cbase);
    return reinterpret_cast<const float2*>(v.stage)[p - v.base];
  }
  return kPacked ? unpack_hit(W.hq[p], cbase) : W.hyw[p];
}

// tie of chi_n: smaller (w, y, input index) of d, then of u (d, bd in segment gd; u, bu in gu)
template <bool kPacked>
__device__ __forceinline__ bool pair_key_less(const Work& W, int gd, int gu, int d, int u, int bd, int bu) {
  const int g = d != bd ? gd : gu;
  const int x = d != bd ? d : u, y = d != bd ? bd : bu;
  const float2 a = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, g, x);
  const float2 b = hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, g, y);
  return key_less(a.y, a.x, W.horig[x], b.y, b.x, W.horig[y]);
}

// positions [p0, p1) of the w-columns of segment g touched by |w - wc| <= W for wc in [lo, hi]; iw0
// is the first of those columns
__device__ __forceinline__ void column_range(const Work& W, int g, float lo, float hi, int& p0, int& p1, int& iw0) {
  const int4 dim = W.seg_dim[g];
  const float4 geo = W.seg_geo[g];
  const uint32_t bb = W.seg_bb[g];
  iw0 = bin_of(lo, geo.x, geo.y, dim.x);
  const int iw1 = bin_of(hi, geo.x, geo.y, dim.x);
  p0 = (int)W.bin_start[bb + (uint32_t)(iw0 * dim.y)];
  p1 = (int)W.bin_start[bb + (uint32_t)((iw1 + 1) * dim.y)];
}

// One warp takes 32 consecutive hits of a row (a chunk); with use_tma >= 1 lane 0 stages the
// w-columns of rows r-1 and r+1 that the 32 windows touch into the warp's own shared-memory slots
// (two bulk copies, one mbarrier per warp), so warps never wait for one another.
//   use_tma 0, 1: each lane walks its own windows, one flat loop over each window's positions
//                 across its w-columns (from the stage when its side is staged: the union of the 32
//                 windows lies inside it; through L1 otherwise), listing the positions inside its
//                 row r+1 and row r-1 windows, then tests every pair of the two lists in one loop;
//   use_tma 2:    when both ranges are staged, the warp scans each staged range once, all lanes
//                 together (one candidate per iteration, broadcast from shared memory): a lane whose
//                 window holds the candidate appends it to its own list; each lane then pairs its
//                 two lists. A lane whose list overflows walks its own bins instead.
// All modes give the same result: the grid only bounds the candidates, the exact window test decides.
constexpr int kK2Slot = 256;  // staged FP32 records per adjacent row per warp (twice as many 16-bit)
constexpr int kK2Cap = 6;     // candidates per lane and adjacent row listed by the converged scan (mode 2)
constexpr int kK2Own = 16;    // candidate positions per lane and adjacent row listed by the own walk

// Shared memory of one warp, by staging mode: the mbarrier (16 B), the two staging slots (modes 1
// and 2; 16-byte aligned, bulk-copy destinations), then one list region: the converged scan's
// per-lane candidate lists of both adjacent rows (mode 2), or the own walk's per-lane position
// lists of both rows (every mode; a chunk uses one or the other: the own walk runs after a
// converged scan only when the scan's lists overflowed, and then replaces them).
constexpr int kK2ListBytes = kK2Cap * 32 * (8 + 4);
constexpr int kK2OwnBytes = 2 * kK2Own * 32 * 4;
__host__ __device__ constexpr int k2_warp_bytes(int mode) {
  return 16 + (mode >= 1 ? 2 * (kK2Slot + 2) * 8 : 0) +
         (mode == 2 && 2 * kK2ListBytes > kK2OwnBytes ? 2 * kK2ListBytes : kK2OwnBytes);
}
struct K2Warp {
  uint64_t* bar;
  float2* stage[2];  // [0] row r-1, [1] row r+1
  float2* cand[2];   // converged scan: [side][n * 32 + lane]
  int* pos[2];
  int* own[2];       // own walk: [side][n * 32 + lane] candidate positions
  __device__ K2Warp(unsigned char* base, int mode) {
    bar = reinterpret_cast<uint64_t*>(base);
    unsigned char* p = base + 16;
    stage[0] = reinterpret_cast<float2*>(p);
    stage[1] = stage[0] + (kK2Slot + 2);
    if (mode >= 1) p += 2 * (kK2Slot + 2) * 8;
    own[0] = reinterpret_cast<int*>(p);
    own[1] = own[0] + kK2Own * 32;
    cand[1] = reinterpret_cast<float2*>(p);
    pos[1] = reinterpret_cast<int*>(p + kK2Cap * 32 * 8);
    p += kK2ListBytes;
    cand[0] = reinterpret_cast<float2*>(p);  // used in mode 2 only
    pos[0] = reinterpret_cast<int*>(p + kK2Cap * 32 * 8);
  }
};

// Positions inside a lane's window of one adjacent row, listed in own[n * 32 + lane] for n < kK2Own:
// one flat loop over the window's positions, a w-column's bin range after the other, so a warp
// iterates as often as its lane with the most positions (nested column / position loops would
// iterate, column by column, as often as the lane with the most positions in that column). Returns
// the lane's count of positions inside the window (beyond kK2Own counted, not listed).
template <bool kPacked>
__device__ __forceinline__ int list_window(const Work& W, const GridWin& q, const RowView& v, bool staged, float yi,
                                           float wi, float wy, float ww, int* own, int lane) {
  int n = 0;
  int cw = q.iw0;
  uint32_t col = q.bb + (uint32_t)(cw * q.ny);
  int p = (int)W.bin_start[col + q.iy0], pe = (int)W.bin_start[col + q.iy1 + 1];
  // the next column's range is loaded one column ahead, so its latency overlaps this column's tests
  int np = 0, npe = 0;
  if (cw < q.iw1) {
    np = (int)W.bin_start[col + (uint32_t)q.ny + q.iy0];
    npe = (int)W.bin_start[col + (uint32_t)q.ny + q.iy1 + 1];
  }
  int cb = col_base(q.cw0, q.cshift, cw);
  for (;;) {
    if (p >= pe) {
      if (++cw > q.iw1) break;
      col += (uint32_t)q.ny;
      p = np;
      pe = npe;
      if (cw < q.iw1) {
        np = (int)W.bin_start[col + (uint32_t)q.ny + q.iy0];
        npe = (int)W.bin_start[col + (uint32_t)q.ny + q.iy1 + 1];
      }
      cb = col_base(q.cw0, q.cshift, cw);
      continue;
    }
    const float2 h = cand_at<kPacked>(W, v, staged, p, cb);
    if (fabsf(h.x - yi) <= wy && fabsf(h.y - wi) <= ww) {
      if (n < kK2Own) own[n * 32 + lane] = p;
      ++n;
    }
    ++p;
  }
  return n;
}

// (y, w) of a listed candidate position of the window q (16-bit storage: its column from hcol)
template <bool kPacked>
__device__ __forceinline__ float2 cand_of(const Work& W, const GridWin& q, const RowView& v, bool staged, int p) {
  return cand_at<kPacked>(W, v, staged, p, kPacked ? col_base(q.cw0, q.cshift, (int)W.hcol[p]) : 0);
}

template <bool kPacked>
__device__ __forceinline__ void pair_step(const Work& W, int gd, int gu, float yi, float wi, float fm,
                                          const float2 hd, int d, const float2 hu, int u, float& best, int& bd,
                                          int& bu) {
  const float py = hd.x + (hu.x - hd.x) * fm;
  const float pw = hd.y + (hu.y - hd.y) * fm;
  const float ey = yi - py, ew = wi - pw;
  const float chi = ey * ey + ew * ew;
  bool better;
  if (bd < 0 || chi < best) better = true;
  else if (chi > best) better = false;
  else better = pair_key_less<kPacked>(W, gd, gu, d, u, bd, bu);
  if (better) { best = chi; bd = d; bu = u; }
}

// Converged scan of the staged positions [p0, p1) of segment gs (staged from position base): every
// lane tests every candidate against its own window and lists the ones inside; returns the lane's
// count (entries beyond kK2Cap are counted, not kept).
template <bool kPacked>
__device__ __forceinline__ int scan_staged(const Work& W, K2Warp& S, int side, int gs, int p0, int p1, int base,
                                           int iw0, bool valid, float yi, float wi, float wy, float ww, int lane) {
  int n = 0;
  int cbase = 0, next = 0, iw = iw0, ny = 0, cw0 = 0, cshift = 0;
  uint32_t bb = 0;
  if (kPacked && p0 < p1) {
    const int4 dim = W.seg_dim[gs];
    bb = W.seg_bb[gs];
    ny = dim.y; cw0 = dim.z; cshift = dim.w;
    cbase = col_base(cw0, cshift, iw);
    next = (int)W.bin_start[bb + (uint32_t)((iw + 1) * ny)];
  }
  for (int p = p0; p < p1; ++p) {
    float2 h;
    if (kPacked) {
      while (p >= next) {  // next w-column (warp-uniform)
        ++iw;
        cbase = col_base(cw0, cshift, iw);
        next = (int)W.bin_start[bb + (uint32_t)((iw + 1) * ny)];
      }
      h = unpack_hit(reinterpret_cast<const uint32_t*>(S.stage[side])[p - base], cbase);
    } else {
      h = S.stage[side][p - base];
    }
    if (valid && fabsf(h.x - yi) <= wy && fabsf(h.y - wi) <= ww) {
      if (n < kK2Cap) {
        S.cand[side][n * 32 + lane] = h;
        S.pos[side][n * 32 + lane] = p;
      }
      ++n;
    }
  }
  return n;
}

// chunks of 32 hits of every segment work item (rows 0 and 151 too: their links are cleared)
__global__ void __launch_bounds__(256) k_chunk_count(Work W) {
  const int nf = W.batch->nf;
  const uint32_t nseg = W.cnt->nseg;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nseg; k += gridDim.x * blockDim.x) {
    const int g = segment_of_item((int)k, nf);
    const uint32_t a = W.bin_start[W.seg_bb[g]], b = W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    W.k2_off[k] = (b - a + 31u) / 32u;
  }
}
// (segment, first position) of every chunk, from the scanned counts
__global__ void __launch_bounds__(256) k_chunk_fill(Work W) {
  const int nf = W.batch->nf;
  const uint32_t nseg = W.cnt->nseg;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nseg; k += gridDim.x * blockDim.x) {
    const int g = segment_of_item((int)k, nf);
    const uint32_t a = W.bin_start[W.seg_bb[g]];
    const uint32_t c1 = W.k2_off[k + 1] < (uint32_t)W.k2cap ? W.k2_off[k + 1] : (uint32_t)W.k2cap;
    for (uint32_t j = W.k2_off[k]; j < c1; ++j) W.k2_tab[j] = make_uint2((uint32_t)g, a + 32u * (j - W.k2_off[k]));
  }
}

template <bool kPacked, int kWarps>
__global__ void __launch_bounds__(32 * kWarps) k_neighbours(Work W, DevParams Q, int use_tma) {
  constexpr int kRec = kPacked ? 4 : 8;       // bytes per staged record
  constexpr int kAlign = 16 / kRec;           // records per 16 bytes
  constexpr int kSlot = kPacked ? 2 * kK2Slot : kK2Slot;
  extern __shared__ __align__(16) unsigned char k2_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  K2Warp S(k2_smem + warp * k2_warp_bytes(use_tma), use_tma);
  if (lane == 0) mbar_init(S.bar, 1);
  __syncwarp();
  uint32_t parity = 0;
  const uint32_t nch = W.cnt->n_chunks < (uint32_t)W.k2cap ? W.cnt->n_chunks : (uint32_t)W.k2cap;
  // lane 0 takes the next chunk one iteration ahead, so the atomic's latency overlaps the work
  uint32_t k_next = 0;
  if (lane == 0) k_next = atomicAdd(&W.cnt->k2_next, 1u);
  for (;;) {
    const uint32_t k = __shfl_sync(0xffffffffu, k_next, 0);
    if (k >= nch) break;
    const uint2 e = W.k2_tab[k];
    if (lane == 0) k_next = atomicAdd(&W.cnt->k2_next, 1u);
    const int g = (int)e.x, c0 = (int)e.y;
    const int r = (g % kSegPerFrame) % kNRow;
    const int b = (int)W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    if (r == 0 || r == kNRow - 1) {
      if (c0 + lane < b) W.links[c0 + lane] = make_int2(-1, -1);
      continue;
    }
    const float wy_dn = Q.wy_dn[r], ww_dn = Q.ww_dn[r], wy_up = Q.wy_up[r], ww_up = Q.ww_up[r];
    const float fm = Q.f_mid[r];
    const int i = c0 + lane;
    const bool valid = i < b;
    const float2 hi = valid ? hit_by_index<kPacked>(W.hyw, W.hq, W.hcol, W.seg_dim, g, i) : make_float2(0.f, 0.f);
    // per side: p0, p1, iw0, staged base (staging modes only: without staging each lane reads its
    // own window through L1, and the chunk needs neither the ranges nor the barrier)
    int rng[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int cnt0 = 0, cnt1 = 0, conv = 0;
    if (use_tma) {
      float lo_w = valid ? hi.y : 3.0e38f, hi_w = valid ? hi.y : -3.0e38f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo_w = fminf(lo_w, __shfl_xor_sync(0xffffffffu, lo_w, o));
        hi_w = fmaxf(hi_w, __shfl_xor_sync(0xffffffffu, hi_w, o));
      }
      // lane 0: ranges of the adjacent rows, then the copies
      if (lane == 0) {
        const float amax = fmaxf(fabsf(lo_w), fabsf(hi_w));
        uint32_t bytes = 0;
        column_range(W, g - 1, (lo_w - ww_dn) - win_pad(amax, ww_dn), (hi_w + ww_dn) + win_pad(amax, ww_dn), rng[0], rng[1],
                     rng[2]);
        int q0 = rng[0] & ~(kAlign - 1), q1 = (rng[1] + kAlign - 1) & ~(kAlign - 1);
        const bool st0 = use_tma && q1 > q0 && q1 - q0 <= kSlot;
        if (st0) { rng[3] = q0; cnt0 = q1 - q0; bytes += (uint32_t)(cnt0 * kRec); }
        column_range(W, g + 1, (lo_w - ww_up) - win_pad(amax, ww_up), (hi_w + ww_up) + win_pad(amax, ww_up), rng[4], rng[5],
                     rng[6]);
        q0 = rng[4] & ~(kAlign - 1);
        q1 = (rng[5] + kAlign - 1) & ~(kAlign - 1);
        const bool st1 = use_tma && q1 > q0 && q1 - q0 <= kSlot;
        if (st1) { rng[7] = q0; cnt1 = q1 - q0; bytes += (uint32_t)(cnt1 * kRec); }
        conv = use_tma == 2 && (st0 || rng[1] <= rng[0]) && (st1 || rng[5] <= rng[4]);
        // the slots were read by this warp's previous chunk (generic proxy): order before the copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(S.bar, bytes);
        const char* src = kPacked ? (const char*)W.hq : (const char*)W.hyw;
        if (cnt0) tma_load_1d(S.stage[0], src + (size_t)rng[3] * kRec, (uint32_t)(cnt0 * kRec), S.bar);
        if (cnt1) tma_load_1d(S.stage[1], src + (size_t)rng[7] * kRec, (uint32_t)(cnt1 * kRec), S.bar);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) rng[j] = __shfl_sync(0xffffffffu, rng[j], 0);
      cnt0 = __shfl_sync(0xffffffffu, cnt0, 0);
      cnt1 = __shfl_sync(0xffffffffu, cnt1, 0);
      conv = __shfl_sync(0xffffffffu, conv, 0);
      const bool ok = mbar_wait_bounded(S.bar, parity);
      if (!__all_sync(0xffffffffu, ok)) {
        // give the copies in flight a second bounded wait, then this warp stops (its stage is not
        // used again; the other warps go on)
        if (!ok) (void)mbar_wait_bounded(S.bar, parity);
        if (lane == 0) atomicOr(&W.cnt->err, kErrTimeout);
        break;
      }
      parity ^= 1u;
    }
    const float yi = hi.x, wi = hi.y;
    float best = __int_as_float(0x7f800000);
    int bd = -1, bu = -1;
    bool own_walk = !conv;
    if (conv) {
      const int nd = scan_staged<kPacked>(W, S, 0, g - 1, rng[0], rng[1], rng[3], rng[2], valid, yi, wi, wy_dn, ww_dn, lane);
      const int nu = scan_staged<kPacked>(W, S, 1, g + 1, rng[4], rng[5], rng[7], rng[6], valid, yi, wi, wy_up, ww_up, lane);
      if (nd > kK2Cap || nu > kK2Cap) {
        own_walk = true;
      } else {
        for (int a = 0; a < nd; ++a) {
          const float2 hd = S.cand[0][a * 32 + lane];
          const int d = S.pos[0][a * 32 + lane];
          for (int c = 0; c < nu; ++c)
            pair_step<kPacked>(W, g - 1, g + 1, yi, wi, fm, hd, d, S.cand[1][c * 32 + lane], S.pos[1][c * 32 + lane],
                               best, bd, bu);
        }
      }
    }
    if (valid && own_walk) {
      const RowView vd{S.stage[0], rng[3], cnt0};
      const RowView vu{S.stage[1], rng[7], cnt1};
      // a staged side holds every window of the chunk (the union of the 32 windows' columns)
      const bool sd = cnt0 > 0, su = cnt1 > 0;
      const GridWin qd = grid_window(W.seg_bb, W.seg_dim, W.seg_geo, g - 1, yi, wi, wy_dn, ww_dn);
      const GridWin qu = grid_window(W.seg_bb, W.seg_dim, W.seg_geo, g + 1, yi, wi, wy_up, ww_up);
      // both windows listed (flat walks), then every (d, u) pair in one flat loop: a warp iterates
      // as often as its lane with the most pairs. A lane whose window holds more than kK2Own
      // positions walks its windows nested instead, each row r-1 candidate against a fresh walk of
      // the row r+1 window (same pairs, same result: the pair order is a total order).
      const int nu = list_window<kPacked>(W, qu, vu, su, yi, wi, wy_up, ww_up, S.own[1], lane);
      const int nd = nu > 0 && nu <= kK2Own ? list_window<kPacked>(W, qd, vd, sd, yi, wi, wy_dn, ww_dn, S.own[0], lane) : 0;
      if (nu > 0 && nu <= kK2Own && nd <= kK2Own) {
        const int np = nd * nu;
        float2 hd = make_float2(0.f, 0.f);
        int d = -1;
        for (int k = 0, a = 0, c = 0; k < np; ++k) {
          if (c == 0) {
            d = S.own[0][a * 32 + lane];
            hd = cand_of<kPacked>(W, qd, vd, sd, d);
          }
          const int u = S.own[1][c * 32 + lane];
          pair_step<kPacked>(W, g - 1, g + 1, yi, wi, fm, hd, d, cand_of<kPacked>(W, qu, vu, su, u), u, best, bd, bu);
          if (++c == nu) { c = 0; ++a; }
        }
      } else if (nu > 0) {
        for (int cwd = qd.iw0; cwd <= qd.iw1; ++cwd) {
          const uint32_t cold = qd.bb + (uint32_t)(cwd * qd.ny);
          const int ped = (int)W.bin_start[cold + qd.iy1 + 1];
          const int cbd = col_base(qd.cw0, qd.cshift, cwd);
          for (int d = (int)W.bin_start[cold + qd.iy0]; d < ped; ++d) {
            const float2 hd = cand_at<kPacked>(W, vd, sd, d, cbd);
            if (!(fabsf(hd.x - yi) <= wy_dn && fabsf(hd.y - wi) <= ww_dn)) continue;
            for (int cw = qu.iw0; cw <= qu.iw1; ++cw) {
              const uint32_t col = qu.bb + (uint32_t)(cw * qu.ny);
              const int pe = (int)W.bin_start[col + qu.iy1 + 1];
              const int cb = col_base(qu.cw0, qu.cshift, cw);
              for (int u = (int)W.bin_start[col + qu.iy0]; u < pe; ++u) {
                const float2 hu = cand_at<kPacked>(W, vu, su, u, cb);
                if (!(fabsf(hu.x - yi) <= wy_up && fabsf(hu.y - wi) <= ww_up)) continue;
                pair_step<kPacked>(W, g - 1, g + 1, yi, wi, fm, hd, d, hu, u, best, bd, bu);
              }
            }
          }
        }
      }
    }
    if (valid) W.links[i] = (bd >= 0 && best <= Q.chi_n_max) ? make_int2(bd, bu) : make_int2(-1, -1);
    __syncwarp();
  }
}

template <bool kPacked, int kWarps>
static void prepare_k2() {
  cudaFuncSetAttribute(k_neighbours<kPacked, kWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kWarps * k2_warp_bytes(2));
}
// Dynamic shared memory limits of the neighbour kernels (once per process and device, before any
// launch or graph capture).
void prepare_neighbours() {
  prepare_k2<false, 4>();
  prepare_k2<false, 8>();
  prepare_k2<true, 4>();
  prepare_k2<true, 8>();
}

// warps per block: 4 or 8 (32-hit row chunks a block works on at a time); mode: k2_tma (0, 1, 2)
bool launch_neighbours(int packed, int warps, int grid, cudaStream_t s, const Work& W, const DevParams& Q, int mode) {
  if (mode < 0 || mode > 2) return false;
  const size_t smem = (size_t)warps * k2_warp_bytes(mode);
  if (warps == 4) {
    if (packed) k_neighbours<true, 4><<<grid, 128, smem, s>>>(W, Q, mode);
    else k_neighbours<false, 4><<<grid, 128, smem, s>>>(W, Q, mode);
  } else if (warps == 8) {
    if (packed) k_neighbours<true, 8><<<grid, 256, smem, s>>>(W, Q, mode);
    else k_neighbours<false, 8><<<grid, 256, smem, s>>>(W, Q, mode);
  } else {
    return false;
  }
  return true;
}
int neighbours_blocks_per_sm(int packed, int warps, int mode) {
  int nb = 0;
  const size_t smem = (size_t)warps * k2_warp_bytes(mode);
  if (warps == 4) {
    if (packed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_neighbours<true, 4>, 128, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_neighbours<false, 4>, 128, smem);
  } else if (warps == 8) {
    if (packed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_neighbours<true, 8>, 256, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_neighbours<false, 8>, 256, smem);
  }
  return nb;
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
  __shared__ int s_item;
  const BatchDesc* B = W.batch;
  for (;;) {
    const int g = next_segment(&W.cnt->seg_next[1], B->nf, &s_item);
    if (g < 0) break;
    const int a = (int)W.bin_start[W.seg_bb[g]];
    const int b = (int)W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    int count = 0;
    for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
      const int u = clean_up(W.links, i), d = clean_dn(W.links, i);
      W.clinks[i] = make_int2(d, u);
      bool st = false;
      if (u >= 0 && d < 0) {
        int len = 2;
        for (int h = clean_up(W.links, u); h >= 0 && len < Q.lmin; h = clean_up(W.links, h)) ++len;
        st = len >= Q.lmin;
      }
      count += st ? 1 : 0;
      if (W.is_start) W.is_start[i] = st ? 1 : 0;
    }
    const int tot = block_sum(count, red);
    if (threadIdx.x == 0) W.seg_nstart[g] = (uint32_t)tot;
  }
}

// ------------------------------------------------------------------------------------ K4
__global__ void __launch_bounds__(256) k_starts(Work W, DevParams Q) {
  __shared__ int warp_off[8];
  __shared__ int s_total;
  __shared__ int s_item;
  const BatchDesc* B = W.batch;
  const uint32_t tcap = (uint32_t)W.tcap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    const int g = next_segment(&W.cnt->seg_next[2], B->nf, &s_item);
    if (g < 0) break;
    const int a = (int)W.bin_start[W.seg_bb[g]];
    const int b = (int)W.bin_start[W.seg_bb[g] + W.seg_nb[g]];
    uint32_t out = W.seg_nstart[g];
    const uint32_t bb = W.seg_bb[g];
    const int4 dim = W.seg_dim[g];
    const float4 geo = W.seg_geo[g];
    for (int c0 = a; c0 < b; c0 += blockDim.x) {
      const int i = c0 + threadIdx.x;
      const bool st = i < b && W.is_start[i];  // set by k_clean
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
          const int iw = W.packed ? (int)W.hcol[i] : bin_of(W.hyw[i].y, geo.x, geo.y, dim.x);
          const uint32_t col = bb + (uint32_t)(iw * dim.y);
          W.starts_raw[pos] = make_uint4((uint32_t)i, (uint32_t)g, col, 0u);
        }
      }
      out += (uint32_t)s_total;
      __syncthreads();
    }
  }
}

// K4b: canonical order of start hits and their rank in the sector (rows, then (w, y, input index)).
// A w-column holds every hit of its w range, so hits of earlier columns are smaller; only the hits
// of the start's own column are compared one by one.
__device__ __forceinline__ float2 hit_any(const Work& W, int g, int p) {
  return W.packed ? hit_by_index<true>(W.hyw, W.hq, W.hcol, W.seg_dim, g, p)
                  : hit_by_index<false>(W.hyw, W.hq, W.hcol, W.seg_dim, g, p);
}

__global__ void __launch_bounds__(256) k_start_order(Work W) {
  const uint32_t n = min(W.cnt->n_starts, (uint32_t)W.tcap);
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint4 e = W.starts_raw[p];
    const int i = (int)e.x, g = (int)e.y;
    const uint32_t col = e.z;
    const float2 hi = hit_any(W, g, i);
    const uint32_t oi = W.horig[i];
    // run of start entries sharing the w-column (contiguous in sorted order)
    uint32_t lo = p, hiq = p;
    while (lo > 0 && W.starts_raw[lo - 1].z == col) --lo;
    while (hiq + 1 < n && W.starts_raw[hiq + 1].z == col) ++hiq;
    uint32_t before = 0;
    for (uint32_t q = lo; q <= hiq; ++q) {
      if (q == p) continue;
      const int j = (int)W.starts_raw[q].x;
      const float2 hj = hit_any(W, g, j);
      if (key_less(hj.y, hj.x, W.horig[j], hi.y, hi.x, oi)) ++before;
    }
    // rank of the hit within its row and sector
    const uint32_t ny = (uint32_t)W.seg_dim[g].y;
    const uint32_t c0 = W.bin_start[col], c1 = W.bin_start[col + ny];
    uint32_t incol = 0;
    for (uint32_t h = c0; h < c1; ++h) {
      if ((int)h == i) continue;
      const float2 hh = hit_any(W, g, (int)h);
      if (key_less(hh.y, hh.x, W.horig[h], hi.y, hi.x, oi)) ++incol;
    }
    const int r = (g % kSegPerFrame) % kNRow;
    const uint32_t sec_first = W.bin_start[W.seg_bb[g - r]];
    const uint32_t rank = (c0 - sec_first) + incol;
    if (rank >= (1u << 24)) atomicOr(&W.cnt->wide_keys, 1u);  // the selection's 32-bit vote keys do not fit
    W.starts[lo + before] = make_uint4((uint32_t)i, (uint32_t)g, rank, 0u);
  }
}

}  // namespace tpc
