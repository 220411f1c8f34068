// tpc_static.cu — cleaned neighbour links of one frame with no device allocation.
//
// Some callers cannot allocate device memory when they call the tracker: code that runs while a
// framework's caching allocator owns all of the device's memory, code under a real-time or
// allocation-free discipline (cudaMalloc and cudaFree synchronise the device and can fail), or
// code that calls in from a context where the allocator must not be touched. tpc_links_static()
// serves them: it runs the search-grid and neighbour kernels (K1-K3) of one frame with all of their
// scratch in one file-scope device array of fixed size, and writes the frame's cleaned links into
// arrays the caller provides.
//
// The array is part of the library's device image: every GPU that loads the library holds it
// (kStaticScratchBytes, about 17.9 MiB) until the process exits. Calls share it and it keeps the last
// call's contents; everything the kernels need zeroed is cleared by the call itself. Two calls that
// overlap on the GPU (from two host threads, or on two streams) race on it and must be serialised by
// the caller.
//
// In host code the array's name is only a host-side stand-in, not a device address. The first call
// on a device (with that device current) looks the real address up with cudaGetSymbolAddress and
// creates the event used for the bounded completion wait; make that first call before any stream
// capture.
#include <chrono>
#include <cstring>
#include <mutex>

#include "tpc_dev.cuh"
#include "tpctrack.h"

namespace tpc {
__global__ void k_scan_reduce(const uint32_t*, const uint32_t*, long long, int, uint32_t*);
__global__ void k_scan_tiles(uint32_t*, const uint32_t*, long long, int, uint32_t*);
__global__ void k_scan_apply(const uint32_t*, const uint32_t*, long long, int, const uint32_t*, const uint32_t*, uint32_t*);
__global__ void k_seg_hist(Work);
__global__ void k_seg_layout(Work, DevParams);
__global__ void k_bin_rank(Work, int);
__global__ void k_scatter(Work, int);
__global__ void k_clean(Work, DevParams);
__global__ void k_reset_counters(Work);
__global__ void k_zero_u32(uint32_t*, const uint32_t*, long long, int, int);
__global__ void k_links_to_input(Work, int, int, int32_t*);
void make_dev_params(const tpc_params& p, DevParams& d);
bool launch_neighbours(int packed, int warps, int grid, cudaStream_t s, const Work& W, const DevParams& Q, int use_tma);
__global__ void k_chunk_count(Work);
void prepare_neighbours();
__global__ void k_chunk_fill(Work);
}  // namespace tpc

using namespace tpc;

namespace {

constexpr long long kStaticMaxClusters = TPC_STATIC_MAX_CLUSTERS;
constexpr double kStaticMinOccupancy = 1.0;  // grid bins are sized for at least 1 cluster per bin

constexpr size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct StaticLayout {
  size_t cnt, desc, seg_cnt, seg_nb, seg_bb, seg_dim, seg_geo, bin_start, rank, hyw, horig, links, clinks,
      seg_nstart, scan_tmp, k2_off, k2_tab, total;
};

constexpr StaticLayout static_layout(long long ncap, long long bcap) {
  StaticLayout L{};
  const long long scap = kSegPerFrame;
  const long long ntiles = (bcap + 1 + 2047) / 2048 + 16;
  size_t o = 0;
  L.cnt = o;        o = al(o + sizeof(DevCounters));
  L.desc = o;       o = al(o + sizeof(BatchDesc));
  L.seg_cnt = o;    o = al(o + 4 * (size_t)scap);
  L.seg_nb = o;     o = al(o + 4 * (size_t)scap);
  L.seg_bb = o;     o = al(o + 4 * (size_t)(scap + 1));
  L.seg_dim = o;    o = al(o + 16 * (size_t)scap);
  L.seg_geo = o;    o = al(o + 16 * (size_t)scap);
  L.bin_start = o;  o = al(o + 4 * (size_t)(bcap + 1));
  L.rank = o;       o = al(o + 4 * (size_t)ncap);
  L.hyw = o;        o = al(o + 8 * (size_t)(ncap + 2));
  L.horig = o;      o = al(o + 4 * (size_t)ncap);
  L.links = o;      o = al(o + 8 * (size_t)ncap);
  L.clinks = o;     o = al(o + 8 * (size_t)ncap);
  L.seg_nstart = o; o = al(o + 4 * (size_t)(scap + 1));
  L.scan_tmp = o;   o = al(o + 4 * (size_t)ntiles);
  L.k2_off = o;     o = al(o + 4 * (size_t)(scap + 1));
  L.k2_tab = o;     o = al(o + 8 * (size_t)(ncap / 32 + scap + 1));
  L.total = o;
  return L;
}

// bins of a frame's grid (FP32 storage): at most 4 ceil(n / occupancy) + 260 per segment (see
// k_seg_layout)
constexpr long long static_bcap(long long n, double occ) {
  return 4 * ((long long)((double)n / occ) + 1 + kSegPerFrame) + 264LL * kSegPerFrame + 16;
}

constexpr size_t kStaticScratchBytes = static_layout(kStaticMaxClusters, static_bcap(kStaticMaxClusters, kStaticMinOccupancy)).total;

// The scratch: one array of fixed size in the library's device image.
static __device__ __align__(256) unsigned char g_links_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
cudaEvent_t g_done[kMaxDevices] = {nullptr};

// Once per device, with that device current: the array's device address and the completion event.
int static_setup(int dev, void** addr, cudaEvent_t* done) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_links_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TPC_E_CUDA;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return TPC_E_CUDA;
    }
    g_done[dev] = e;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *done = g_done[dev];
  return TPC_OK;
}

}  // namespace

extern "C" int tpc_links_static(const tpc_params* params, const tpc_clusters* clusters, int32_t* up, int32_t* down,
                                void* cuda_stream) {
  if (!clusters || !up || !down) return TPC_E_INVAL;
  if (!clusters->on_device) return TPC_E_INVAL;
  const long long n = clusters->n;
  if (n < 0) return TPC_E_INVAL;
  if (n > kStaticMaxClusters) return TPC_E_CAPACITY;  // larger than the fixed scratch holds
  if (n > 0 && (!clusters->sector || !clusters->row || !clusters->y || !clusters->w)) return TPC_E_INVAL;
  tpc_params p;
  if (params) {
    if (params->struct_size != sizeof(tpc_params)) return TPC_E_INVAL;
    p = *params;
  } else {
    tpc_default_params(&p);
  }
  if (p.bin_occupancy <= 0.f) p.bin_occupancy = 2.0f;
  if (p.packed) return TPC_E_INVAL;  // FP32 cluster storage only
  if (p.bin_occupancy < kStaticMinOccupancy) return TPC_E_CAPACITY;  // finer grids need more bins
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { cudaGetLastError(); return TPC_E_CUDA; }
  void* base = nullptr;
  cudaEvent_t done = nullptr;
  int rc = static_setup(dev, &base, &done);
  if (rc) return rc;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { cudaGetLastError(); return TPC_E_CUDA; }
  DevParams Q;
  make_dev_params(p, Q);

  // carve the work arrays out of the scratch (capacities of the largest frame accepted)
  const long long bcap = static_bcap(kStaticMaxClusters, kStaticMinOccupancy);
  constexpr StaticLayout L = static_layout(kStaticMaxClusters, static_bcap(kStaticMaxClusters, kStaticMinOccupancy));
  char* b = (char*)base;
  Work W;
  memset(&W, 0, sizeof(W));
  W.cnt = (DevCounters*)(b + L.cnt);
  W.batch = (const BatchDesc*)(b + L.desc);
  W.seg_cnt = (uint32_t*)(b + L.seg_cnt);
  W.seg_nb = (uint32_t*)(b + L.seg_nb);
  W.seg_bb = (uint32_t*)(b + L.seg_bb);
  W.seg_dim = (int4*)(b + L.seg_dim);
  W.seg_geo = (float4*)(b + L.seg_geo);
  W.bin_start = (uint32_t*)(b + L.bin_start);
  W.rank = (uint32_t*)(b + L.rank);
  W.hyw = (float2*)(b + L.hyw);
  W.horig = (uint32_t*)(b + L.horig);
  W.links = (int2*)(b + L.links);
  W.clinks = (int2*)(b + L.clinks);
  W.seg_nstart = (uint32_t*)(b + L.seg_nstart);
  W.scan_tmp = (uint32_t*)(b + L.scan_tmp);
  W.k2_off = (uint32_t*)(b + L.k2_off);
  W.k2_tab = (uint2*)(b + L.k2_tab);
  W.ncap = kStaticMaxClusters;
  W.scap = kSegPerFrame;
  W.bcap = bcap;
  W.tcap = 0;
  W.scan_tmp_cap = (bcap + 1 + 2047) / 2048 + 16;
  W.k2cap = kStaticMaxClusters / 32 + kSegPerFrame + 1;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the frame descriptor, copied from the stack (a pageable source: the copy is staged before return)
  BatchDesc desc;
  memset(&desc, 0, sizeof(desc));
  desc.nf = 1;
  desc.ntot = n;
  desc.f[0].sector = clusters->sector;
  desc.f[0].row = clusters->row;
  desc.f[0].y = clusters->y;
  desc.f[0].w = clusters->w;
  desc.f[0].n = n;
  desc.f[0].off = 0;
  cudaMemcpyAsync(b + L.desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, s);

  const int G = sms;
  DevCounters* C = W.cnt;
  auto scan = [&](const uint32_t* in, uint32_t* out, const uint32_t* n_dev, long long n_cap, uint32_t* total) {
    k_scan_reduce<<<2 * G, 256, 0, s>>>(in, n_dev, n_cap, 0, W.scan_tmp);
    k_scan_tiles<<<1, 1024, 0, s>>>(W.scan_tmp, n_dev, n_cap, 0, total);
    k_scan_apply<<<2 * G, 256, 0, s>>>(in, n_dev, n_cap, 0, W.scan_tmp, total, out);
  };
  k_reset_counters<<<1, 128, 0, s>>>(W);
  k_zero_u32<<<G, 256, 0, s>>>(W.seg_cnt, &C->nseg, W.scap, 0, 1);
  k_seg_hist<<<G, kHistThreads, 0, s>>>(W);
  k_seg_layout<<<G, 256, 0, s>>>(W, Q);
  scan(W.seg_nb, W.seg_bb, &C->nseg, W.scap, &C->n_bins);
  k_zero_u32<<<4 * G, 256, 0, s>>>(W.bin_start, &C->n_bins, W.bcap + 1, 1, 1);
  k_bin_rank<<<8 * G, 256, 0, s>>>(W, 0);
  scan(W.bin_start, W.bin_start, &C->n_bins, W.bcap, &C->n_sorted);
  k_scatter<<<8 * G, 256, 0, s>>>(W, 0);
  prepare_neighbours();
  k_chunk_count<<<G, 256, 0, s>>>(W);
  scan(W.k2_off, W.k2_off, &C->nseg, W.scap, &C->n_chunks);
  k_chunk_fill<<<G, 256, 0, s>>>(W);
  launch_neighbours(0, p.k2_warps == 4 ? 4 : 8, 4 * G, s, W, Q, p.k2_tma >= 0 && p.k2_tma <= 2 ? p.k2_tma : 1);
  k_clean<<<4 * G, 256, 0, s>>>(W, Q);
  if (n > 0) {
    cudaMemsetAsync(up, 0xFF, 4 * (size_t)n, s);
    cudaMemsetAsync(down, 0xFF, 4 * (size_t)n, s);
    k_links_to_input<<<2 * G, 256, 0, s>>>(W, 0, 2, up);
    k_links_to_input<<<2 * G, 256, 0, s>>>(W, 0, 3, down);
  }
  if (cudaEventRecord(done, s) != cudaSuccess) { cudaGetLastError(); return TPC_E_CUDA; }
  if (cudaGetLastError() != cudaSuccess) return TPC_E_CUDA;
  // bounded wait for completion (two minutes), then read the device error word
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) { cudaGetLastError(); return TPC_E_CUDA; }
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(120)) return TPC_E_TIMEOUT;
  }
  // the error word, read on the caller's stream only (a device-to-pageable copy returns once it has
  // landed; the legacy default stream would also wait for unrelated work of other streams)
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, &C->err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
    cudaGetLastError();
    return TPC_E_CUDA;
  }
  if (err & kErrInput) return TPC_E_INVAL;
  if (err & kErrTimeout) return TPC_E_TIMEOUT;
  if (err & kErrBins) return TPC_E_CAPACITY;
  return TPC_OK;
}
