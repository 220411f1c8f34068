// tpc_api.cu — host runtime and C-ABI of libtpctrack.so (see include/tpctrack.h).
//
// A context owns a stream, a device memory pool, a pool of batch workspaces and the frames loaded
// into it. Tracking a frame (or a batch of frames) enqueues the kernel sequence K1..K8 on a stream:
// every kernel is persistent (grid = SMs x resident blocks) and reads its sizes from device
// memory, so the same sequence is captured once per workspace into a CUDA graph and replayed.
// Serving (tpc_submit_frame / tpc_poll) keeps frames in a host queue, admits them against the HBM
// budget, and launches a new batch of admitted frames whenever a stream slot is free, so work of
// requests that arrive while others run overlaps on the device (continuous batching).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "cf_dev.cuh"
#include "tpctrack.h"

namespace tpc {
__global__ void k_scan_reduce(const uint32_t*, const uint32_t*, long long, int, uint32_t*);
__global__ void k_scan_tiles(uint32_t*, const uint32_t*, long long, int, uint32_t*);
__global__ void k_scan_apply(const uint32_t*, const uint32_t*, long long, int, const uint32_t*, const uint32_t*, uint32_t*);
struct SmallScan {
  const uint32_t* in[2];
  uint32_t* out[2];
  const uint32_t* n_dev[2];
  long long n_host[2];
  uint32_t* total[2];
};
__global__ void k_scan_small(SmallScan);
__global__ void k_seg_hist(Work);
__global__ void k_seg_layout(Work, DevParams);
__global__ void k_bin_rank(Work, int);
__global__ void k_scatter(Work, int);
__global__ void k_seg_bucket(Work);
__global__ void k_bin_rank_seg(Work);
__global__ void k_scatter_seg(Work);
__global__ void k_chunk_count(Work);
__global__ void k_chunk_fill(Work);
__global__ void k_clean(Work, DevParams);
__global__ void k_starts(Work, DevParams);
__global__ void k_start_order(Work);
__global__ void k_chains(Work, int);
__global__ void k_one_pass_bins(Work);
__global__ void k_length_offsets(Work);
__global__ void k_length_scatter(Work, int);
bool launch_tracklets(int threads, int regs, int ilp, int packed, int grid, cudaStream_t s, const Work& W, const DevParams& Q,
                      int ordered);
int tracklets_blocks_per_sm(int threads, int regs, int ilp, int packed);
bool launch_neighbours(int packed, int warps, int grid, cudaStream_t s, const Work& W, const DevParams& Q, int use_tma);
int neighbours_blocks_per_sm(int packed, int warps, int mode);
void prepare_neighbours();
void launch_wait_probe(uint32_t* status, unsigned long long limit_ns, cudaStream_t s);
void launch_votes(int lanes, int grid, cudaStream_t s, const Work& W, const DevParams& Q);
void launch_kept(int lanes, int grid, cudaStream_t s, const Work& W, const DevParams& Q);
void launch_write_tracks(int lanes, int grid, cudaStream_t s, const Work& W, const DevParams& Q);
void launch_compress(int packed, int grid, cudaStream_t s, const Work& W, const DevParams& Q);
__global__ void k_frame_offsets(Work);
__global__ void k_beamline(Work, DevParams);
__global__ void k_reset_counters(Work);
__global__ void k_zero_u32(uint32_t*, const uint32_t*, long long, int, int);
__global__ void k_set_ntracklets(Work);
__global__ void k_links_to_input(Work, int, int, int32_t*);
__global__ void k_merge_outer(Work, DevParams);
__global__ void k_merge_fill(Work);
__global__ void k_merge_match(Work, DevParams);
__global__ void k_merge_link(Work);
__global__ void k_merge_heads(Work);
__global__ void k_merge_refit(Work, DevParams);
__global__ void k_merge_frames(Work);
__global__ void k_cf_fill(CfArgs);
__global__ void k_cf_peaks(CfArgs);
__global__ void k_cf_copy(CfArgs);
__global__ void k_cf_clear(CfArgs);
__global__ void k_cf_flag(CfArgs);
__global__ void k_cf_emit(CfArgs);
__global__ void k_cf_gcount(CfArgs);
__global__ void k_cf_gscan(CfArgs);
__global__ void k_cf_gplace(CfArgs);
__global__ void k_cf_wfill(CfArgs);
__global__ void k_cf_wclear(CfArgs);

// Cluster finding: device buffers sized by a digit capacity, the charge map (kept zero between
// calls), page-locked host copies of the last call's clusters, timing events.
constexpr int kCfKernels = 5;
struct CfState {
  void* dev = nullptr;
  long long cap = 0;
  uint8_t *in_sector = nullptr, *in_row = nullptr;
  uint16_t *in_pad = nullptr, *in_time = nullptr, *in_adc = nullptr;
  uint32_t *wcount = nullptr, *woff = nullptr, *wsrc = nullptr, *scan_tmp = nullptr, *small = nullptr;
  uint32_t* wflag = nullptr;
  uint32_t *glist = nullptr, *gwide = nullptr, *gwin = nullptr, *gcnt = nullptr, *gbeg = nullptr, *gcur = nullptr;
  int windows = 1;                  // time windows of the last call (1: the whole frame in one map)
  uint8_t *t_sector = nullptr, *t_row = nullptr;
  float *t_y = nullptr, *t_w = nullptr, *t_sp = nullptr, *t_st = nullptr;
  uint32_t *t_qtot = nullptr, *t_digit = nullptr;
  uint16_t* t_qmax = nullptr;
  uint16_t* npads = nullptr;
  uint8_t *o_sector = nullptr, *o_row = nullptr;
  float *o_y = nullptr, *o_w = nullptr, *o_sp = nullptr, *o_st = nullptr;
  uint32_t *o_qtot = nullptr, *o_digit = nullptr;
  uint16_t* o_qmax = nullptr;
  uint16_t* map = nullptr;
  size_t map_bytes = 0;
  int lines = 0, stride = 0;
  bool map_clean = false;
  uint32_t* h_small = nullptr;      // page-locked: total, error bits
  void* host = nullptr;
  size_t host_bytes = 0;
  cudaEvent_t ev[kCfKernels + 1] = {nullptr};
  cudaEvent_t done = nullptr;
  float ms[kCfKernels] = {0};
  int64_t launches[kCfKernels] = {0};
};
}  // namespace tpc

namespace tpc {
// Host-side derived constants: computed in double, rounded once; row geometry and window sizes in
// float arithmetic exactly as they are defined (IEEE operations on the host).
void make_dev_params(const tpc_params& p, DevParams& d) {
  memset(&d, 0, sizeof(d));
  d.kq = (float)(-0.0029979246 * p.bz);
  d.chi_n_max = (float)p.chi_n_max;
  d.lmin = p.lmin;
  d.r00 = (float)(p.sigma_y * p.sigma_y);
  d.r11 = (float)(p.sigma_w * p.sigma_w);
  d.chi2_max = (float)p.chi2_hit_max;
  d.n_miss_max = p.n_miss_max;
  d.win_nsig = (float)p.win_nsig;
  d.win_add = (float)p.win_add;
  d.ms_on = p.x0_per_row > 0;
  d.x0_row = (float)p.x0_per_row;
  const double hl = p.x0_per_row > 0 ? 0.0136 * (1.0 + 0.038 * std::log(p.x0_per_row)) : 0.0;
  d.ms_c = (float)(hl * hl);
  d.mass2 = (float)(0.13957039 * 0.13957039);
  d.max_sin = (float)p.max_sin;
  d.y_margin = (float)p.y_margin;
  d.tan10 = (float)0.17632698070846498;
  d.nmin = p.nmin;
  for (int i = 0; i < 5; ++i) d.cov0[i] = (float)p.cov0[i];
  d.ext_stop = p.ext_stop ? 1 : 0;
  d.drift_len = (float)p.drift_length;
  d.vdrift = (float)p.drift_velocity;
  d.keep_vy = (float)p.keep_vy;
  d.keep_vw = (float)p.keep_vw;
  d.keep_qpt_max = (float)p.keep_qpt_max;
  d.merge_gap_rows = p.merge_gap_rows;
  d.merge_dw = (float)p.merge_dw;
  d.merge_chi2_max = (float)p.merge_chi2_max;
  d.rot_c = (float)0.93969262078590838;  // cos(20 deg)
  d.rot_s = (float)0.34202014332566873;  // sin(20 deg)
  d.refit_scale = (float)p.refit_scale;
  d.refit_passes = p.refit_passes;
  d.occ = p.bin_occupancy > 0 ? p.bin_occupancy : 2.0f;
  volatile float pitch = (float)160 / (float)151;
  d.pitch = pitch;
  for (int r = 0; r < kNRow; ++r) {
    volatile float xr = (float)r * pitch;
    d.x[r] = (float)85 + xr;
  }
  const float ky = (float)p.ky, kw = (float)p.kw, eps = (float)p.eps;
  for (int r = 1; r + 1 < kNRow; ++r) {
    volatile float dxm = d.x[r] - d.x[r - 1];
    volatile float dxp = d.x[r + 1] - d.x[r];
    volatile float a = ky * dxm, b = kw * dxm, c = ky * dxp, e = kw * dxp, s = dxm + dxp;
    d.wy_dn[r] = a + eps;
    d.ww_dn[r] = b + eps;
    d.wy_up[r] = c + eps;
    d.ww_up[r] = e + eps;
    d.f_mid[r] = dxm / s;
  }
  for (int r = 0; r < kNRow; ++r) d.yext[r] = d.x[r] * d.tan10 + 1.0f;
  d.aspect = (float)((p.kw * (160.0 / 151.0) + p.eps) / (p.ky * (160.0 / 151.0) + p.eps));
}

}  // namespace tpc

using namespace tpc;

namespace {

const char* kKernelNames[] = {"reset",  "seg_hist", "seg_layout", "scan_seg",  "zero_bins", "bin_rank", "scan_bins",
                              "scatter", "neighbours", "clean",   "scan_start", "starts",   "start_order",
                              "chains", "tracklets", "zero_w", "votes",    "kept",      "scan_kept", "write_tracks", "compress", "beamline",
                              "frame_off", "merge"};
constexpr int kNumKernels = sizeof(kKernelNames) / sizeof(kKernelNames[0]);

// Launch shape: the knobs that change the speed of the sequence, never its results.
struct Shape {
  float occ = 2.0f;      // grid bin occupancy
  int k2_warps = 8, k2_tma = 1;
  int k5_block = 128, k5_regs = 64, k5_bps = 0, k5_order = 0, k5_ilp = 1;
  int sel_lanes = 32;
  bool operator==(const Shape& o) const {
    return occ == o.occ && k2_warps == o.k2_warps && k2_tma == o.k2_tma && k5_block == o.k5_block &&
           k5_regs == o.k5_regs && k5_bps == o.k5_bps && k5_order == o.k5_order && k5_ilp == o.k5_ilp &&
           sel_lanes == o.sel_lanes;
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Workspace {
  long long ncap = 0, scap = 0, bcap = 0, tcap = 0, scan_cap = 0;
  Shape shape;                     // launch shape of the captured graph (occ fixed at allocation)
  DevParams dp{};                  // the context's parameters with this workspace's occupancy
  int nf_cap = 0;
  size_t bytes = 0;
  void* block = nullptr;
  Work W{};
  BatchDesc* d_desc = nullptr;
  BatchDesc* h_desc = nullptr;     // pinned
  DevCounters* h_cnt = nullptr;    // pinned
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  int users = 0;                   // frames whose results live here
  bool busy = false;
  std::vector<tpc_frame_t> batch_ids;  // frames of the last batch run here, in order
};

struct Frame {
  tpc_frame_t id = 0;
  long long n = 0;
  uint8_t* d_sector = nullptr;
  uint8_t* d_row = nullptr;
  float* d_y = nullptr;
  float* d_w = nullptr;
  void* d_block = nullptr;         // owned input allocation (nullptr when borrowed)
  int state = 0;                   // 0 loaded, 1 queued, 2 admitted, 3 running, 4 results in copy, 5 fetched
  std::shared_ptr<Workspace> ws;
  int fidx = 0;
  std::vector<char> host_copy;      // serving: clusters submitted from host memory, until admitted
  const void* borrowed[4] = {};     // serving: borrowed page-locked host input (on_device = 2)
  bool is_borrowed = false;
  bool served = false;
  size_t input_bytes = 0;           // serving: device input counted against the waiting-input reserve
  double t_submit = 0, t_done = 0;
  // host results: views into one page-locked block (from the context's pinned cache)
  void* res = nullptr;
  size_t res_cap = 0;
  int64_t n_tracks = 0;
  int32_t *sector = nullptr, *ndf = nullptr;
  float *xref = nullptr, *param = nullptr, *cov = nullptr, *chi2 = nullptr, *beam = nullptr;
  int32_t *residual = nullptr, *n_pred = nullptr;
  bool fetch_compress = false;
  int64_t* hoff = nullptr;
  uint32_t* hits = nullptr;
  size_t fetch_nt = 0, fetch_nh = 0;  // tracks and hits copied into res (split by fetch_finish)
  uint32_t fetch_h0 = 0;              // the frame's first hit in the batch's hit list
  // merged tracks (K12), views into the same block
  bool fetch_merge = false;
  size_t fetch_nm = 0, fetch_nmh = 0;
  uint32_t fetch_mh0 = 0;
  int64_t n_merged = 0;
  int32_t *m_sector = nullptr, *m_nseg = nullptr, *m_head = nullptr, *m_ndf = nullptr, *m_nfit = nullptr;
  float *m_xref = nullptr, *m_param = nullptr, *m_cov = nullptr, *m_chi2 = nullptr;
  int64_t* m_hoff = nullptr;
  uint32_t* m_hits = nullptr;
  int32_t* tr_next = nullptr;
  float* tr_mchi2 = nullptr;
};

// Page-locked host blocks for results, cached by capacity (powers of two from 1 MiB), so a frame's
// read-back is a direct DMA into memory that stays valid until the frame is released.
struct PinnedCache {
  std::multimap<size_t, void*> free_blocks;
  size_t cached = 0;
  static constexpr size_t kMaxCached = size_t(4) << 30;
  void* get(size_t need, size_t& cap) {
    auto it = free_blocks.lower_bound(need);
    if (it != free_blocks.end() && it->first <= 2 * need + (size_t(1) << 20)) {
      cap = it->first;
      void* p = it->second;
      cached -= cap;
      free_blocks.erase(it);
      return p;
    }
    cap = size_t(1) << 20;
    while (cap < need) cap <<= 1;
    void* p = nullptr;
    if (cudaMallocHost(&p, cap) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t cap) {
    if (!p) return;
    if (cached + cap > kMaxCached) {
      cudaFreeHost(p);
      return;
    }
    free_blocks.emplace(cap, p);
    cached += cap;
  }
  void clear() {
    for (auto& kv : free_blocks) cudaFreeHost(kv.second);
    free_blocks.clear();
    cached = 0;
  }
};

}  // namespace

struct tpc_ctx {
  tpc_params p{};
  DevParams dp{};
  int device = 0, sms = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  std::map<tpc_frame_t, std::unique_ptr<Frame>> frames;
  tpc_frame_t next_id = 1;
  std::string err;
  std::vector<std::shared_ptr<Workspace>> wspool;
  Shape shape;                     // launch shape of the next runs (parameters or autotuned)
  bool tuned = false;
  std::vector<tpc_tune_entry> tune_entries;
  std::map<long long, int> blocks_cache;  // resident blocks per SM of each kernel shape
  bool timing = false;
  cudaEvent_t ev[kNumKernels + 1] = {nullptr};
  cudaEvent_t ev_sync = nullptr;
  // serving: end of the last launched tracking of a large batch (kServeSerialClusters), which the
  // next large batch's tracking waits for on its own slot
  cudaEvent_t ev_track = nullptr;
  bool large_launched = false;
  float ms[kNumKernels] = {0};
  int64_t launches[kNumKernels] = {0};
  int64_t stage_launches[kNumKernels] = {0};
  // serving: each stream slot owns one workspace of slot_clusters clusters carved from the HBM
  // budget; a batch is the queued frames that fit it, launched as soon as the slot is free
  std::deque<tpc_frame_t> queue;  // submitted, not yet admitted
  struct Slot {
    cudaStream_t stream = nullptr;
    std::shared_ptr<Workspace> ws;
    std::vector<tpc_frame_t> frames;
    bool busy = false;
  };
  std::vector<Slot> slots;
  long long slot_clusters = 0;
  size_t queued_input_bytes = 0;    // device inputs of submitted frames not yet retired
  std::deque<tpc_frame_t> finished;
  PinnedCache pinned;               // result blocks of fetched frames
  // serving: result copies in flight (one event per retired batch, recorded on its slot's stream
  // after the copies; the slot's next batch is queued behind them)
  struct Fetching {
    cudaEvent_t ev = nullptr;
    std::vector<tpc_frame_t> frames;
  };
  std::deque<Fetching> fetching;
  std::vector<cudaEvent_t> spare_events;
  CfState cf;
};

namespace {

// exclusive scans of at most this many entries (by capacity: the per-segment scans of workspaces of
// up to 11 frames) run as one single-block launch; larger ones are faster as reduce / scan / apply
constexpr long long kSmallScanCap = 1LL << 16;

// serving: queued frames join one batch only up to this many clusters (a larger frame goes alone)
constexpr long long kServeBatchClusters = 1LL << 21;
// Batches above this many clusters track one at a time across the slots: each fills the GPU for
// tens of milliseconds, and two of them side by side left their uploads and result copies exposed
// (the end-to-end time of a full-size frame was about its tracking plus its copies). One after the
// other, a slot's uploads and result copies run during the other slot's tracking. Smaller batches
// still run side by side, where the overlap of their latency-bound tails pays.
constexpr long long kServeSerialClusters = 1LL << 24;

// grid occupancies the autotuner times, finest first
constexpr float kTunerOccupancies[] = {0.35f, 0.5f, 0.7f, 1.0f, 2.0f};

int fail(tpc_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, TPC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void free_workspace(Workspace* w) {
  if (!w) return;
  if (w->graph) cudaGraphExecDestroy(w->graph);
  if (w->block) cudaFree(w->block);
  if (w->h_desc) cudaFreeHost(w->h_desc);
  if (w->h_cnt) cudaFreeHost(w->h_cnt);
  if (w->done) cudaEventDestroy(w->done);
  w->block = nullptr;
}

// Lay out one device block for the capacities (dry: only compute its size into *dry_bytes).
int alloc_workspace(tpc_ctx* ctx, long long ncap, long long tcap, int nf_cap, std::shared_ptr<Workspace>& out,
                    size_t* dry_bytes = nullptr) {
  auto ws = std::shared_ptr<Workspace>(new Workspace, [](Workspace* w) { free_workspace(w); delete w; });
  ws->ncap = std::max(ncap, 1024LL);
  ws->tcap = (std::max(tcap, 1024LL) + 31) / 32 * 32;  // whole warps of tracklets
  ws->nf_cap = nf_cap;
  ws->scap = (long long)nf_cap * kSegPerFrame;
  ws->shape = ctx->shape;
  ws->dp = ctx->dp;
  ws->dp.occ = ctx->shape.occ;
  const double occ = ws->dp.occ;
  // a segment grid has at most 4 ceil(n / occ) + 260 bins, 513 in the 16-bit storage (k_seg_layout)
  ws->bcap = 4 * ((long long)std::ceil((double)ws->ncap / occ) + ws->scap) + (ctx->p.packed ? 520 : 264) * ws->scap + 16;
  const bool merge = ctx->p.merge != 0;        // merging and refit (K12)
  const long long mbcap = merge ? (long long)nf_cap * kNSec * kMergeBins : 0;
  long long maxscan = std::max({ws->bcap + 1, ws->scap + 1, ws->tcap + 1, mbcap + 1});
  const bool compress = ctx->p.compress != 0;  // compression inputs (K10)
  ws->scan_cap = (maxscan + 2047) / 2048 + 16;
  struct Item { void** ptr; size_t bytes; };
  Work& W = ws->W;
  void* p_cnt; void* p_desc;
  std::vector<Item> items = {
      {&p_cnt, sizeof(DevCounters)},
      {&p_desc, sizeof(BatchDesc)},
      {(void**)&W.seg_cnt, 4 * (size_t)ws->scap},
      {(void**)&W.seg_nb, 4 * (size_t)ws->scap},
      {(void**)&W.seg_bb, 4 * (size_t)(ws->scap + 1)},
      {(void**)&W.seg_dim, 16 * (size_t)ws->scap},
      {(void**)&W.seg_geo, 16 * (size_t)ws->scap},
      {(void**)&W.bin_start, 4 * (size_t)(ws->bcap + 1)},
      {(void**)&W.rank, 4 * (size_t)ws->ncap},
      {(void**)&W.seg_start, 4 * (size_t)(ws->scap + 1)},
      {(void**)&W.seg_cur, 4 * (size_t)ws->scap},
      {(void**)&W.rec, 16 * (size_t)ws->ncap},
      {(void**)&W.hyw, ctx->p.packed ? 0 : 8 * (size_t)(ws->ncap + 2)},
      {(void**)&W.hq, ctx->p.packed ? 4 * (size_t)(ws->ncap + 4) : 0},
      {(void**)&W.hcol, ctx->p.packed ? 2 * (size_t)ws->ncap : 0},
      {(void**)&W.horig, 4 * (size_t)ws->ncap},
      {(void**)&W.k2_off, 4 * (size_t)(ws->scap + 1)},
      {(void**)&W.k2_tab, 8 * (size_t)(ws->ncap / 32 + ws->scap + 1)},
      {(void**)&W.links, 8 * (size_t)ws->ncap},
      {(void**)&W.clinks, 8 * (size_t)ws->ncap},
      {(void**)&W.is_start, (size_t)ws->ncap},
      {(void**)&W.seg_nstart, 4 * (size_t)(ws->scap + 1)},
      {(void**)&W.starts_raw, 16 * (size_t)ws->tcap},
      {(void**)&W.starts, 16 * (size_t)ws->tcap},
      {(void**)&W.chains, 16 * (size_t)ws->tcap},
      {(void**)&W.order, 4 * (size_t)ws->tcap},
      {(void**)&W.len_cnt, 4 * (size_t)(kNRow + 2)},
      {(void**)&W.tl_state, 96 * (size_t)ws->tcap},
      {(void**)&W.tl_info, 4 * (size_t)ws->tcap},
      {(void**)&W.slab, 4 * (size_t)kNRow * (size_t)ws->tcap},
      {(void**)&W.hit_w, 8 * (size_t)ws->ncap},
      {(void**)&W.tl_kept, 4 * (size_t)(ws->tcap + 1)},
      {(void**)&W.tl_nkept, 4 * (size_t)(ws->tcap + 1)},
      {(void**)&W.tr_param, 20 * (size_t)ws->tcap},
      {(void**)&W.tr_cov, 60 * (size_t)ws->tcap},
      {(void**)&W.tr_chi2, 4 * (size_t)ws->tcap},
      {(void**)&W.tr_xref, 4 * (size_t)ws->tcap},
      {(void**)&W.tr_sector, 4 * (size_t)ws->tcap},
      {(void**)&W.tr_ndf, 4 * (size_t)ws->tcap},
      {(void**)&W.tr_hoff, 8 * (size_t)ws->tcap},
      {(void**)&W.tr_beam, 20 * (size_t)ws->tcap},
      {(void**)&W.tr_res, compress ? 8 * (size_t)ws->ncap : 0},
      {(void**)&W.tr_npred, compress ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.keep, compress ? (size_t)(ws->ncap + 3) / 4 * 4 : 0},
      {(void**)&W.tr_hits, 4 * (size_t)ws->ncap},
      {(void**)&W.scan_tmp, 4 * (size_t)ws->scan_cap},
      {(void**)&W.m_state, merge ? 80 * (size_t)ws->tcap : 0},
      {(void**)&W.m_info, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.m_bin, merge ? 4 * (size_t)(mbcap + 1) : 0},
      {(void**)&W.m_list, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.m_bestA, merge ? 8 * (size_t)ws->tcap : 0},
      {(void**)&W.m_bestB, merge ? 8 * (size_t)ws->tcap : 0},
      {(void**)&W.m_chi, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.m_next, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.m_prev, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.m_hidx, merge ? 4 * (size_t)(ws->tcap + 1) : 0},
      {(void**)&W.m_hoff, merge ? 4 * (size_t)(ws->tcap + 1) : 0},
      {(void**)&W.mt_param, merge ? 20 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_cov, merge ? 60 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_chi2, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_xref, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_sector, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_ndf, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_nfit, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_nseg, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_head, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_hoff, merge ? 8 * (size_t)ws->tcap : 0},
      {(void**)&W.mt_hits, merge ? 4 * (size_t)ws->ncap : 0},
      {(void**)&W.tr_next, merge ? 4 * (size_t)ws->tcap : 0},
      {(void**)&W.tr_mchi2, merge ? 4 * (size_t)ws->tcap : 0},
  };
  size_t total = 0;
  std::vector<size_t> offs;
  for (auto& it : items) { offs.push_back(total); total = align_up(total + it.bytes, 256); }
  ws->bytes = total;
  if (dry_bytes) {
    *dry_bytes = total;
    return TPC_OK;
  }
  cudaError_t e = cudaMalloc(&ws->block, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TPC_E_NOMEM, "workspace allocation of " + std::to_string(total) + " bytes failed");
  }
  for (size_t k = 0; k < items.size(); ++k) *items[k].ptr = (char*)ws->block + offs[k];
  if (!compress) {
    W.tr_res = nullptr;
    W.tr_npred = nullptr;
    W.keep = nullptr;
  }
  if (!merge) {
    W.m_state = nullptr; W.m_info = nullptr; W.m_bin = nullptr; W.m_list = nullptr; W.m_bestA = nullptr;
    W.m_bestB = nullptr; W.m_chi = nullptr; W.m_next = nullptr; W.m_prev = nullptr; W.m_hidx = nullptr;
    W.m_hoff = nullptr; W.mt_param = nullptr; W.mt_cov = nullptr; W.mt_chi2 = nullptr; W.mt_xref = nullptr;
    W.mt_sector = nullptr; W.mt_ndf = nullptr; W.mt_nfit = nullptr; W.mt_nseg = nullptr; W.mt_head = nullptr;
    W.mt_hoff = nullptr; W.mt_hits = nullptr; W.tr_next = nullptr; W.tr_mchi2 = nullptr;
  }
  W.mbcap = mbcap;
  W.cnt = (DevCounters*)p_cnt;
  ws->d_desc = (BatchDesc*)p_desc;
  W.batch = ws->d_desc;
  W.ncap = ws->ncap; W.scap = ws->scap; W.bcap = ws->bcap; W.tcap = ws->tcap; W.scan_tmp_cap = ws->scan_cap;
  W.k2cap = ws->ncap / 32 + ws->scap + 1;
  W.packed = ctx->p.packed ? 1 : 0;
  W.wide_votes = ctx->p.wide_votes ? 1 : 0;
  CK(cudaMallocHost(&ws->h_desc, sizeof(BatchDesc)));
  CK(cudaMallocHost(&ws->h_cnt, sizeof(DevCounters)));
  memset(ws->h_desc, 0, sizeof(BatchDesc));
  memset(ws->h_cnt, 0, sizeof(DevCounters));
  CK(cudaEventCreateWithFlags(&ws->done, cudaEventDisableTiming));
  out = ws;
  return TPC_OK;
}

int wait_ws(tpc_ctx* ctx, Workspace& ws, double timeout_s);
void release_ws_user(tpc_ctx* ctx, Frame* f);

size_t workspace_bytes(tpc_ctx* ctx, long long ncap, int nf_cap) {
  std::shared_ptr<Workspace> ws;
  size_t b = 0;
  const long long tcap = (long long)std::ceil((double)ncap * ctx->p.tracklet_capacity) + 1024;
  alloc_workspace(ctx, ncap, tcap, nf_cap, ws, &b);
  return b;
}

// Workspace from the pool (a free one large enough), else a new one.
int get_workspace(tpc_ctx* ctx, long long ntot, int nf, std::shared_ptr<Workspace>& out) {
  const long long tneed = (long long)std::ceil((double)ntot * ctx->p.tracklet_capacity) + 1024;
  for (auto& w : ctx->wspool)
    if (!w->busy && w->users == 0 && w->ncap >= ntot && w->tcap >= tneed && w->nf_cap >= nf &&
        w->dp.occ == ctx->shape.occ) {
      out = w;
      return TPC_OK;
    }
  // a busy workspace without result holders becomes free once its run ends: wait (bounded)
  for (auto& w : ctx->wspool)
    if (w->busy && w->users == 0 && w->ncap >= ntot && w->tcap >= tneed && w->nf_cap >= nf &&
        w->dp.occ == ctx->shape.occ) {
      int rc = wait_ws(ctx, *w, 120.0);
      if (rc) return rc;
      out = w;
      return TPC_OK;
    }
  // drop idle workspaces that are too small
  ctx->wspool.erase(std::remove_if(ctx->wspool.begin(), ctx->wspool.end(),
                                   [](const std::shared_ptr<Workspace>& w) { return !w->busy && w->users == 0; }),
                    ctx->wspool.end());
  int nfc = std::max(nf, 1);
  std::shared_ptr<Workspace> ws;
  int rc = alloc_workspace(ctx, ntot + ntot / 8 + 1024, tneed + tneed / 8, nfc, ws);
  if (rc) return rc;
  ctx->wspool.push_back(ws);
  out = ws;
  return TPC_OK;
}


// Enqueue the whole kernel sequence for the batch described in ws->h_desc (already uploaded).
// resident blocks per SM of a kernel shape (cached: the occupancy query is not free); kernel 0 the
// neighbour search (a warps, b staging mode), kernel 1 the tracklets (a threads, b registers, c
// tracklets per lane)
int blocks_per_sm(tpc_ctx* ctx, int kernel, int a, int b, int c = 1) {
  const long long key = ((long long)kernel << 40) | ((long long)c << 36) | ((long long)a << 20) | ((long long)b << 1) |
                        (ctx->p.packed ? 1 : 0);
  auto it = ctx->blocks_cache.find(key);
  if (it != ctx->blocks_cache.end()) return it->second;
  const int nb = kernel == 0 ? neighbours_blocks_per_sm(ctx->p.packed, a, b) : tracklets_blocks_per_sm(a, b, c, ctx->p.packed);
  ctx->blocks_cache[key] = nb;
  return nb;
}

int enqueue_sequence(tpc_ctx* ctx, Workspace& ws, cudaStream_t s, bool timing) {
  Work W = ws.W;
  const DevParams& Q = ws.dp;
  const Shape& sh = ws.shape;
  DevCounters* C = W.cnt;
  const int G = ctx->sms;
  int ki = 0;
  int nl = 0;  // kernel launches of the current stage
  auto mark = [&](int idx) {
    if (idx > 0) ctx->stage_launches[idx - 1] = nl;
    nl = 0;
    if (timing) cudaEventRecord(ctx->ev[idx], s);
  };
  // scan lengths are device-side counts clamped to the buffer capacity n_cap
  // Exclusive scans: arrays of a small capacity in one single-block launch (two of them in one
  // launch where the sequence has a pair), larger ones by reduce / tile scan / apply.
  auto scan2 = [&](const uint32_t* in0, uint32_t* out0, const uint32_t* n0, long long h0, uint32_t* t0,
                   const uint32_t* in1, uint32_t* out1, const uint32_t* n1, long long h1, uint32_t* t1) {
    SmallScan a{{in0, in1}, {out0, out1}, {n0, n1}, {h0, h1}, {t0, t1}};
    nl += 1;
    k_scan_small<<<in1 ? 2 : 1, 1024, 0, s>>>(a);
  };
  auto scan = [&](const uint32_t* in, uint32_t* out, const uint32_t* n_dev, long long n_host, uint32_t* total) {
    if (n_host <= kSmallScanCap) {
      scan2(in, out, n_dev, n_host, total, nullptr, nullptr, nullptr, 0, nullptr);
      return;
    }
    nl += 3;
    k_scan_reduce<<<8 * G, 256, 0, s>>>(in, n_dev, n_host, 0, W.scan_tmp);
    k_scan_tiles<<<1, 1024, 0, s>>>(W.scan_tmp, n_dev, n_host, 0, total);
    k_scan_apply<<<8 * G, 256, 0, s>>>(in, n_dev, n_host, 0, W.scan_tmp, total, out);
  };
  mark(ki++);  // reset
  ++nl; k_reset_counters<<<1, 128, 0, s>>>(W);
  ++nl; k_zero_u32<<<G, 256, 0, s>>>(W.seg_cnt, &C->nseg, W.scap, 0, 1);
  mark(ki++);  // seg_hist
  ++nl; k_seg_hist<<<2 * G, kHistThreads, 0, s>>>(W);
  mark(ki++);  // seg_layout
  ++nl; k_seg_layout<<<G, 256, 0, s>>>(W, Q);
  mark(ki++);  // scan_seg
  if (W.scap <= kSmallScanCap) {
    scan2(W.seg_nb, W.seg_bb, &C->nseg, W.scap, &C->n_bins, W.seg_cnt, W.seg_start, &C->nseg, W.scap, &C->n_sorted);
  } else {
    scan(W.seg_nb, W.seg_bb, &C->nseg, W.scap, &C->n_bins);
    scan(W.seg_cnt, W.seg_start, &C->nseg, W.scap, &C->n_sorted);
  }
  ++nl; k_one_pass_bins<<<1, 1, 0, s>>>(W);
  mark(ki++);  // zero_bins (the one-pass placement's; the per-segment passes zero their own)
  ++nl; k_zero_u32<<<4 * G, 256, 0, s>>>(W.bin_start, &C->n_bins_1p, W.bcap + 1, 1, 1);
  ++nl; k_zero_u32<<<G, 256, 0, s>>>(W.seg_cur, &C->nseg, W.scap, 0, 1);
  mark(ki++);  // bin_rank: one pass for small batches; for large ones the clusters are appended to
  // their segments, then ranked in their bins per segment (each kernel returns at once on the
  // other side of kTwoPassMin, so one captured graph serves every batch size)
  ++nl; k_bin_rank<<<8 * G, 256, 0, s>>>(W, 1);
  ++nl; k_seg_bucket<<<8 * G, 256, 0, s>>>(W);
  ++nl; k_bin_rank_seg<<<2 * G, 1024, 0, s>>>(W);
  mark(ki++);  // scan_bins (the one-pass placement's; the per-segment passes scan in k_bin_rank_seg)
  scan(W.bin_start, W.bin_start, &C->n_bins_1p, W.bcap, &C->scan_sink);
  mark(ki++);  // scatter: one pass, or per segment into the segment's range of sorted positions
  ++nl; k_scatter<<<8 * G, 256, 0, s>>>(W, 1);
  ++nl; k_scatter_seg<<<(G / kScatterParts) * kScatterParts, 1024, 0, s>>>(W);
  mark(ki++);  // neighbours
  ++nl; k_chunk_count<<<G, 256, 0, s>>>(W);
  scan(W.k2_off, W.k2_off, &C->nseg, W.scap, &C->n_chunks);
  ++nl; k_chunk_fill<<<G, 256, 0, s>>>(W);
  ++nl; launch_neighbours(ctx->p.packed, sh.k2_warps, G * std::max(blocks_per_sm(ctx, 0, sh.k2_warps, sh.k2_tma), 1), s,
                          W, Q, sh.k2_tma);
  mark(ki++);  // clean
  ++nl; k_clean<<<8 * G, 256, 0, s>>>(W, Q);
  mark(ki++);  // scan_start
  scan(W.seg_nstart, W.seg_nstart, &C->nseg, W.scap, &C->n_starts);
  mark(ki++);  // starts
  ++nl; k_starts<<<8 * G, 256, 0, s>>>(W, Q);
  ++nl; k_set_ntracklets<<<1, 32, 0, s>>>(W);
  mark(ki++);  // start_order
  ++nl; k_start_order<<<8 * G, 256, 0, s>>>(W);
  mark(ki++);  // chains
  const int order = sh.k5_order;
  if (order) { ++nl; k_zero_u32<<<1, 256, 0, s>>>(W.len_cnt, nullptr, kNRow + 1, 0, 1); }
  ++nl; k_chains<<<4 * G, 256, 0, s>>>(W, order);
  if (order) {
    ++nl; k_length_offsets<<<1, 32, 0, s>>>(W);
    ++nl; k_length_scatter<<<4 * G, 256, 0, s>>>(W, order);
  }
  mark(ki++);  // tracklets
  {
    const int nb = std::max(blocks_per_sm(ctx, 1, sh.k5_block, sh.k5_regs, sh.k5_ilp), 1);
    const int bps = sh.k5_bps > 0 ? std::min(sh.k5_bps, nb) : nb;
    ++nl; launch_tracklets(sh.k5_block, sh.k5_regs, sh.k5_ilp, ctx->p.packed, G * bps, s, W, Q, order ? 1 : 0);
  }
  mark(ki++);  // zero_w
  ++nl; k_zero_u32<<<4 * G, 256, 0, s>>>((uint32_t*)W.hit_w, &C->ntot, 2 * W.ncap, 0, 2);
  mark(ki++);  // votes
  ++nl; launch_votes(sh.sel_lanes, 8 * G, s, W, Q);
  mark(ki++);  // kept
  ++nl; launch_kept(sh.sel_lanes, 8 * G, s, W, Q);
  mark(ki++);  // scan_kept
  if (W.tcap <= kSmallScanCap) {
    scan2(W.tl_kept, W.tl_kept, &C->n_tracklets, W.tcap, &C->n_tracks, W.tl_nkept, W.tl_nkept, &C->n_tracklets,
          W.tcap, &C->n_track_hits);
  } else {
    scan(W.tl_kept, W.tl_kept, &C->n_tracklets, W.tcap, &C->n_tracks);
    scan(W.tl_nkept, W.tl_nkept, &C->n_tracklets, W.tcap, &C->n_track_hits);
  }
  mark(ki++);  // write_tracks
  ++nl; launch_write_tracks(sh.sel_lanes, 8 * G, s, W, Q);
  mark(ki++);  // compress
  if (W.tr_res) {
    ++nl; k_zero_u32<<<2 * G, 256, 0, s>>>((uint32_t*)W.keep, nullptr, (W.ncap + 3) / 4, 0, 1);
    ++nl; launch_compress(ctx->p.packed, 4 * G, s, W, Q);
  }
  mark(ki++);  // beamline
  ++nl; k_beamline<<<2 * G, 256, 0, s>>>(W, Q);
  mark(ki++);  // frame_off
  ++nl; k_frame_offsets<<<1, 128, 0, s>>>(W);
  mark(ki++);  // merge
  if (W.m_state) {
    ++nl; k_zero_u32<<<2 * G, 256, 0, s>>>(W.m_bin, nullptr, W.mbcap + 1, 0, 1);
    ++nl; k_merge_outer<<<4 * G, 256, 0, s>>>(W, Q);
    scan(W.m_bin, W.m_bin, nullptr, W.mbcap, &C->n_merge_bins);
    ++nl; k_merge_fill<<<2 * G, 256, 0, s>>>(W);
    ++nl; k_merge_match<<<4 * G, 256, 0, s>>>(W, Q);
    ++nl; k_merge_link<<<2 * G, 256, 0, s>>>(W);
    ++nl; k_merge_heads<<<2 * G, 256, 0, s>>>(W);
    if (W.tcap <= kSmallScanCap) {
      scan2(W.m_hidx, W.m_hidx, &C->n_tracks, W.tcap, &C->n_merged, W.m_hoff, W.m_hoff, &C->n_tracks, W.tcap,
            &C->n_merged_hits);
    } else {
      scan(W.m_hidx, W.m_hidx, &C->n_tracks, W.tcap, &C->n_merged);
      scan(W.m_hoff, W.m_hoff, &C->n_tracks, W.tcap, &C->n_merged_hits);
    }
    ++nl; k_merge_refit<<<5 * G, 128, 0, s>>>(W, Q);
    ++nl; k_merge_frames<<<1, 128, 0, s>>>(W);
  }
  ctx->stage_launches[kNumKernels - 1] = nl;
  if (timing) cudaEventRecord(ctx->ev[kNumKernels], s);
  cudaMemcpyAsync(ws.h_cnt, W.cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return TPC_OK;
}

// A workspace's graph is valid for the launch shape it was captured with; occupancy is fixed by
// its allocation (a workspace of another occupancy is never handed out for a shape).
void set_shape(Workspace& ws, const Shape& want) {
  Shape sh = want;
  sh.occ = ws.dp.occ;
  if (ws.shape == sh) return;
  if (ws.graph) cudaGraphExecDestroy(ws.graph);
  ws.graph = nullptr;
  ws.shape = sh;
}

// The kernel sequence on stream s: a replay of the workspace's graph (captured on first use, on
// the context's non-default stream; replays may go to any stream), or eager launches when graphs
// are off or per-stage timing is on.
int launch_ws(tpc_ctx* ctx, Workspace& ws, cudaStream_t s) {
  if (!ctx->p.use_graphs || ctx->timing) return enqueue_sequence(ctx, ws, s, ctx->timing);
  if (!ws.graph) {
    cudaStream_t cs = ctx->stream;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_sequence(ctx, ws, cs, false);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ws.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  CK(cudaGraphLaunch(ws.graph, s));
  return TPC_OK;
}

int run_batch(tpc_ctx* ctx, const std::vector<Frame*>& fr, cudaStream_t s, std::shared_ptr<Workspace>& ws_out,
              std::shared_ptr<Workspace> fixed = nullptr) {
  // The same batch tracked again on the same workspace (e.g. a frame re-tracked in a loop): the
  // descriptor in device memory is already right and the stream orders the runs.
  if (!fixed) {
    std::shared_ptr<Workspace> same = fr[0]->ws;
    bool reuse = same && same->batch_ids.size() == fr.size() && same->dp.occ == ctx->shape.occ;
    for (size_t k = 0; reuse && k < fr.size(); ++k) reuse = fr[k]->ws == same && same->batch_ids[k] == fr[k]->id;
    if (reuse) {
      same->busy = true;
      set_shape(*same, ctx->shape);
      int rc = launch_ws(ctx, *same, s);
      if (rc) return rc;
      CK(cudaEventRecord(same->done, s));
      for (Frame* f : fr) f->state = 3;
      ws_out = same;
      return TPC_OK;
    }
  }
  for (Frame* f : fr) release_ws_user(ctx, f);
  long long ntot = 0;
  for (auto* f : fr) ntot += f->n;
  std::shared_ptr<Workspace> ws = fixed;
  int rc = TPC_OK;
  if (!ws) rc = get_workspace(ctx, ntot, (int)fr.size(), ws);
  if (rc) return rc;
  ws->batch_ids.clear();
  for (auto* f : fr) ws->batch_ids.push_back(f->id);
  BatchDesc* d = ws->h_desc;
  memset(d, 0, sizeof(BatchDesc));
  d->nf = (int)fr.size();
  long long off = 0;
  for (size_t k = 0; k < fr.size(); ++k) {
    FrameIn& fi = d->f[k];
    fi.sector = fr[k]->d_sector; fi.row = fr[k]->d_row; fi.y = fr[k]->d_y; fi.w = fr[k]->d_w;
    fi.n = fr[k]->n; fi.off = off;
    off += fr[k]->n;
  }
  d->ntot = ntot;
  ws->busy = true;
  CK(cudaMemcpyAsync(ws->d_desc, d, sizeof(BatchDesc), cudaMemcpyHostToDevice, s));
  set_shape(*ws, ctx->shape);
  rc = launch_ws(ctx, *ws, s);
  if (rc) return rc;
  CK(cudaEventRecord(ws->done, s));
  for (size_t k = 0; k < fr.size(); ++k) {
    fr[k]->ws = ws;
    fr[k]->fidx = (int)k;
    fr[k]->state = 3;
    ws->users++;
  }
  ws_out = ws;
  return TPC_OK;
}

// bounded wait for a workspace's run; collects the kernel times when timing is on
int wait_ws(tpc_ctx* ctx, Workspace& ws, double timeout_s) {
  const double t0 = now_s();
  for (;;) {
    cudaError_t e = cudaEventQuery(ws.done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return fail(ctx, TPC_E_CUDA, std::string("device: ") + cudaGetErrorString(e));
    if (now_s() - t0 > timeout_s) return fail(ctx, TPC_E_TIMEOUT, "tracking did not complete in time");
    std::this_thread::yield();
  }
  ws.busy = false;
  if (ctx->timing) {
    for (int k = 0; k < kNumKernels; ++k) {
      float m = 0;
      if (cudaEventElapsedTime(&m, ctx->ev[k], ctx->ev[k + 1]) == cudaSuccess) ctx->ms[k] = m;
    }
  }
  return TPC_OK;
}

int wait_event(tpc_ctx* ctx, cudaEvent_t e, double timeout_s) {
  const double t0 = now_s();
  for (;;) {
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) return TPC_OK;
    if (q != cudaErrorNotReady) return fail(ctx, TPC_E_CUDA, std::string("device: ") + cudaGetErrorString(q));
    if (now_s() - t0 > timeout_s) return fail(ctx, TPC_E_TIMEOUT, "copy did not complete in time");
    std::this_thread::yield();
  }
}

int check_ws_errors(tpc_ctx* ctx, const Workspace& ws) {
  const DevCounters& c = *ws.h_cnt;
  if (c.err & kErrInput) return fail(ctx, TPC_E_INVAL, "malformed cluster (sector >= 36, row >= 152 or non-finite y/w)");
  if (c.err & kErrTimeout) return fail(ctx, TPC_E_TIMEOUT, "a bounded shared-memory copy wait expired");
  if (c.err & (kErrBins | kErrTracks)) return fail(ctx, TPC_E_CAPACITY, "grid or output capacity exceeded");
  return TPC_OK;
}

Frame* find_frame(tpc_ctx* ctx, tpc_frame_t h) {
  auto it = ctx->frames.find(h);
  return it == ctx->frames.end() ? nullptr : it->second.get();
}

void release_results(tpc_ctx* ctx, Frame* f) {
  ctx->pinned.put(f->res, f->res_cap);
  f->res = nullptr;
  f->res_cap = 0;
  f->n_tracks = 0;
}

// Layout of a frame's results in its page-locked block: the output arrays, each copied from the
// workspace's track arrays as one block.
struct ResLayout {
  size_t hits, sec, ndf, xref, chi2, par, cov, hoff, beam, res, npred;
  size_t mhits, msec, mnseg, mhead, mndf, mnfit, mxref, mpar, mcov, mchi2, mhoff, tnext, tmchi2, bytes;
};
ResLayout res_layout(size_t nt, size_t nh, bool compress, size_t nm = 0, size_t nmh = 0, bool merge = false) {
  ResLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, 256); return o; };
  L.hits = take(nh * 4); L.sec = take(nt * 4); L.ndf = take(nt * 4); L.xref = take(nt * 4);
  L.chi2 = take(nt * 4); L.par = take(nt * 20); L.cov = take(nt * 60); L.hoff = take((nt + 1) * 8);
  L.beam = take(nt * 20);
  L.res = take(compress ? nh * 8 : 0);
  L.npred = take(compress ? nt * 4 : 0);
  if (!merge) nm = nmh = 0;
  L.mhits = take(nmh * 4); L.msec = take(nm * 4); L.mnseg = take(nm * 4); L.mhead = take(nm * 4);
  L.mndf = take(nm * 4); L.mnfit = take(nm * 4); L.mxref = take(nm * 4); L.mpar = take(nm * 20);
  L.mcov = take(nm * 60); L.mchi2 = take(nm * 4); L.mhoff = take(merge ? (nm + 1) * 8 : 0);
  L.tnext = take(merge ? nt * 4 : 0); L.tmchi2 = take(merge ? nt * 4 : 0);
  L.bytes = off;
  return L;
}

// The frame's tracks into one page-locked block, step 1: the DMA of the track arrays, queued on
// stream s (work queued after it on s may reuse the workspace). The frame's batch has finished.
int fetch_enqueue(tpc_ctx* ctx, Frame* f, cudaStream_t s) {
  Workspace& ws = *f->ws;
  const DevCounters& c = *ws.h_cnt;
  const int k = f->fidx;
  const uint32_t t0 = c.frame_track0[k], t1 = c.frame_track0[k + 1];
  const uint32_t h0 = c.frame_hit0[k], h1 = c.frame_hit0[k + 1];
  const size_t nt = t1 - t0, nh = h1 - h0;
  const bool compress = ws.W.tr_res != nullptr;
  const bool merge = ws.W.m_state != nullptr;
  const uint32_t m0 = merge ? c.frame_merged0[k] : 0, mh0 = merge ? c.frame_mhit0[k] : 0;
  const size_t nm = merge ? c.frame_merged0[k + 1] - m0 : 0, nmh = merge ? c.frame_mhit0[k + 1] - mh0 : 0;
  const ResLayout L = res_layout(nt, nh, compress, nm, nmh, merge);
  release_results(ctx, f);
  size_t cap = 0;
  char* b = (char*)ctx->pinned.get(L.bytes, cap);
  if (!b) return fail(ctx, TPC_E_NOMEM, "page-locked result allocation failed");
  f->res = b;
  f->res_cap = cap;
  f->fetch_nt = nt;
  f->fetch_nh = nh;
  f->fetch_h0 = h0;
  f->fetch_compress = compress;
  f->fetch_merge = merge;
  f->fetch_nm = nm;
  f->fetch_nmh = nmh;
  f->fetch_mh0 = mh0;
  const Work& W = ws.W;
  const auto d2h = [&](size_t o, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(b + o, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
  };
  CK(d2h(L.par, W.tr_param + (size_t)t0 * 5, nt * 20));
  CK(d2h(L.cov, W.tr_cov + (size_t)t0 * 15, nt * 60));
  CK(d2h(L.chi2, W.tr_chi2 + t0, nt * 4));
  CK(d2h(L.xref, W.tr_xref + t0, nt * 4));
  CK(d2h(L.sec, W.tr_sector + t0, nt * 4));
  CK(d2h(L.ndf, W.tr_ndf + t0, nt * 4));
  CK(d2h(L.hoff, W.tr_hoff + t0, nt * 8));
  CK(d2h(L.beam, W.tr_beam + (size_t)t0 * 5, nt * 20));
  CK(d2h(L.hits, W.tr_hits + h0, nh * 4));
  if (compress) {
    CK(d2h(L.res, W.tr_res + 2 * (size_t)h0, nh * 8));
    CK(d2h(L.npred, W.tr_npred + t0, nt * 4));
  }
  if (merge) {
    CK(d2h(L.mhits, W.mt_hits + mh0, nmh * 4));
    CK(d2h(L.msec, W.mt_sector + m0, nm * 4));
    CK(d2h(L.mnseg, W.mt_nseg + m0, nm * 4));
    CK(d2h(L.mhead, W.mt_head + m0, nm * 4));
    CK(d2h(L.mndf, W.mt_ndf + m0, nm * 4));
    CK(d2h(L.mnfit, W.mt_nfit + m0, nm * 4));
    CK(d2h(L.mxref, W.mt_xref + m0, nm * 4));
    CK(d2h(L.mpar, W.mt_param + (size_t)m0 * 5, nm * 20));
    CK(d2h(L.mcov, W.mt_cov + (size_t)m0 * 15, nm * 60));
    CK(d2h(L.mchi2, W.mt_chi2 + m0, nm * 4));
    CK(d2h(L.mhoff, W.mt_hoff + m0, nm * 8));
    CK(d2h(L.tnext, W.tr_next + t0, nt * 4));
    CK(d2h(L.tmchi2, W.tr_mchi2 + t0, nt * 4));
  }
  return TPC_OK;
}

// Step 2, once the copies have completed: the arrays' views, hit offsets made frame-relative.
void fetch_finish(Frame* f) {
  const size_t nt = f->fetch_nt, nh = f->fetch_nh;
  const ResLayout L = res_layout(nt, nh, f->fetch_compress, f->fetch_nm, f->fetch_nmh, f->fetch_merge);
  char* b = (char*)f->res;
  f->hits = (uint32_t*)(b + L.hits);
  f->sector = (int32_t*)(b + L.sec);
  f->ndf = (int32_t*)(b + L.ndf);
  f->xref = (float*)(b + L.xref);
  f->chi2 = (float*)(b + L.chi2);
  f->param = (float*)(b + L.par);
  f->cov = (float*)(b + L.cov);
  f->hoff = (int64_t*)(b + L.hoff);
  f->beam = (float*)(b + L.beam);
  f->residual = f->fetch_compress ? (int32_t*)(b + L.res) : nullptr;
  f->n_pred = f->fetch_compress ? (int32_t*)(b + L.npred) : nullptr;
  if (f->fetch_h0)
    for (size_t i = 0; i < nt; ++i) f->hoff[i] -= (int64_t)f->fetch_h0;
  f->hoff[nt] = (int64_t)nh;
  f->n_tracks = (int64_t)nt;
  if (f->fetch_merge) {
    const size_t nm = f->fetch_nm;
    f->m_hits = (uint32_t*)(b + L.mhits);
    f->m_sector = (int32_t*)(b + L.msec);
    f->m_nseg = (int32_t*)(b + L.mnseg);
    f->m_head = (int32_t*)(b + L.mhead);
    f->m_ndf = (int32_t*)(b + L.mndf);
    f->m_nfit = (int32_t*)(b + L.mnfit);
    f->m_xref = (float*)(b + L.mxref);
    f->m_param = (float*)(b + L.mpar);
    f->m_cov = (float*)(b + L.mcov);
    f->m_chi2 = (float*)(b + L.mchi2);
    f->m_hoff = (int64_t*)(b + L.mhoff);
    f->tr_next = (int32_t*)(b + L.tnext);
    f->tr_mchi2 = (float*)(b + L.tmchi2);
    for (size_t i = 0; i < nm; ++i) f->m_hoff[i] -= (int64_t)f->fetch_mh0;
    f->m_hoff[nm] = (int64_t)f->fetch_nmh;
    f->n_merged = (int64_t)nm;
  }
  f->state = 5;
}

int fetch_results(tpc_ctx* ctx, Frame* f) {
  int rc = fetch_enqueue(ctx, f, ctx->stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  fetch_finish(f);
  return TPC_OK;
}

// Finished result copies of retired batches: split the fit rows and hand the frames to tpc_poll
// (wait: block until every copy in flight has completed).
int finish_fetches(tpc_ctx* ctx, bool wait) {
  while (!ctx->fetching.empty()) {
    auto& fe = ctx->fetching.front();
    cudaError_t e = wait ? cudaEventSynchronize(fe.ev) : cudaEventQuery(fe.ev);
    if (e == cudaErrorNotReady) break;
    if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("device: ") + cudaGetErrorString(e));
    for (auto id : fe.frames) {
      Frame* f = find_frame(ctx, id);
      if (!f) continue;
      fetch_finish(f);
      f->t_done = now_s();
      ctx->finished.push_back(id);
    }
    ctx->spare_events.push_back(fe.ev);
    ctx->fetching.pop_front();
  }
  return TPC_OK;
}

void release_ws_user(tpc_ctx* ctx, Frame* f) {
  if (f->ws) {
    f->ws->users--;
    f->ws.reset();
  }
  (void)ctx;
}

int load_frame(tpc_ctx* ctx, const tpc_clusters* cl, Frame*& out) {
  if (!cl || cl->n < 0 || cl->n >= (1LL << 31)) return fail(ctx, TPC_E_INVAL, "bad cluster descriptor");
  if (cl->n > 0 && (!cl->sector || !cl->row || !cl->y || !cl->w)) return fail(ctx, TPC_E_INVAL, "null cluster array");
  if (cl->on_device < 0 || cl->on_device > 2) return fail(ctx, TPC_E_INVAL, "bad on_device value");
  auto f = std::make_unique<Frame>();
  f->n = cl->n;
  if (cl->on_device == 1) {
    f->d_sector = (uint8_t*)cl->sector; f->d_row = (uint8_t*)cl->row;
    f->d_y = (float*)cl->y; f->d_w = (float*)cl->w;
  } else {
    const size_t n = (size_t)cl->n;
    const size_t o1 = align_up(n, 256), o2 = o1 + align_up(n, 256), o3 = o2 + align_up(4 * n, 256);
    const size_t bytes = o3 + align_up(4 * n, 256) + 256;
    cudaError_t e = cudaMallocFromPoolAsync(&f->d_block, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(ctx, TPC_E_NOMEM, "input allocation failed"); }
    char* b = (char*)f->d_block;
    f->d_sector = (uint8_t*)b; f->d_row = (uint8_t*)(b + o1); f->d_y = (float*)(b + o2); f->d_w = (float*)(b + o3);
    if (n) {
      CK(cudaMemcpyAsync(f->d_sector, cl->sector, n, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(f->d_row, cl->row, n, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(f->d_y, cl->y, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(f->d_w, cl->w, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    }
  }
  f->id = ctx->next_id++;
  out = f.get();
  ctx->frames[f->id] = std::move(f);
  return TPC_OK;
}

void drop_frame(tpc_ctx* ctx, Frame* f) {
  auto it = std::find(ctx->finished.begin(), ctx->finished.end(), f->id);
  if (it != ctx->finished.end()) ctx->finished.erase(it);
  if (f->d_block) cudaFreeAsync(f->d_block, ctx->stream);
  release_results(ctx, f);
  release_ws_user(ctx, f);
  ctx->frames.erase(f->id);
}


// ------------------------------------------------------------------------- cluster finding

// pads of a row: 2 ceil(x_r tan(10 deg) / pitch), in double
int cf_npads(double pitch, int r) {
  const double x = 85.0 + (double)r * (160.0 / 151.0);
  return 2 * (int)std::ceil(x * std::tan(10.0 * 3.14159265358979323846 / 180.0) / pitch);
}

// device buffers for n digits (one allocation; grown by 1/8 beyond the request)
int cf_reserve(tpc_ctx* ctx, long long n) {
  CfState& cf = ctx->cf;
  if (cf.dev && cf.cap >= n) return TPC_OK;
  const long long cap = std::max<long long>(n + n / 8, 1 << 16);
  // temporary slots: the peak kernel's blocks (at most 8 per SM) each own a region of whole tiles
  const long long nw = (cap + 31) / 32, cap32 = nw * 32 + (long long)ctx->sms * 8 * kCfTile;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_is = take(cap), o_ir = take(cap), o_ip = take(2 * cap), o_it = take(2 * cap), o_ia = take(2 * cap);
  const size_t o_wc = take(4 * nw), o_wo = take(4 * (nw + 1)), o_ws = take(4 * nw), o_wf = take(4 * nw);
  const size_t o_gl = take(4 * 2 * nw), o_gw = take(4 * nw), o_gn = take(4 * nw);
  const size_t o_gc = take(4 * 3 * (size_t)(kCfMaxWindows + 1));
  const size_t o_tmp = take(4 * (nw / 2048 + 2)), o_small = take(16), o_np = take(2 * kNRow);
  const size_t t_s = take(cap32), t_r = take(cap32), t_y = take(4 * cap32), t_w = take(4 * cap32);
  const size_t t_sp = take(4 * cap32), t_st = take(4 * cap32), t_q = take(4 * cap32), t_d = take(4 * cap32);
  const size_t t_qm = take(2 * cap32);
  const size_t o_os = take(cap), o_or = take(cap), o_y = take(4 * cap), o_w = take(4 * cap), o_sp = take(4 * cap);
  const size_t o_st = take(4 * cap), o_q = take(4 * cap), o_d = take(4 * cap), o_qm = take(2 * cap);
  if (cf.dev) {
    cudaFree(cf.dev);
    cf.dev = nullptr;
    cf.cap = 0;
  }
  if (cudaMalloc(&cf.dev, off) != cudaSuccess) {
    cudaGetLastError();
    cf.dev = nullptr;
    return fail(ctx, TPC_E_NOMEM, "cluster-finder buffers of " + std::to_string(off) + " bytes");
  }
  char* b = static_cast<char*>(cf.dev);
  cf.in_sector = (uint8_t*)(b + o_is);
  cf.in_row = (uint8_t*)(b + o_ir);
  cf.in_pad = (uint16_t*)(b + o_ip);
  cf.in_time = (uint16_t*)(b + o_it);
  cf.in_adc = (uint16_t*)(b + o_ia);
  cf.wcount = (uint32_t*)(b + o_wc);
  cf.woff = (uint32_t*)(b + o_wo);
  cf.wsrc = (uint32_t*)(b + o_ws);
  cf.wflag = (uint32_t*)(b + o_wf);
  cf.glist = (uint32_t*)(b + o_gl);
  cf.gwide = (uint32_t*)(b + o_gw);
  cf.gwin = (uint32_t*)(b + o_gn);
  cf.gcnt = (uint32_t*)(b + o_gc);
  cf.gbeg = cf.gcnt + (kCfMaxWindows + 1);
  cf.gcur = cf.gbeg + (kCfMaxWindows + 1);
  cf.t_sector = (uint8_t*)(b + t_s);
  cf.t_row = (uint8_t*)(b + t_r);
  cf.t_y = (float*)(b + t_y);
  cf.t_w = (float*)(b + t_w);
  cf.t_sp = (float*)(b + t_sp);
  cf.t_st = (float*)(b + t_st);
  cf.t_qtot = (uint32_t*)(b + t_q);
  cf.t_digit = (uint32_t*)(b + t_d);
  cf.t_qmax = (uint16_t*)(b + t_qm);
  cf.scan_tmp = (uint32_t*)(b + o_tmp);
  cf.small = (uint32_t*)(b + o_small);
  cf.npads = (uint16_t*)(b + o_np);
  cf.o_sector = (uint8_t*)(b + o_os);
  cf.o_row = (uint8_t*)(b + o_or);
  cf.o_y = (float*)(b + o_y);
  cf.o_w = (float*)(b + o_w);
  cf.o_sp = (float*)(b + o_sp);
  cf.o_st = (float*)(b + o_st);
  cf.o_qtot = (uint32_t*)(b + o_q);
  cf.o_digit = (uint32_t*)(b + o_d);
  cf.o_qmax = (uint16_t*)(b + o_qm);
  cf.cap = cap;
  return TPC_OK;
}

// the charge map for a geometry (zero everywhere): reused while it is clean and large enough
int cf_map(tpc_ctx* ctx, int lines, int stride, cudaStream_t s) {
  CfState& cf = ctx->cf;
  const size_t need = (size_t)kSegPerFrame * (size_t)lines * (size_t)stride * 2;
  if (need > (size_t)std::max<int64_t>(ctx->p.hbm_budget, 0) / 2)
    return fail(ctx, TPC_E_BUDGET, "charge map of " + std::to_string(need) + " bytes exceeds half of the HBM budget");
  if (!cf.map || cf.map_bytes < need) {
    if (cf.map) cudaFree(cf.map);
    cf.map = nullptr;
    cf.map_bytes = 0;
    cf.map_clean = false;
    if (cudaMalloc(&cf.map, need) != cudaSuccess) {
      cudaGetLastError();
      cf.map = nullptr;
      return fail(ctx, TPC_E_NOMEM, "charge map of " + std::to_string(need) + " bytes");
    }
    cf.map_bytes = need;
  }
  if (!cf.map_clean) {
    CK(cudaMemsetAsync(cf.map, 0, cf.map_bytes, s));
    cf.map_clean = true;
  }
  cf.lines = lines;
  cf.stride = stride;
  return TPC_OK;
}

}  // namespace

// ============================================================================== C-ABI
extern "C" {

void tpc_default_params(tpc_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(tpc_params);
  p->bz = 0.5;
  p->ky = 2.0; p->kw = 2.4; p->eps = 0.5;
  p->chi_n_max = 0.2;
  p->lmin = 6;
  p->sigma_y = 0.1; p->sigma_w = 0.1;
  p->chi2_hit_max = 16.0;
  p->n_miss_max = 5;
  p->win_nsig = 3.0; p->win_add = 0.3;
  p->x0_per_row = 0.03 / 152.0;
  p->max_sin = 0.999;
  p->y_margin = 1.0;
  p->nmin = 10;
  p->cov0[0] = 1.0; p->cov0[1] = 1.0; p->cov0[2] = 1.0; p->cov0[3] = 1.0; p->cov0[4] = 100.0;
  p->ext_stop = 1;
  p->drift_length = 250.0;
  p->drift_velocity = 250.0 / 90.0;
  p->keep_vy = 1.0;
  p->keep_vw = 1.0;
  p->keep_qpt_max = 20.0;
  p->packed = 0;
  p->bin_occupancy = 1.0f;
  p->tracklet_capacity = 0.08f;
  p->hbm_budget = 80LL << 30;
  p->max_batch_frames = 16;
  p->use_graphs = 1;
  p->k2_warps = 8;
  p->k2_tma = 1;
  p->k5_block = 128;
  p->k5_regs = 80;
  p->k5_blocks_per_sm = 0;
  p->k5_order = 1;
  p->sel_lanes = 32;
  p->autotune = 0;
  p->merge = 0;
  p->merge_gap_rows = 10;
  p->merge_dw = 5.0;
  p->merge_chi2_max = 50.0;
  p->refit_passes = 3;
  p->refit_scale = 100.0;
  p->k5_ilp = 1;
  p->wide_votes = 0;
}

const char* tpc_version(void) { return "tpctrack 0.1 (sm_103a)"; }

// the tracklet kernel shapes that are compiled (k_tracklet.cu)
static bool k5_shape_compiled(int block, int regs, int ilp) {
  if (ilp == 1) return (block == 64 || block == 128 || block == 256) && (regs == 64 || regs == 72 || regs == 80);
  if (ilp == 2) return (block == 64 || block == 128) && regs == 128;
  return false;
}

int tpc_create(const tpc_params* p, tpc_ctx** out) {
  if (!out) return TPC_E_INVAL;
  *out = nullptr;
  tpc_ctx* ctx = new tpc_ctx();
  if (p) {
    if (p->struct_size != sizeof(tpc_params)) { delete ctx; return TPC_E_INVAL; }
    ctx->p = *p;
  } else {
    tpc_default_params(&ctx->p);
  }
  const tpc_params& q = ctx->p;
  if (q.nmin < 1 || q.lmin < 3 || q.n_miss_max < 1 || !(q.tracklet_capacity > 0) || q.max_batch_frames < 1 ||
      q.max_batch_frames > kMaxFrames || (q.k2_warps != 4 && q.k2_warps != 8) ||
      !k5_shape_compiled(q.k5_block, q.k5_regs, q.k5_ilp) || q.wide_votes < 0 || q.wide_votes > 1 ||
      q.k2_tma < 0 || q.k2_tma > 2 || (q.sel_lanes != 1 && q.sel_lanes != 32) ||
      q.k5_blocks_per_sm < 0 || q.k5_order < 0 || q.k5_order > 3 || q.bin_occupancy > 64.0f ||
      q.merge_gap_rows < 1 || q.merge_gap_rows > 150 || !(q.merge_dw >= 0) || !(q.merge_chi2_max >= 0) ||
      q.refit_passes < 1 || q.refit_passes % 2 == 0 || q.refit_passes > 15 || !(q.refit_scale > 0)) {
    delete ctx;
    return TPC_E_INVAL;
  }
  ctx->shape.occ = q.bin_occupancy > 0 ? q.bin_occupancy : 2.0f;
  ctx->shape.k2_warps = q.k2_warps;
  ctx->shape.k2_tma = q.k2_tma;
  ctx->shape.k5_block = q.k5_block;
  ctx->shape.k5_regs = q.k5_regs;
  ctx->shape.k5_bps = q.k5_blocks_per_sm;
  ctx->shape.k5_order = q.k5_order;
  ctx->shape.k5_ilp = q.k5_ilp;
  ctx->shape.sel_lanes = q.sel_lanes;
  make_dev_params(ctx->p, ctx->dp);
  int rc = TPC_OK;
  do {
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) { rc = fail(ctx, TPC_E_CUDA, "no CUDA device"); break; }
    e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) { rc = fail(ctx, TPC_E_CUDA, "device query failed"); break; }
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = TPC_E_CUDA; break; }
    prepare_neighbours();
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) { rc = fail(ctx, TPC_E_CUDA, "memory pool"); break; }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    for (int k = 0; k <= kNumKernels; ++k) cudaEventCreate(&ctx->ev[k]);
    cudaEventCreateWithFlags(&ctx->ev_sync, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ctx->ev_track, cudaEventDisableTiming);
    ctx->slots.resize(2);
    for (auto& sl : ctx->slots) cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    // slot capacity: the largest batch whose workspace and inputs fit half of the HBM budget at
    // the finest grid the autotuner may choose (the grid's bin arrays grow as the occupancy falls)
    {
      const float occ0 = ctx->shape.occ;
      ctx->shape.occ = std::min(occ0, kTunerOccupancies[0]);
      const size_t half = (size_t)std::max<int64_t>(ctx->p.hbm_budget, 1 << 20) / ctx->slots.size();
      long long lo = 0, hi = 1LL << 31;
      while (lo < hi) {
        const long long mid = lo + (hi - lo + 1) / 2;
        const size_t need = workspace_bytes(ctx, mid, ctx->p.max_batch_frames) + (size_t)mid * 10;
        if (need <= half) lo = mid; else hi = mid - 1;
      }
      ctx->slot_clusters = lo;
      ctx->shape.occ = occ0;
    }
    if (cudaGetLastError() != cudaSuccess) { rc = fail(ctx, TPC_E_CUDA, "context setup failed"); break; }
  } while (0);
  if (rc) { tpc_destroy(ctx); return rc; }
  *out = ctx;
  return TPC_OK;
}

void tpc_destroy(tpc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& sl : ctx->slots) {
    if (!sl.stream) continue;
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
  }
  for (auto& kv : ctx->frames) {
    if (kv.second->d_block) cudaFreeAsync(kv.second->d_block, ctx->stream);
    if (kv.second->res) cudaFreeHost(kv.second->res);
  }
  ctx->frames.clear();
  ctx->pinned.clear();
  ctx->slots.clear();
  for (auto& fe : ctx->fetching) cudaEventDestroy(fe.ev);
  for (auto ev : ctx->spare_events) cudaEventDestroy(ev);
  ctx->fetching.clear();
  ctx->spare_events.clear();
  ctx->wspool.clear();
  if (ctx->stream) { cudaStreamSynchronize(ctx->stream); cudaStreamDestroy(ctx->stream); }
  for (int k = 0; k <= kNumKernels; ++k)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  if (ctx->ev_sync) cudaEventDestroy(ctx->ev_sync);
  if (ctx->ev_track) cudaEventDestroy(ctx->ev_track);
  CfState& cf = ctx->cf;
  if (cf.dev) cudaFree(cf.dev);
  if (cf.map) cudaFree(cf.map);
  if (cf.h_small) cudaFreeHost(cf.h_small);
  if (cf.host) cudaFreeHost(cf.host);
  for (auto& e : cf.ev)
    if (e) cudaEventDestroy(e);
  if (cf.done) cudaEventDestroy(cf.done);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
}

const char* tpc_last_error(const tpc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tpc_load_clusters(tpc_ctx* ctx, const tpc_clusters* clusters, tpc_frame_t* out) {
  if (!ctx || !out) return TPC_E_INVAL;
  Frame* f = nullptr;
  int rc = load_frame(ctx, clusters, f);
  if (rc) return rc;
  *out = f->id;
  return TPC_OK;
}

int tpc_track_batch(tpc_ctx* ctx, const tpc_frame_t* frames, int32_t n_frames, void* cuda_stream) {
  if (!ctx || !frames || n_frames < 1 || n_frames > kMaxFrames) return fail(ctx, TPC_E_INVAL, "bad frame list");
  std::vector<Frame*> fr;
  for (int k = 0; k < n_frames; ++k) {
    Frame* f = find_frame(ctx, frames[k]);
    if (!f) return fail(ctx, TPC_E_INVAL, "unknown frame handle");
    if (f->state == 1 || f->state == 2) return fail(ctx, TPC_E_STATE, "frame is queued for serving");
    for (Frame* g : fr)
      if (g == f) return fail(ctx, TPC_E_INVAL, "frame listed twice");
    fr.push_back(f);
  }
  // The kernels run on the caller's stream (NULL: the context's stream), after the uploads that
  // tpc_load_clusters queued on the context's stream.
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  if (s != ctx->stream) {
    CK(cudaEventRecord(ctx->ev_sync, ctx->stream));
    CK(cudaStreamWaitEvent(s, ctx->ev_sync, 0));
  }
  if (ctx->p.autotune && !ctx->tuned) {
    int rc = tpc_autotune(ctx, frames, n_frames, 3, nullptr);
    if (rc) return rc;
  }
  std::shared_ptr<Workspace> ws;
  return run_batch(ctx, fr, s, ws);
}

int tpc_track_sectors(tpc_ctx* ctx, tpc_frame_t frame, void* cuda_stream) {
  return tpc_track_batch(ctx, &frame, 1, cuda_stream);
}

int tpc_get_tracks(tpc_ctx* ctx, tpc_frame_t frame, tpc_tracks* out) {
  if (!ctx || !out) return TPC_E_INVAL;
  Frame* f = find_frame(ctx, frame);
  if (!f) return fail(ctx, TPC_E_INVAL, "unknown frame handle");
  if (f->state == 4) {  // served, results in copy
    int rc = finish_fetches(ctx, true);
    if (rc) return rc;
  }
  if (f->state < 3) return fail(ctx, TPC_E_STATE, "frame has not been tracked");
  if (f->state < 5) {
    int rc = wait_ws(ctx, *f->ws, 120.0);
    if (rc) return rc;
    rc = check_ws_errors(ctx, *f->ws);
    if (rc) return rc;
    if (f->ws->h_cnt->n_starts > (uint32_t)f->ws->tcap) {
      // tracklet capacity overflow: track this frame again alone with room for every start hit
      const float old = ctx->p.tracklet_capacity;
      ctx->p.tracklet_capacity = std::max(old, 1.25f * (float)f->ws->h_cnt->n_starts / (float)std::max(1LL, f->n));
      release_ws_user(ctx, f);
      f->ws.reset();
      std::vector<Frame*> one{f};
      std::shared_ptr<Workspace> ws;
      rc = run_batch(ctx, one, ctx->stream, ws);
      ctx->p.tracklet_capacity = old;
      if (rc) return rc;
      rc = wait_ws(ctx, *f->ws, 120.0);
      if (rc) return rc;
      rc = check_ws_errors(ctx, *f->ws);
      if (rc) return rc;
      if (f->ws->h_cnt->n_starts > (uint32_t)f->ws->tcap) return fail(ctx, TPC_E_CAPACITY, "tracklet capacity");
    }
    rc = fetch_results(ctx, f);
    if (rc) return rc;
  }
  static const int64_t zero_offset = 0;
  out->n_tracks = f->n_tracks;
  out->sector = f->sector;
  out->x_ref = f->xref;
  out->param = f->param;
  out->cov = f->cov;
  out->chi2 = f->chi2;
  out->ndf = f->ndf;
  out->hit_offset = f->hoff ? f->hoff : &zero_offset;
  out->hit_index = f->hits;
  out->beam = f->beam;
  out->residual = f->residual;
  out->n_pred = f->n_pred;
  return TPC_OK;
}

int tpc_get_merged_tracks(tpc_ctx* ctx, tpc_frame_t frame, tpc_merged_tracks* out) {
  if (!ctx || !out) return TPC_E_INVAL;
  if (!ctx->p.merge) return fail(ctx, TPC_E_STATE, "merging is off (tpc_params.merge = 0)");
  tpc_tracks t;
  int rc = tpc_get_tracks(ctx, frame, &t);
  if (rc) return rc;
  Frame* f = find_frame(ctx, frame);
  if (!f->fetch_merge) return fail(ctx, TPC_E_STATE, "frame was tracked without merging");
  static const int64_t zero_offset = 0;
  out->n_merged = f->n_merged;
  out->sector = f->m_sector;
  out->n_seg = f->m_nseg;
  out->head = f->m_head;
  out->x_ref = f->m_xref;
  out->param = f->m_param;
  out->cov = f->m_cov;
  out->chi2 = f->m_chi2;
  out->ndf = f->m_ndf;
  out->n_fit = f->m_nfit;
  out->hit_offset = f->m_hoff ? f->m_hoff : &zero_offset;
  out->hit_index = f->m_hits;
  out->n_tracks = f->n_tracks;
  out->track_next = f->tr_next;
  out->track_merge_chi2 = f->tr_mchi2;
  return TPC_OK;
}

int tpc_get_counts(tpc_ctx* ctx, tpc_frame_t frame, int64_t* n_start, int64_t* n_tracks) {
  if (!ctx) return TPC_E_INVAL;
  Frame* f = find_frame(ctx, frame);
  if (!f || !f->ws) return fail(ctx, TPC_E_STATE, "frame has no tracking results");
  int rc = wait_ws(ctx, *f->ws, 120.0);
  if (rc) return rc;
  const DevCounters& c = *f->ws->h_cnt;
  if (n_start) *n_start = (int64_t)(c.frame_start0[f->fidx + 1] - c.frame_start0[f->fidx]);
  if (n_tracks) *n_tracks = (int64_t)(c.frame_track0[f->fidx + 1] - c.frame_track0[f->fidx]);
  return TPC_OK;
}

int tpc_get_stats(tpc_ctx* ctx, tpc_frame_t frame, int64_t* out, int32_t n) {
  if (!ctx || !out || n < 0) return TPC_E_INVAL;
  Frame* f = find_frame(ctx, frame);
  if (!f || !f->ws) return fail(ctx, TPC_E_STATE, "frame has no tracking results");
  int rc = wait_ws(ctx, *f->ws, 120.0);
  if (rc) return rc;
  const DevCounters& c = *f->ws->h_cnt;
  const int64_t v[] = {(int64_t)c.ntot, (int64_t)c.n_sorted, (int64_t)c.n_bins, (int64_t)c.n_starts,
                       (int64_t)c.n_tracklets, (int64_t)c.n_steps, (int64_t)c.n_tracklet_hits, (int64_t)c.n_tracks,
                       (int64_t)c.n_track_hits, (int64_t)c.err};
  const int nv = (int)(sizeof(v) / sizeof(v[0]));
  for (int k = 0; k < n && k < nv; ++k) out[k] = v[k];
  return nv;
}

int tpc_get_keep_mask(tpc_ctx* ctx, tpc_frame_t frame, uint8_t* host_out, int64_t n) {
  if (!ctx || !host_out) return TPC_E_INVAL;
  Frame* f = find_frame(ctx, frame);
  if (!f || !f->ws) return fail(ctx, TPC_E_STATE, "frame has no tracking results");
  if (!f->ws->W.keep) return fail(ctx, TPC_E_STATE, "the context does not compute compression inputs");
  if (n != f->n) return fail(ctx, TPC_E_INVAL, "length mismatch");
  int rc = wait_ws(ctx, *f->ws, 120.0);
  if (rc) return rc;
  if (n) {
    const long long off = f->ws->h_desc->f[f->fidx].off;
    CK(cudaMemcpyAsync(host_out, f->ws->W.keep + off, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return TPC_OK;
}

int tpc_get_links(tpc_ctx* ctx, tpc_frame_t frame, int32_t what, int32_t* host_out, int64_t n) {
  if (!ctx || !host_out || what < 0 || what > 3) return TPC_E_INVAL;
  Frame* f = find_frame(ctx, frame);
  if (!f || !f->ws) return fail(ctx, TPC_E_STATE, "frame has no tracking results");
  if (n != f->n) return fail(ctx, TPC_E_INVAL, "length mismatch");
  int rc = wait_ws(ctx, *f->ws, 120.0);
  if (rc) return rc;
  int32_t* d = nullptr;
  CK(cudaMallocAsync((void**)&d, 4 * (size_t)std::max<int64_t>(n, 1), ctx->stream));
  CK(cudaMemsetAsync(d, 0xFF, 4 * (size_t)std::max<int64_t>(n, 1), ctx->stream));
  k_links_to_input<<<ctx->sms * 2, 256, 0, ctx->stream>>>(f->ws->W, f->fidx, what, d);
  CK(cudaMemcpyAsync(host_out, d, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaFreeAsync(d, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return TPC_OK;
}

int tpc_release_frame(tpc_ctx* ctx, tpc_frame_t frame) {
  if (!ctx) return TPC_E_INVAL;
  Frame* f = find_frame(ctx, frame);
  if (!f) return fail(ctx, TPC_E_INVAL, "unknown frame handle");
  if (f->state == 4) {  // served, results in copy: the copy completes before its block is reused
    int rc = finish_fetches(ctx, true);
    if (rc) return rc;
  }
  if (f->state == 3 && f->ws) {
    int rc = wait_ws(ctx, *f->ws, 120.0);
    if (rc) return rc;
  }
  if (f->state == 1) {
    auto it = std::find(ctx->queue.begin(), ctx->queue.end(), frame);
    if (it != ctx->queue.end()) ctx->queue.erase(it);
  }
  ctx->queued_input_bytes -= std::min(ctx->queued_input_bytes, f->input_bytes);
  f->input_bytes = 0;
  if (f->served && (f->state == 2 || f->state == 3)) return fail(ctx, TPC_E_STATE, "frame is being tracked");
  drop_frame(ctx, f);
  return TPC_OK;
}

// ------------------------------------------------------------------------------ serving
int tpc_submit_frame(tpc_ctx* ctx, const tpc_clusters* clusters, tpc_frame_t* ticket) {
  if (!ctx || !ticket || !clusters) return TPC_E_INVAL;
  if (clusters->n < 0 || clusters->n >= (1LL << 31)) return fail(ctx, TPC_E_INVAL, "bad cluster descriptor");
  if (clusters->n > 0 && (!clusters->sector || !clusters->row || !clusters->y || !clusters->w))
    return fail(ctx, TPC_E_INVAL, "null cluster array");
  if (clusters->on_device < 0 || clusters->on_device > 2) return fail(ctx, TPC_E_INVAL, "bad on_device value");
  if (clusters->n > ctx->slot_clusters) return fail(ctx, TPC_E_BUDGET, "frame larger than a serving slot of the HBM budget");
  auto fr = std::make_unique<Frame>();
  Frame* f = fr.get();
  f->n = clusters->n;
  f->served = true;
  const size_t in_bytes = (size_t)f->n * 10;
  if (clusters->on_device == 1) {
    f->d_sector = (uint8_t*)clusters->sector; f->d_row = (uint8_t*)clusters->row;
    f->d_y = (float*)clusters->y; f->d_w = (float*)clusters->w;
  } else if (clusters->on_device == 2) {
    // borrowed host memory: read by an asynchronous copy on the slot's stream at admission, so
    // neither a host copy nor device memory is held while the frame waits
    f->borrowed[0] = clusters->sector; f->borrowed[1] = clusters->row;
    f->borrowed[2] = clusters->y; f->borrowed[3] = clusters->w;
    f->is_borrowed = true;
  } else if (ctx->queued_input_bytes + in_bytes <= (size_t)(ctx->p.hbm_budget / 8)) {
    // uploaded now (inputs of waiting frames may use an eighth of the budget); the copy ends
    // before return, so the caller's buffers are free again
    Frame* tmp = nullptr;
    int rc = load_frame(ctx, clusters, tmp);
    if (rc) return rc;
    CK(cudaEventRecord(ctx->ev_sync, ctx->stream));
    rc = wait_event(ctx, ctx->ev_sync, 120.0);
    if (rc) return rc;
    tmp->served = true;
    tmp->input_bytes = in_bytes;
    ctx->queued_input_bytes += in_bytes;
    tmp->state = 1;
    tmp->t_submit = now_s();
    ctx->queue.push_back(tmp->id);
    *ticket = tmp->id;
    return TPC_OK;
  } else {
    // kept on the host until admission: this frame holds no device memory while it waits
    const size_t n = (size_t)f->n;
    f->host_copy.resize(10 * n + 1);
    char* h = f->host_copy.data();
    memcpy(h, clusters->sector, n);
    memcpy(h + n, clusters->row, n);
    memcpy(h + 2 * n, clusters->y, 4 * n);
    memcpy(h + 6 * n, clusters->w, 4 * n);
  }
  f->id = ctx->next_id++;
  f->state = 1;
  f->t_submit = now_s();
  ctx->queue.push_back(f->id);
  *ticket = f->id;
  ctx->frames[f->id] = std::move(fr);
  return TPC_OK;
}

namespace {
// upload a queued host frame on the slot's stream
int upload_frame(tpc_ctx* ctx, Frame* f, cudaStream_t s) {
  if ((f->host_copy.empty() && !f->is_borrowed) || f->d_block) return TPC_OK;
  const size_t n = (size_t)f->n;
  const size_t o1 = align_up(n, 256), o2 = o1 + align_up(n, 256), o3 = o2 + align_up(4 * n, 256);
  const size_t bytes = o3 + align_up(4 * n, 256) + 256;
  cudaError_t e = cudaMallocFromPoolAsync(&f->d_block, bytes, ctx->pool, s);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(ctx, TPC_E_NOMEM, "input allocation failed"); }
  char* b = (char*)f->d_block;
  f->d_sector = (uint8_t*)b; f->d_row = (uint8_t*)(b + o1); f->d_y = (float*)(b + o2); f->d_w = (float*)(b + o3);
  if (n && f->is_borrowed) {
    CK(cudaMemcpyAsync(f->d_sector, f->borrowed[0], n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f->d_row, f->borrowed[1], n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f->d_y, f->borrowed[2], 4 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f->d_w, f->borrowed[3], 4 * n, cudaMemcpyHostToDevice, s));
  } else if (n) {
    const char* h = f->host_copy.data();
    CK(cudaMemcpyAsync(f->d_sector, h, n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f->d_row, h + n, n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f->d_y, h + 2 * n, 4 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(f->d_w, h + 6 * n, 4 * n, cudaMemcpyHostToDevice, s));
  }
  return TPC_OK;
}

// The input and the workspace reference of a retired frame (its results are fetched or in copy).
void retire_inputs(tpc_ctx* ctx, Frame* f, cudaStream_t s) {
  release_ws_user(ctx, f);
  if (f->d_block) { cudaFreeAsync(f->d_block, s); f->d_block = nullptr; }
  ctx->queued_input_bytes -= std::min(ctx->queued_input_bytes, f->input_bytes);
  f->input_bytes = 0;
  f->host_copy.clear();
  f->host_copy.shrink_to_fit();
}

int serve_step(tpc_ctx* ctx) {
  // retire finished batches: the results' copies are queued on the slot's stream (its next batch
  // runs behind them), inputs and workspace references are freed
  for (auto& sl : ctx->slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.ws->done);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("device: ") + cudaGetErrorString(e));
    sl.ws->busy = false;
    const DevCounters& c = *sl.ws->h_cnt;
    const bool overflow = c.n_starts > (uint32_t)sl.ws->tcap || (c.err & (kErrBins | kErrTracks));
    if (!overflow) {
      int rc = check_ws_errors(ctx, *sl.ws);
      if (rc) return rc;
      tpc_ctx::Fetching fe;
      for (auto id : sl.frames) {
        Frame* f = find_frame(ctx, id);
        if (!f) continue;
        rc = fetch_enqueue(ctx, f, sl.stream);
        if (rc) return rc;
        retire_inputs(ctx, f, sl.stream);
        f->state = 4;
        fe.frames.push_back(id);
      }
      if (ctx->spare_events.empty()) {
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ctx->spare_events.push_back(ev);
      }
      fe.ev = ctx->spare_events.back();
      ctx->spare_events.pop_back();
      CK(cudaEventRecord(fe.ev, sl.stream));
      ctx->fetching.push_back(std::move(fe));
    } else {
      // capacity overflow of the batch: track each frame alone (its own workspace) and fetch
      for (auto id : sl.frames) {
        Frame* f = find_frame(ctx, id);
        if (!f) continue;
        release_ws_user(ctx, f);
        const float old = ctx->p.tracklet_capacity;
        ctx->p.tracklet_capacity = std::max(old, 1.25f * (float)c.n_starts / (float)std::max(1LL, f->n));
        std::vector<Frame*> one{f};
        std::shared_ptr<Workspace> ws;
        int rc = run_batch(ctx, one, ctx->stream, ws);
        ctx->p.tracklet_capacity = old;
        if (!rc) rc = wait_ws(ctx, *f->ws, 120.0);
        if (!rc) rc = check_ws_errors(ctx, *f->ws);
        if (!rc) rc = fetch_results(ctx, f);
        if (rc) return rc;
        retire_inputs(ctx, f, sl.stream);
        f->state = 5;
        f->t_done = now_s();
        ctx->finished.push_back(id);
      }
    }
    sl.frames.clear();
    sl.busy = false;
  }
  // launch: every free slot takes queued frames in arrival order. A batch grows only while it stays
  // small: a frame of a few million clusters fills the GPU alone, and putting two of them in one
  // batch would serialise work that two slots run side by side (and delay the first one's result).
  for (auto& sl : ctx->slots) {
    if (sl.busy || ctx->queue.empty()) continue;
    std::vector<Frame*> batch;
    long long n = 0;
    while (!ctx->queue.empty() && (int)batch.size() < ctx->p.max_batch_frames) {
      Frame* f = find_frame(ctx, ctx->queue.front());
      if (!f) { ctx->queue.pop_front(); continue; }
      if (n + f->n > ctx->slot_clusters) break;
      if (!batch.empty() && n + f->n > kServeBatchClusters) break;
      n += f->n;
      batch.push_back(f);
      ctx->queue.pop_front();
    }
    if (batch.empty()) break;
    if (sl.ws && sl.ws->dp.occ != ctx->shape.occ) {  // retuned grid occupancy
      CK(cudaStreamSynchronize(sl.stream));            // result copies from the old workspace done
      sl.ws.reset();
    }
    if (!sl.ws) {
      const long long tcap = (long long)std::ceil((double)ctx->slot_clusters * ctx->p.tracklet_capacity) + 1024;
      int rc = alloc_workspace(ctx, ctx->slot_clusters, tcap, ctx->p.max_batch_frames, sl.ws);
      if (rc) return rc;
    }
    CK(cudaEventRecord(ctx->ev_sync, ctx->stream));  // uploads made at submit time
    CK(cudaStreamWaitEvent(sl.stream, ctx->ev_sync, 0));
    for (Frame* f : batch) {
      int rc = upload_frame(ctx, f, sl.stream);
      if (rc) return rc;
      f->state = 2;
    }
    const bool large = n > kServeSerialClusters;
    if (large && ctx->large_launched) CK(cudaStreamWaitEvent(sl.stream, ctx->ev_track, 0));
    std::shared_ptr<Workspace> ws;
    int rc = run_batch(ctx, batch, sl.stream, ws, sl.ws);
    if (rc) return rc;
    if (large) {
      CK(cudaEventRecord(ctx->ev_track, sl.stream));
      ctx->large_launched = true;
    }
    sl.frames.clear();
    for (Frame* f : batch) sl.frames.push_back(f->id);
    sl.busy = true;
  }
  // last, so that a free slot was relaunched before the host splits fetched results
  return finish_fetches(ctx, false);
}
}  // namespace

int tpc_poll(tpc_ctx* ctx, tpc_frame_t* done, int32_t max_done, int32_t timeout_us) {
  if (!ctx || (max_done > 0 && !done) || max_done < 0) return TPC_E_INVAL;
  const double t0 = now_s();
  for (;;) {
    int rc = serve_step(ctx);
    if (rc) return rc;
    bool busy = !ctx->fetching.empty();
    for (auto& sl : ctx->slots) busy |= sl.busy;
    if (!ctx->finished.empty() || (!busy && ctx->queue.empty())) break;
    if ((now_s() - t0) * 1e6 >= timeout_us) break;
    std::this_thread::yield();
  }
  int k = 0;
  while (k < max_done && !ctx->finished.empty()) {
    done[k++] = ctx->finished.front();
    ctx->finished.pop_front();
  }
  return k;
}

int tpc_autotune(tpc_ctx* ctx, const tpc_frame_t* frames, int32_t n_frames, int32_t reps, tpc_tune_report* out) {
  if (!ctx || !frames || n_frames < 1 || n_frames > kMaxFrames || reps < 1) return fail(ctx, TPC_E_INVAL, "bad tuning request");
  std::vector<Frame*> fr;
  for (int k = 0; k < n_frames; ++k) {
    Frame* f = find_frame(ctx, frames[k]);
    if (!f) return fail(ctx, TPC_E_INVAL, "unknown frame handle");
    if (f->state == 1 || f->state == 2 || f->served) return fail(ctx, TPC_E_STATE, "frame is queued for serving");
    for (Frame* g : fr)
      if (g == f) return fail(ctx, TPC_E_INVAL, "frame listed twice");
    fr.push_back(f);
  }
  ctx->tune_entries.clear();
  const bool old_timing = ctx->timing;
  const Shape start = ctx->shape;
  ctx->timing = true;  // eager launches with events between stages on the context's stream
  const int i_nb = 8, i_ch = 13, i_tl = 14, i_vo = 16, i_ke = 17, i_wt = 19;  // stage indices
  // time one shape: median over reps runs (after one discarded run) of the stage group and total
  auto measure = [&](const Shape& sh, int stage, float& obj) -> int {
    for (const auto& e : ctx->tune_entries) {
      Shape o;
      o.occ = e.bin_occupancy; o.k2_warps = e.k2_warps; o.k2_tma = e.k2_tma; o.k5_block = e.k5_block;
      o.k5_regs = e.k5_regs; o.k5_bps = e.k5_blocks_per_sm; o.k5_order = e.k5_order; o.sel_lanes = e.sel_lanes;
      o.k5_ilp = e.k5_ilp;
      if (o == sh && e.stage == stage) { obj = e.ms; return TPC_OK; }
    }
    ctx->shape = sh;
    std::vector<float> vo, vt;
    for (int r = 0; r <= reps; ++r) {
      std::shared_ptr<Workspace> ws;
      int rc = run_batch(ctx, fr, ctx->stream, ws);
      if (!rc) rc = wait_ws(ctx, *ws, 120.0);
      if (!rc) rc = check_ws_errors(ctx, *ws);
      if (rc) return rc;
      if (r == 0) continue;
      float tot = 0;
      for (int k = 0; k < kNumKernels; ++k) tot += ctx->ms[k];
      vt.push_back(tot);
      vo.push_back(stage == 0   ? tot
                   : stage == 1 ? ctx->ms[i_nb]
                   : stage == 2 ? ctx->ms[i_ch] + ctx->ms[i_tl]
                                : ctx->ms[i_vo] + ctx->ms[i_ke] + ctx->ms[i_wt]);
    }
    std::sort(vo.begin(), vo.end());
    std::sort(vt.begin(), vt.end());
    tpc_tune_entry e{};
    e.bin_occupancy = sh.occ; e.k2_warps = sh.k2_warps; e.k2_tma = sh.k2_tma; e.k5_block = sh.k5_block;
    e.k5_regs = sh.k5_regs; e.k5_blocks_per_sm = sh.k5_bps; e.k5_order = sh.k5_order; e.sel_lanes = sh.sel_lanes;
    e.k5_ilp = sh.k5_ilp;
    e.ms = vo[vo.size() / 2];
    e.total_ms = vt[vt.size() / 2];
    e.stage = stage;
    ctx->tune_entries.push_back(e);
    obj = e.ms;
    return TPC_OK;
  };
  Shape best = start;
  int best_idx = -1;
  // one knob group: time every candidate, keep the fastest on the group's stages
  auto descend = [&](const std::vector<Shape>& cands, int stage) -> int {
    float bo = 0;
    int rc = measure(best, stage, bo);
    if (rc) return rc;
    Shape bs = best;
    for (const Shape& c : cands) {
      float o = 0;
      rc = measure(c, stage, o);
      if (rc) return rc;
      if (o < bo) { bo = o; bs = c; }
    }
    best = bs;
    return TPC_OK;
  };
  int rc = TPC_OK;
  do {
    std::vector<Shape> c;
    for (float occ : kTunerOccupancies) { Shape t = best; t.occ = occ; c.push_back(t); }
    if ((rc = descend(c, 0))) break;
    c.clear();
    for (int w : {4, 8})
      for (int tma : {0, 1, 2}) { Shape t = best; t.k2_warps = w; t.k2_tma = tma; c.push_back(t); }
    if ((rc = descend(c, 1))) break;
    c.clear();
    for (int b : {64, 128, 256})
      for (int r : {64, 72, 80}) { Shape t = best; t.k5_block = b; t.k5_regs = r; t.k5_ilp = 1; t.k5_bps = 0; c.push_back(t); }
    for (int b : {64, 128}) { Shape t = best; t.k5_block = b; t.k5_regs = 128; t.k5_ilp = 2; t.k5_bps = 0; c.push_back(t); }
    if ((rc = descend(c, 2))) break;
    c.clear();
    for (int o : {0, 1, 2, 3}) { Shape t = best; t.k5_order = o; c.push_back(t); }
    if ((rc = descend(c, 2))) break;
    c.clear();
    const int nb = std::max(blocks_per_sm(ctx, 1, best.k5_block, best.k5_regs, best.k5_ilp), 1);
    for (int q : {4, 3, 2, 1}) {  // all resident blocks, then 3/4, 1/2, 1/4 of them
      Shape t = best;
      t.k5_bps = q == 4 ? 0 : std::max(nb * q / 4, 1);
      c.push_back(t);
    }
    if ((rc = descend(c, 2))) break;
    c.clear();
    for (int lanes : {1, 32}) { Shape t = best; t.sel_lanes = lanes; c.push_back(t); }
    if ((rc = descend(c, 3))) break;
  } while (0);
  ctx->timing = old_timing;
  if (rc) {
    ctx->shape = start;
    return rc;
  }
  ctx->shape = best;
  ctx->tuned = true;
  for (size_t k = 0; k < ctx->tune_entries.size(); ++k) {
    const auto& e = ctx->tune_entries[k];
    if (e.bin_occupancy == best.occ && e.k2_warps == best.k2_warps && e.k2_tma == best.k2_tma &&
        e.k5_block == best.k5_block && e.k5_regs == best.k5_regs && e.k5_blocks_per_sm == best.k5_bps &&
        e.k5_order == best.k5_order && e.sel_lanes == best.sel_lanes && e.k5_ilp == best.k5_ilp)
      best_idx = (int)k;
  }
  if (out) {
    out->n_entries = (int32_t)ctx->tune_entries.size();
    out->entries = ctx->tune_entries.data();
    out->best = best_idx;
  }
  return TPC_OK;
}

int tpc_check_wait_timeout(int32_t limit_us, void* cuda_stream) {
  if (limit_us < 1 || limit_us > 1000000) return TPC_E_INVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  uint32_t* d = nullptr;
  if (cudaMalloc((void**)&d, sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return TPC_E_CUDA; }
  uint32_t st = 2;
  cudaError_t e = cudaMemsetAsync(d, 0xFF, sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    launch_wait_probe(d, 1000ull * (unsigned long long)limit_us, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) { cudaGetLastError(); return TPC_E_CUDA; }
  return st == 1u ? TPC_E_TIMEOUT : st == 0u ? TPC_OK : TPC_E_CUDA;
}

int tpc_set_timing(tpc_ctx* ctx, int32_t enable) {
  if (!ctx) return TPC_E_INVAL;
  ctx->timing = enable != 0;
  return TPC_OK;
}

int tpc_get_kernel_times(tpc_ctx* ctx, tpc_kernel_times* out) {
  if (!ctx || !out) return TPC_E_INVAL;
  for (int k = 0; k < kNumKernels; ++k) ctx->launches[k] = ctx->stage_launches[k];
  out->n_kernels = kNumKernels;
  out->names = kKernelNames;
  out->ms = ctx->ms;
  out->launches = ctx->launches;
  return TPC_OK;
}

void tpc_cf_default_params(tpc_cf_params* p) {
  if (!p) return;
  p->pad_pitch = 0.4;
  p->time_bin_w = (250.0 / 90.0) * 0.2;
  p->q_peak_min = 3;
  p->q_total_min = 10;
}

int tpc_find_clusters(tpc_ctx* ctx, const tpc_cf_params* params, const tpc_digits* d, int32_t to_host,
                      tpc_cluster_list* out, void* cuda_stream) {
  if (!ctx) return TPC_E_INVAL;
  if (!d || !out) return fail(ctx, TPC_E_INVAL, "null digits or output");
  tpc_cf_params P;
  if (params) P = *params;
  else tpc_cf_default_params(&P);
  if (!(P.pad_pitch >= 0.01 && P.pad_pitch <= 100.0) || !(P.time_bin_w > 0.0 && P.time_bin_w <= 1e4) ||
      P.q_peak_min < 1 || P.q_total_min < 0)
    return fail(ctx, TPC_E_INVAL, "bad cluster-finder parameters");
  if (d->n < 0 || d->n >= (1LL << 31) || d->n_time < 0 || d->n_time > 65535)
    return fail(ctx, TPC_E_INVAL, "bad digit descriptor");
  if (d->n > 0 && (!d->sector || !d->row || !d->pad || !d->time || !d->adc))
    return fail(ctx, TPC_E_INVAL, "null digit array");
  CfState& cf = ctx->cf;
  memset(out, 0, sizeof(*out));
  out->on_device = to_host ? 0 : 1;
  if (d->n == 0) return TPC_OK;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  uint16_t np[kNRow];
  int npmax = 0;
  for (int r = 0; r < kNRow; ++r) {
    const int v = cf_npads(P.pad_pitch, r);
    np[r] = (uint16_t)v;
    npmax = std::max(npmax, v);
  }
  const int stride = (int)align_up((size_t)npmax + 2 * kCfGuard, 16);
  // the charge map holds the whole frame when it fits half of the budget, else a time window of as
  // many bins as fit (the frame then runs in two passes over its windows)
  int lines = d->n_time + 2 * kCfGuard, tw = d->n_time;
  {
    const size_t line_bytes = (size_t)kSegPerFrame * (size_t)stride * 2;
    const size_t half = (size_t)std::max<int64_t>(ctx->p.hbm_budget, 0) / 2;
    if ((size_t)lines * line_bytes > half) {
      const long long max_lines = (long long)(half / line_bytes);
      if (max_lines < 2 * kCfGuard + 16)
        return fail(ctx, TPC_E_BUDGET, "a charge map of 16 time bins exceeds half of the HBM budget");
      tw = (int)(max_lines - 2 * kCfGuard);
      lines = tw + 2 * kCfGuard;
    }
  }
  const bool windowed = tw < d->n_time;
  int rc = cf_reserve(ctx, d->n);
  if (rc) return rc;
  if (!cf.done) {
    for (auto& e : cf.ev) CK(cudaEventCreate(&e));
    CK(cudaEventCreateWithFlags(&cf.done, cudaEventDisableTiming));
    CK(cudaMallocHost((void**)&cf.h_small, 16));
  }
  rc = cf_map(ctx, lines, stride, s);
  if (rc) return rc;
  const long long n = d->n;
  CK(cudaMemcpyAsync(cf.npads, np, sizeof(np), cudaMemcpyHostToDevice, s));
  CfArgs A{};
  if (d->on_device) {
    A.sector = d->sector; A.row = d->row; A.pad = d->pad; A.time = d->time; A.adc = d->adc;
  } else {
    CK(cudaMemcpyAsync(cf.in_sector, d->sector, n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cf.in_row, d->row, n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cf.in_pad, d->pad, 2 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cf.in_time, d->time, 2 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cf.in_adc, d->adc, 2 * n, cudaMemcpyHostToDevice, s));
    A.sector = cf.in_sector; A.row = cf.in_row; A.pad = cf.in_pad; A.time = cf.in_time; A.adc = cf.in_adc;
  }
  A.n = n;
  A.n_time = d->n_time;
  A.lines = lines;
  A.stride = stride;
  A.t_lo = 0;
  A.t_hi = d->n_time;
  A.wflag = cf.wflag;
  A.q_peak_min = P.q_peak_min;
  A.q_total_min = P.q_total_min;
  A.pitch = (float)P.pad_pitch;
  A.dw = (float)P.time_bin_w;
  A.map = cf.map;
  A.wcount = cf.wcount;
  A.woff = cf.woff;
  A.wsrc = cf.wsrc;
  A.t_sector = cf.t_sector; A.t_row = cf.t_row; A.t_y = cf.t_y; A.t_w = cf.t_w; A.t_qtot = cf.t_qtot;
  A.t_qmax = cf.t_qmax; A.t_sig_pad = cf.t_sp; A.t_sig_time = cf.t_st; A.t_digit = cf.t_digit;
  A.err = cf.small + 1;
  A.o_sector = cf.o_sector; A.o_row = cf.o_row; A.o_y = cf.o_y; A.o_w = cf.o_w; A.o_qtot = cf.o_qtot;
  A.o_qmax = cf.o_qmax; A.o_sig_pad = cf.o_sp; A.o_sig_time = cf.o_st; A.o_digit = cf.o_digit;
  A.npads = cf.npads;
  CK(cudaMemsetAsync(cf.small, 0, 16, s));
  const long long tiles = (n + kCfTile - 1) / kCfTile;
  const int grid = (int)std::min<long long>(tiles, (long long)ctx->sms * (2048 / kCfTile));
  const int G = ctx->sms;
  const bool timing = ctx->timing;
  cf.map_clean = false;
  const long long nwarps = (n + 31) / 32;
  auto scan_counts = [&]() {
    k_scan_reduce<<<2 * G, 256, 0, s>>>(cf.wcount, nullptr, nwarps, 0, cf.scan_tmp);
    k_scan_tiles<<<1, 1024, 0, s>>>(cf.scan_tmp, nullptr, nwarps, 0, cf.small);
    k_scan_apply<<<2 * G, 256, 0, s>>>(cf.wcount, nullptr, nwarps, 0, cf.scan_tmp, cf.small, cf.woff);
  };
  if (!windowed) {
    cf.windows = 1;
    if (timing) cudaEventRecord(cf.ev[0], s);
    k_cf_fill<<<grid, kCfTile, 0, s>>>(A);
    if (timing) cudaEventRecord(cf.ev[1], s);
    k_cf_peaks<<<grid, kCfTile, 0, s>>>(A);
    if (timing) cudaEventRecord(cf.ev[2], s);
    scan_counts();
    if (timing) cudaEventRecord(cf.ev[3], s);
    k_cf_copy<<<(int)std::min<long long>((nwarps + kCfTile - 1) / kCfTile, (long long)G * (2048 / kCfTile)), kCfTile,
                0, s>>>(A);
    if (timing) cudaEventRecord(cf.ev[4], s);
    k_cf_clear<<<grid, kCfTile, 0, s>>>(A);
    if (timing) cudaEventRecord(cf.ev[5], s);
    const int64_t nl[kCfKernels] = {1, 1, 3, 1, 1};
    for (int k = 0; k < kCfKernels; ++k) cf.launches[k] = nl[k];
  } else {
    // the group lists of the windows; pass 1 over the windows: fill, flag the kept peaks, clear;
    // then the scan of their counts; pass 2: fill, write each kept peak's cluster to its slot, clear
    // (stage times: cf_fill holds the lists and pass 1, cf_copy pass 2)
    const int nwin = (d->n_time + tw - 1) / tw;  // <= kCfMaxWindows: tw >= 16, n_time <= 65535
    A.tw = tw;
    A.nwin = nwin;
    A.glist = cf.glist; A.gwide = cf.gwide; A.gwin = cf.gwin; A.gcnt = cf.gcnt; A.gbeg = cf.gbeg; A.gcur = cf.gcur;
    CK(cudaMemsetAsync(cf.wcount, 0, 4 * (size_t)nwarps, s));
    CK(cudaMemsetAsync(cf.wflag, 0, 4 * (size_t)nwarps, s));
    CK(cudaMemsetAsync(cf.gcnt, 0, 4 * (size_t)(kCfMaxWindows + 1), s));
    if (timing) cudaEventRecord(cf.ev[0], s);
    const size_t list_smem = 4 * (size_t)(nwin + 1);
    k_cf_gcount<<<grid, kCfTile, list_smem, s>>>(A);
    k_cf_gscan<<<1, 1024, 0, s>>>(A);
    k_cf_gplace<<<grid, kCfTile, 2 * list_smem, s>>>(A);
    for (int w = 0; w < nwin; ++w) {
      A.win = w;
      A.t_lo = w * tw;
      A.t_hi = std::min(A.t_lo + tw, d->n_time);
      k_cf_wfill<<<grid, kCfTile, 0, s>>>(A);
      k_cf_flag<<<grid, kCfTile, 0, s>>>(A);
      k_cf_wclear<<<grid, kCfTile, 0, s>>>(A);
    }
    if (timing) { cudaEventRecord(cf.ev[1], s); cudaEventRecord(cf.ev[2], s); }
    scan_counts();
    if (timing) cudaEventRecord(cf.ev[3], s);
    for (int w = 0; w < nwin; ++w) {
      A.win = w;
      A.t_lo = w * tw;
      A.t_hi = std::min(A.t_lo + tw, d->n_time);
      k_cf_wfill<<<grid, kCfTile, 0, s>>>(A);
      k_cf_emit<<<grid, kCfTile, 0, s>>>(A);
      k_cf_wclear<<<grid, kCfTile, 0, s>>>(A);
    }
    if (timing) { cudaEventRecord(cf.ev[4], s); cudaEventRecord(cf.ev[5], s); }
    cf.windows = nwin;
    const int64_t nl[kCfKernels] = {3 * nwin, 0, 6, 3 * nwin, 0};  // cf_scan: the count scan and the three list kernels
    for (int k = 0; k < kCfKernels; ++k) cf.launches[k] = nl[k];
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("cluster-finder launch: ") + cudaGetErrorString(e));
  CK(cudaMemcpyAsync(cf.h_small, cf.small, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(cf.done, s));
  rc = wait_event(ctx, cf.done, 120.0);
  if (rc) return rc;
  cf.map_clean = true;
  if (timing)
    for (int k = 0; k < kCfKernels; ++k) {
      float m = 0;
      if (cudaEventElapsedTime(&m, cf.ev[k], cf.ev[k + 1]) == cudaSuccess) cf.ms[k] = m;
    }
  const uint32_t total = cf.h_small[0], err = cf.h_small[1];
  // After any refused frame the next call re-zeros the whole map: two digits in one cell may have
  // carried charge into a neighbouring cell (also one the clear kernel does not visit), whatever
  // other error was found beside it.
  if (err) cf.map_clean = false;
  if (err & kCfErrDigit) return fail(ctx, TPC_E_INVAL, "malformed digit (cell outside the pad row or frame, or zero charge)");
  if (err & kCfErrTwice) return fail(ctx, TPC_E_INVAL, "two digits in one cell");
  const long long m = total;
  out->n_clusters = m;
  if (!to_host) {
    out->sector = cf.o_sector; out->row = cf.o_row; out->y = cf.o_y; out->w = cf.o_w; out->q_tot = cf.o_qtot;
    out->q_max = cf.o_qmax; out->sigma_pad = cf.o_sp; out->sigma_time = cf.o_st; out->digit = cf.o_digit;
    return TPC_OK;
  }
  const size_t need = (size_t)std::max<long long>(m, 1) * 28 + 64;
  if (cf.host_bytes < need) {
    if (cf.host) cudaFreeHost(cf.host);
    cf.host = nullptr;
    cf.host_bytes = 0;
    if (cudaMallocHost(&cf.host, need + need / 4) != cudaSuccess) {
      cudaGetLastError();
      cf.host = nullptr;
      return fail(ctx, TPC_E_NOMEM, "page-locked cluster copies");
    }
    cf.host_bytes = need + need / 4;
  }
  char* h = static_cast<char*>(cf.host);
  size_t o = 0;
  auto put = [&](const void* src, size_t bytes) -> void* {
    void* dst = h + o;
    if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    o = align_up(o + bytes, 4);
    return dst;
  };
  out->y = (const float*)put(cf.o_y, 4 * m);
  out->w = (const float*)put(cf.o_w, 4 * m);
  out->sigma_pad = (const float*)put(cf.o_sp, 4 * m);
  out->sigma_time = (const float*)put(cf.o_st, 4 * m);
  out->q_tot = (const uint32_t*)put(cf.o_qtot, 4 * m);
  out->digit = (const uint32_t*)put(cf.o_digit, 4 * m);
  out->q_max = (const uint16_t*)put(cf.o_qmax, 2 * m);
  out->sector = (const uint8_t*)put(cf.o_sector, m);
  out->row = (const uint8_t*)put(cf.o_row, m);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, TPC_E_CUDA, std::string("cluster copies: ") + cudaGetErrorString(e));
  CK(cudaEventRecord(cf.done, s));
  return wait_event(ctx, cf.done, 120.0);
}

int tpc_get_cf_kernel_times(tpc_ctx* ctx, tpc_kernel_times* out) {
  static const char* names[kCfKernels] = {"cf_fill", "cf_peaks", "cf_scan", "cf_copy", "cf_clear"};
  if (!ctx || !out) return TPC_E_INVAL;
  out->n_kernels = kCfKernels;
  out->names = names;
  out->ms = ctx->cf.ms;
  out->launches = ctx->cf.launches;
  return TPC_OK;
}

}  // extern "C"
