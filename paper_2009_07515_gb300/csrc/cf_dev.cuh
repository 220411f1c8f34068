// cf_dev.cuh — device-side definitions of the cluster finder (k_cf.cu, sm_103a).
#pragma once
#include "tpc_dev.cuh"

namespace tpc {

// Arguments of the cluster-finder kernels (k_cf.cu). The charge map holds one plane per
// (sector, row): lines = (t_hi - t_lo) + 4 time lines of `stride` u16 cells, cell (k, j) at
// (j - t_lo + 2) * stride + (k + 2); the two guard lines and guard pads on each side hold no digit
// of the window's peaks, so every 5x5 window read stays inside the plane and sees 0 outside the
// row. A frame whose map does not fit the budget is processed in time windows.
constexpr int kCfTile = 256;          // digits per block iteration (8 warps)
constexpr int kCfGuard = 2;
constexpr uint32_t kCfErrDigit = 1u;  // a digit outside the pad row / frame, or with zero charge
constexpr uint32_t kCfErrTwice = 2u;  // two digits in one cell
constexpr int kCfMaxWindows = 4096;   // a window holds at least 16 of at most 65536 time bins
struct CfArgs {
  const uint8_t* sector;
  const uint8_t* row;
  const uint16_t* pad;
  const uint16_t* time;
  const uint16_t* adc;
  long long n;
  int n_time, lines, stride;
  // time window of this pass (the whole frame when the map holds it): peaks of digits with time in
  // [t_lo, t_hi) are evaluated; digits with time in [t_lo - 2, t_hi + 2) are filled and cleared;
  // map line = time - t_lo + 2
  int t_lo, t_hi;
  uint32_t* wflag;    // [ceil(n / 32)] windowed mode: bit l set when digit 32 g + l is a kept peak
  int q_peak_min, q_total_min;
  float pitch, dw;
  uint16_t* map;
  uint32_t* wcount;   // [ceil(n / 32)] kept clusters per 32 digits (one warp's digits)
  uint32_t* woff;     // [ceil(n / 32) + 1] exclusive scan of wcount: their first output slot
  uint32_t* wsrc;     // [ceil(n / 32)] first temporary slot of their clusters
  uint32_t* err;
  // the kept clusters of each 32 digits, in digit order from slot wsrc on (each block of the peak
  // kernel fills its own region of the temporary arrays)
  uint8_t* t_sector;
  uint8_t* t_row;
  float* t_y;
  float* t_w;
  uint32_t* t_qtot;
  uint16_t* t_qmax;
  float* t_sig_pad;
  float* t_sig_time;
  uint32_t* t_digit;
  // clusters, in the input order of their peak digits
  uint8_t* o_sector;
  uint8_t* o_row;
  float* o_y;
  float* o_w;
  uint32_t* o_qtot;
  uint16_t* o_qmax;
  float* o_sig_pad;
  float* o_sig_time;
  uint32_t* o_digit;
  const uint16_t* npads;  // [kNRow] pads of each row
  // windowed mode: the groups of 32 digits (digits 32 g .. 32 g + 31) a window's passes visit
  int win, tw, nwin;      // this pass's window, bins per window, windows
  uint32_t* glist;        // [2 * groups] by window: the groups whose valid digits reach one or two
                          // windows' maps (window + 2 halo bins on each side)
  uint32_t* gwide;        // [groups] the groups that reach more windows (visited in every window)
  uint32_t* gwin;         // [groups] each group's first and last window
  uint32_t* gcnt;         // [kCfMaxWindows + 1] groups listed per window; [kCfMaxWindows]: wide groups
  uint32_t* gbeg;         // [kCfMaxWindows + 1] first entry of each window's list (exclusive scan)
  uint32_t* gcur;         // [kCfMaxWindows + 1] placement cursors; [kCfMaxWindows]: the wide list's
};

}  // namespace tpc
