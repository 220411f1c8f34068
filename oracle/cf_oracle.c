/*
 * cf_oracle.c — plain, slow CPU reference cluster finder.
 *
 * TEST INFRASTRUCTURE ONLY, under the same rules as tpc_oracle.c: only the tests, the package smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product path shares no code with it.
 *
 * What it computes: the cluster finding of the synchronous reconstruction (Table 1 of Sec. 7.2 times
 * it as the first GPU step; Sec. 2: the TPC records, per pad, the charge of each time bin, and the
 * clusters of a pad row are reconstructed from these digits). The paper names the step but not its
 * rules, so this file states the reading the project takes:
 *
 *   Input: digits (sector s, row r, pad k, time bin j, charge q >= 1), at most one per cell, with
 *   k < n_pads(r) = 2 ceil(x_r tan(10 deg) / pad_pitch), j < n_time. Any other input is rejected.
 *   q(s, r, k, j) is the charge of the digit at that cell, 0 where there is none (also outside the row).
 *
 *   1. Peak: a digit c with q_c >= q_peak_min that wins against each of its 8 neighbours n in the
 *      3x3 window: q_n < q_c, or q_n = q_c and n comes later in (time, pad) order (dj > 0, or dj = 0
 *      and dk > 0). A plateau of equal charges thus has a single peak, its first cell.
 *   2. Cluster of a peak: the charges of the 3x3 window, and of each cell of the 5x5 ring around it
 *      whose charge does not exceed that of the window cell next to it on the way to the peak
 *      (step the +-2 coordinates one cell inwards), so that a rising charge, which belongs to a
 *      neighbouring cluster, is left out. Integer sums Q = sum q, Sk = sum q dk, Sj = sum q dj,
 *      Skk = sum q dk^2, Sjj = sum q dj^2 over the included cells (dk, dj relative to the peak).
 *   3. The cluster is kept if Q >= q_total_min. Its position and widths, in REAL arithmetic:
 *        mk = Sk / Q, mj = Sj / Q; pad = k + mk; time = j + mj;
 *        y = (pad - (n_pads/2 - 1/2)) * pad_pitch;  w = (time + 1/2) * time_bin_w;
 *        sigma_pad = sqrt(max(0, Skk / Q - mk * mk)), sigma_time likewise (in pads and time bins).
 *   Output: the kept clusters in the input order of their peak digits.
 *
 * Precision: REAL = double or float (compiled with -DORACLE_F32), -ffp-contract=off, no fast-math;
 * every REAL value is a fixed sequence of correctly rounded +, -, *, / and sqrt.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(ORACLE_F32) && defined(ORACLE_PLAIN)
/* the plain-FP32 build of the tracker oracle links this file too; the cluster finder has no fused
 * multiply-add or reciprocal to undo, so it is the FP32 cluster finder under that build's prefix */
typedef float real;
#define CF_SQRT sqrtf
#define CF_SYM(name) oracle_f32plain_##name
#elif defined(ORACLE_F32)
typedef float real;
#define CF_SQRT sqrtf
#define CF_SYM(name) oracle_f32_##name
#else
typedef double real;
#define CF_SQRT sqrt
#define CF_SYM(name) oracle_f64_##name
#endif

#define CF_NSEC 36
#define CF_NROW 152

typedef struct {
  double pad_pitch;     /* cm */
  double time_bin_w;    /* cm of drift coordinate per time bin */
  int32_t q_peak_min;
  int32_t q_total_min;
} oracle_cf_params;

typedef struct {
  int64_t n_clusters;
  int32_t* sector;
  int32_t* row;
  int32_t* pad;         /* peak cell */
  int32_t* time;
  int64_t* digit;       /* input index of the peak digit */
  int64_t* q_tot;
  int32_t* q_max;
  double* y;
  double* w;
  double* sigma_pad;
  double* sigma_time;
} oracle_cf_result;

void CF_SYM(cf_default_params)(oracle_cf_params* p) {
  p->pad_pitch = 0.4;
  p->time_bin_w = (250.0 / 90.0) * 0.2;
  p->q_peak_min = 3;
  p->q_total_min = 10;
}

int CF_SYM(n_pads)(double pitch, int r) {
  const double x = 85.0 + (double)r * (160.0 / 151.0);
  return 2 * (int)ceil(x * tan(10.0 * 3.14159265358979323846 / 180.0) / pitch);
}

typedef struct { uint64_t key; int32_t q; } cell_t;

static uint64_t cell_key(int s, int r, int k, int j) {
  return ((uint64_t)(s * CF_NROW + r) << 32) | ((uint64_t)(uint32_t)j << 16) | (uint64_t)(uint32_t)k;
}
static int cmp_cell(const void* a, const void* b) {
  const uint64_t x = ((const cell_t*)a)->key, y = ((const cell_t*)b)->key;
  return x < y ? -1 : x > y;
}

typedef struct {
  const cell_t* cells;
  int64_t n;
  const int* np;
  int n_time;
} map_t;

/* charge at a cell: binary search in the sorted cell list, 0 where there is no digit */
static int32_t charge(const map_t* m, int s, int r, int k, int j) {
  if (k < 0 || k >= m->np[r] || j < 0 || j >= m->n_time) return 0;
  const uint64_t key = cell_key(s, r, k, j);
  int64_t lo = 0, hi = m->n;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (m->cells[mid].key < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < m->n && m->cells[lo].key == key) ? m->cells[lo].q : 0;
}

static int sgn(int v) { return (v > 0) - (v < 0); }

void CF_SYM(free_cf_result)(oracle_cf_result* R) {
  if (!R) return;
  free(R->sector); free(R->row); free(R->pad); free(R->time); free(R->digit); free(R->q_tot);
  free(R->q_max); free(R->y); free(R->w); free(R->sigma_pad); free(R->sigma_time);
  free(R);
}

int CF_SYM(find_clusters)(const oracle_cf_params* p, int64_t n, const uint8_t* sector, const uint8_t* row,
                          const uint16_t* pad, const uint16_t* time, const uint16_t* adc, int32_t n_time,
                          int n_threads, oracle_cf_result** out) {
  if (!p || !out || n < 0 || n_time < 0 || p->pad_pitch <= 0 || p->time_bin_w <= 0) return -1;
  *out = NULL;
  int np[CF_NROW];
  for (int r = 0; r < CF_NROW; ++r) np[r] = CF_SYM(n_pads)(p->pad_pitch, r);
  for (int64_t i = 0; i < n; ++i)
    if (sector[i] >= CF_NSEC || row[i] >= CF_NROW || pad[i] >= np[row[i]] || time[i] >= n_time || adc[i] == 0)
      return -1;
  cell_t* cells = (cell_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(cell_t));
  uint8_t* keep = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int64_t (*sums)[5] = malloc((size_t)(n > 0 ? n : 1) * sizeof(*sums));
  if (!cells || !keep || !sums) { free(cells); free(keep); free(sums); return -2; }
  for (int64_t i = 0; i < n; ++i) {
    cells[i].key = cell_key(sector[i], row[i], pad[i], time[i]);
    cells[i].q = adc[i];
  }
  qsort(cells, (size_t)n, sizeof(cell_t), cmp_cell);
  for (int64_t i = 1; i < n; ++i)
    if (cells[i].key == cells[i - 1].key) { free(cells); free(keep); free(sums); return -1; }
  const map_t m = {cells, n, np, n_time};
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static, 4096)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const int s = sector[i], r = row[i], k = pad[i], j = time[i];
    const int32_t qc = adc[i];
    int peak = qc >= p->q_peak_min;
    for (int dj = -1; dj <= 1 && peak; ++dj)
      for (int dk = -1; dk <= 1 && peak; ++dk) {
        if (dk == 0 && dj == 0) continue;
        const int32_t qn = charge(&m, s, r, k + dk, j + dj);
        const int later = dj > 0 || (dj == 0 && dk > 0);
        if (!(qn < qc || (qn == qc && later))) peak = 0;
      }
    if (!peak) continue;
    int64_t Q = 0, Sk = 0, Sj = 0, Skk = 0, Sjj = 0;
    for (int dj = -2; dj <= 2; ++dj)
      for (int dk = -2; dk <= 2; ++dk) {
        const int32_t q = charge(&m, s, r, k + dk, j + dj);
        if (abs(dk) == 2 || abs(dj) == 2) {
          const int ik = dk - (abs(dk) == 2 ? sgn(dk) : 0), ij = dj - (abs(dj) == 2 ? sgn(dj) : 0);
          if (q > charge(&m, s, r, k + ik, j + ij)) continue;
        }
        Q += q; Sk += (int64_t)q * dk; Sj += (int64_t)q * dj;
        Skk += (int64_t)q * dk * dk; Sjj += (int64_t)q * dj * dj;
      }
    if (Q < p->q_total_min) continue;
    keep[i] = 1;
    sums[i][0] = Q; sums[i][1] = Sk; sums[i][2] = Sj; sums[i][3] = Skk; sums[i][4] = Sjj;
  }
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) nc += keep[i];
  oracle_cf_result* R = (oracle_cf_result*)calloc(1, sizeof(oracle_cf_result));
  const size_t na = (size_t)(nc > 0 ? nc : 1);
  if (R) {
    R->sector = malloc(na * 4); R->row = malloc(na * 4); R->pad = malloc(na * 4); R->time = malloc(na * 4);
    R->digit = malloc(na * 8); R->q_tot = malloc(na * 8); R->q_max = malloc(na * 4);
    R->y = malloc(na * 8); R->w = malloc(na * 8); R->sigma_pad = malloc(na * 8); R->sigma_time = malloc(na * 8);
  }
  if (!R || !R->sector || !R->row || !R->pad || !R->time || !R->digit || !R->q_tot || !R->q_max || !R->y ||
      !R->w || !R->sigma_pad || !R->sigma_time) {
    CF_SYM(free_cf_result)(R); free(cells); free(keep); free(sums);
    return -2;
  }
  const real pitch = (real)p->pad_pitch, dw = (real)p->time_bin_w, half = (real)0.5;
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!keep[i]) continue;
    const int r = row[i];
    const real Q = (real)sums[i][0];
    const real mk = (real)sums[i][1] / Q, mj = (real)sums[i][2] / Q;
    const real pc = (real)pad[i] + mk, tc = (real)time[i] + mj;
    const real centre = (real)(np[r] / 2) - half;
    const real y = (pc - centre) * pitch;
    const real w = (tc + half) * dw;
    const real ak = (real)sums[i][3] / Q, aj = (real)sums[i][4] / Q;
    const real bk = mk * mk, bj = mj * mj;
    const real vk = ak - bk, vj = aj - bj;
    R->sector[o] = sector[i]; R->row[o] = r; R->pad[o] = pad[i]; R->time[o] = time[i];
    R->digit[o] = i; R->q_tot[o] = sums[i][0]; R->q_max[o] = adc[i];
    R->y[o] = (double)y; R->w[o] = (double)w;
    R->sigma_pad[o] = (double)(vk > 0 ? CF_SQRT(vk) : (real)0);
    R->sigma_time[o] = (double)(vj > 0 ? CF_SQRT(vj) : (real)0);
    ++o;
  }
  R->n_clusters = nc;
  free(cells); free(keep); free(sums);
  *out = R;
  return 0;
}
