/*
 * tpc_oracle.c — plain, slow CPU reference tracker for TPC sector tracking.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark may load this. The product path never calls it and shares no code with it.
 *
 * What it computes: the standalone TPC sector tracking of the paper's synchronous reconstruction
 * (Sec. 6: the TPC tracking runs first standalone, without space-charge, field or hit-error
 * corrections, on clusters whose z is unknown in continuous readout, Sec. 2; the algorithm is
 * derived from the Run-2 HLT tracker). The paper names the method but defers its steps to the HLT
 * papers it cites, so each step below states the reading this project takes:
 *
 *   1. per-(sector, row) search index (here: the row's hits sorted by drift coordinate w);
 *   2. cellular-automaton neighbour finding: for each hit, the best (down, up) pair in rows r-1/r+1
 *      by the mid-point deviation chi_n inside slope windows;
 *   3. neighbour cleaning: keep only reciprocal links;
 *   4. start hits: heads of cleaned chains (up link, no down link) of at least lmin hits;
 *   5. tracklet construction: 3-point circle seed, Kalman filter (exact helix propagation in the
 *      solenoid field, multiple-scattering noise, Joseph-form update) along the chain, outward
 *      extension by row-by-row search (ending, with ext_stop, right after it accepts the start hit
 *      of another tracklet, which covers the rows beyond), then an inward refit (covariance reset)
 *      through the found hits and inward extension;
 *   6. tracklet selection: each hit goes to the tracklet with the largest (nhits, -start index) key;
 *      a tracklet becomes a track if it keeps >= nmin hits and at least half of its hits;
 *   7. beam line (Sec. 6: track seeds are extrapolated to the beam line, and the most likely z is
 *      computed assuming a primary from a vertex at the origin): each track's fit is transported
 *      by the same exact helix step, without scattering, from x_ref to the plane x = 0 through the
 *      beam axis; there y0 and the drift coordinate w0 (with its variance) are read. A primary from
 *      z = 0 has w0 = v_d t_c + L (continuous readout, Sec. 2: w = v_d t_c + L - |z|), so its
 *      collision time is t0 = (w0 - L) / v_d and its z at x_ref is +-(w0 - w_ref) by drift side;
 *   8. compression inputs (Sec. 4: hits of good tracks are stored as residuals to the extrapolated
 *      track position; strategy B removes every hit not in the vicinity of a good track): each
 *      track's fit is transported (state only, no scattering) from x_ref directly to every row up
 *      to its last hit's row, one exact helix step per row (rows independent; once a transport
 *      fails, |sin phi| only grows further out, so every later one fails too). At every row a
 *      good track (|q/pT| <= keep_qpt_max) protects the row's clusters
 *      within +-(keep_vy, keep_vw) of its predicted (y, w); at a row with one of its hits the hit
 *      is stored as q(hit) - q(prediction), q(v) = rint(512 v) (the 2^-9 cm quantum of the 16-bit
 *      storage). A decoder with the same arithmetic restores q(hit) exactly. If the transport
 *      fails, the remaining hits are stored as q(hit) (n_pred counts the predicted ones).
 *
 * Precision: compiled twice, REAL = double (FP64 oracle) and REAL = float (FP32 oracle), with
 * -ffp-contract=off and no fast-math. Only +, -, *, /, sqrt and fused multiply-add (every sum of
 * products of the Kalman filter accumulates with one fma per term, in index order) are used on REAL
 * values; asin is evaluated by half-angle argument reduction and its Maclaurin series
 * (oracle_asin), so every REAL result is a fixed sequence of correctly rounded operations.
 *
 * Coordinates: sector s in [0,36) (s/18 = drift side, s%18 = phi sector), row r in [0,152) at
 * x_r = 85 + r * 160/151 cm (sector-local, radial), y along the pad row, w = v_d * t_arrival.
 * Track state at x: (y, w, sin(phi), t = dw/ds_xy, q/pT); curvature k = kq * (q/pT),
 * kq = -0.0029979246 * Bz; d(sin phi)/dx = k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(ORACLE_F32) && defined(ORACLE_PLAIN)
/* plain FP32: every sum of products rounds each product and each sum (no fused multiply-add), and
 * every quotient is a true division (no reciprocal formed once and multiplied) */
typedef float real;
#define SQRT sqrtf
#define RINT rintf
#define FMA(a, b, c) ((a) * (b) + (c))
#define ORACLE_SYM(name) oracle_f32plain_##name
#elif defined(ORACLE_F32)
typedef float real;
#define SQRT sqrtf
#define RINT rintf
#define FMA fmaf
#define ORACLE_SYM(name) oracle_f32_##name
#else
typedef double real;
#define SQRT sqrt
#define RINT rint
#define FMA fma
#define ORACLE_SYM(name) oracle_f64_##name
#endif

/* x / v, written with the reciprocal iv = 1 / v formed once (default) or as a true division (plain) */
#ifdef ORACLE_PLAIN
#define QUO(x, v, iv) ((x) / (v))
#else
#define QUO(x, v, iv) ((x) * (iv))
#endif

#define NSEC 36
#define NROW 152

/* ------------------------------------------------------------------------------------------------
 * Parameters (interface in double; converted to REAL once)
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  double bz;          /* T */
  double ky, kw, eps; /* neighbour windows: |dy| <= ky*dx + eps, |dw| <= kw*dx + eps */
  double chi_n_max;   /* cut on the mid-point deviation dy^2 + dw^2 (cm^2) */
  int32_t lmin;       /* minimum chain length for a start hit */
  double sigma_y, sigma_w;
  double chi2_hit_max;
  int32_t n_miss_max; /* consecutive rows without a hit that end an extension */
  double win_nsig, win_add; /* extension search window: nsig*sqrt(C) + add */
  double x0_per_row;  /* X/X0 per row for the scattering noise; 0 = off */
  double max_sin;
  double y_margin;    /* stop when |y| > x*tan(10 deg) + y_margin */
  int32_t nmin;       /* minimum hits of a voting tracklet and of a track */
  double cov0[5];     /* initial diagonal covariance of the seed */
  int32_t ext_stop;   /* 1: an outward extension ends at an accepted start hit of another chain */
  double drift_length;   /* cm, L: w of a cluster at the central membrane minus v_d t_c */
  double drift_velocity; /* cm per microsecond */
  double keep_vy, keep_vw; /* strategy-B vicinity of a good track's prediction (cm) */
  double keep_qpt_max;     /* good track: |q/pT| <= this (c/GeV) */
  int32_t merge_gap_rows;  /* step 9: the outer segment starts 1 .. this many rows above the inner one */
  double merge_dw;         /* step 9: |w difference| of a candidate pair at the outer segment's start (cm) */
  double merge_chi2_max;   /* step 9: 5-parameter chi2 cut of a merge */
  int32_t refit_passes;    /* step 9: refit passes, alternately inward and outward (odd, >= 1) */
  double refit_scale;      /* step 9: a refit pass starts from the previous covariance times this */
} oracle_params;

void ORACLE_SYM(default_params)(oracle_params* p) {
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
  p->merge_gap_rows = 10;
  p->merge_dw = 5.0;
  p->merge_chi2_max = 50.0;
  p->refit_passes = 3;
  p->refit_scale = 100.0;
}

typedef struct {
  real kq;                 /* dk/d(q/pT) = -0.0029979246 * Bz */
  real ky, kw, eps, chi_n_max;
  int lmin;
  real r00, r11;           /* measurement variances */
  real chi2_hit_max;
  int n_miss_max;
  real win_nsig, win_add;
  int ms_on;
  real x0_row, ms_c, mass2;
  real max_sin, y_margin, tan10;
  int nmin;
  real cov0[5];
  real x[NROW];
  int want_margins;
  int ext_stop;
  real drift_len, vdrift;
  real keep_vy, keep_vw, keep_qpt_max;
  int merge_gap_rows;
  real merge_dw, merge_chi2_max;
  real rot_c, rot_s;       /* cos and sin of the 20-degree angle between neighbouring sectors */
  real refit_scale;        /* step 9: a refit pass starts from the previous covariance times this */
  int refit_passes;        /* step 9: passes of the refit, alternately inward and outward (odd) */
} ctx_t;

static void make_ctx(const oracle_params* p, ctx_t* c) {
  c->kq = (real)(-0.0029979246 * p->bz);
  c->ky = (real)p->ky; c->kw = (real)p->kw; c->eps = (real)p->eps;
  c->chi_n_max = (real)p->chi_n_max;
  c->lmin = p->lmin;
  c->r00 = (real)(p->sigma_y * p->sigma_y);
  c->r11 = (real)(p->sigma_w * p->sigma_w);
  c->chi2_hit_max = (real)p->chi2_hit_max;
  c->n_miss_max = p->n_miss_max;
  c->win_nsig = (real)p->win_nsig; c->win_add = (real)p->win_add;
  c->ms_on = p->x0_per_row > 0;
  c->x0_row = (real)p->x0_per_row;
  /* Highland: theta0 = 0.0136/(beta p) sqrt(x/X0) (1 + 0.038 ln(x/X0)); the log term is taken at
   * the nominal per-row thickness, so theta0^2 = ms_c * (x/X0) / (beta^2 p^2). */
  {
    double hl = p->x0_per_row > 0 ? 0.0136 * (1.0 + 0.038 * log(p->x0_per_row)) : 0.0;
    c->ms_c = (real)(hl * hl);
  }
  c->mass2 = (real)(0.13957039 * 0.13957039);
  c->max_sin = (real)p->max_sin;
  c->y_margin = (real)p->y_margin;
  c->tan10 = (real)0.17632698070846498;
  c->nmin = p->nmin;
  for (int i = 0; i < 5; ++i) c->cov0[i] = (real)p->cov0[i];
  c->ext_stop = p->ext_stop;
  c->drift_len = (real)p->drift_length;
  c->vdrift = (real)p->drift_velocity;
  c->keep_vy = (real)p->keep_vy;
  c->keep_vw = (real)p->keep_vw;
  c->keep_qpt_max = (real)p->keep_qpt_max;
  c->merge_gap_rows = p->merge_gap_rows;
  c->merge_dw = (real)p->merge_dw;
  c->merge_chi2_max = (real)p->merge_chi2_max;
  c->rot_c = (real)0.93969262078590838;  /* cos(20 deg) */
  c->rot_s = (real)0.34202014332566873;  /* sin(20 deg) */
  c->refit_scale = (real)p->refit_scale;
  c->refit_passes = p->refit_passes;
  for (int r = 0; r < NROW; ++r) c->x[r] = (real)85 + (real)r * ((real)160 / (real)151);
  c->want_margins = 1;
}

static inline real absr(real v) { return v < 0 ? -v : v; }

/* 16-bit fixed-point cluster storage (Sec. 4 of the paper: custom formats that keep only the bits
 * the intrinsic resolution needs). y is stored as qy = rint((y + 64) * 512) clamped to [0, 65535],
 * read back as qy / 512 - 64; w is stored as a 16-bit offset, in steps of 2^-9 cm, from the lower
 * edge of its search-grid bin (bins are aligned power-of-two widths of at most 128 cm), which reads
 * back as rint(512 w) / 512 whatever the bin. Both read-back values are exact floats for
 * |w| < 32768 cm; the tracker then sees only them. */
static void pack_roundtrip(real* y, real* w) {
  real qy = RINT((*y + (real)64) * (real)512);
  if (qy < 0) qy = 0;
  if (qy > 65535) qy = 65535;
  *y = qy * ((real)1 / (real)512) - (real)64;
  *w = RINT(*w * (real)512) * ((real)1 / (real)512);
}

/* Relative distance of a decision variable from its cut, for tracing disagreements. */
static inline void note_margin(double* m, real value, real cut) {
  if (!m) return;
  double d = fabs((double)value - (double)cut);
  double s = fabs((double)cut);
  double rel = s > 1e-30 ? d / s : d;
  if (rel < *m) *m = rel;
}

/* ------------------------------------------------------------------------------------------------
 * asin by half-angle reduction + Maclaurin series (no library transcendental):
 *   asin(t)/t = 1 + t^2/6 + 3t^4/40 + 5t^6/112 + 35t^8/1152 + 63t^10/2816 + ...   for |t| < 0.1,
 *   sin(a/2) = sin(a) / sqrt(2 (1 + cos a))  ->  asin(t) = 2 asin(t / sqrt(2 (1 + sqrt(1 - t^2)))).
 * ---------------------------------------------------------------------------------------------- */
static real asin_series_ratio(real t) { /* Horner, one fused multiply-add per coefficient */
  const real t2 = t * t;
  real p = (real)0.022372159090909092;
  p = FMA(t2, p, (real)0.030381944444444444);
  p = FMA(t2, p, (real)0.044642857142857144);
  p = FMA(t2, p, (real)0.075);
  p = FMA(t2, p, (real)0.16666666666666666);
  return FMA(t2, p, (real)1);
}
static real asin_hr(real t) {
  real scale = (real)1;
  while (absr(t) >= (real)0.1) {
    t = t / SQRT((real)2 * ((real)1 + SQRT((real)1 - t * t)));
    scale = scale * (real)2;
  }
  return scale * t * asin_series_ratio(t);
}
/* asin(t)/t: arc length over chord for a circle, t = chord * k / 2 */
static real arc_ratio(real t) {
  if (absr(t) < (real)0.1) return asin_series_ratio(t);
  return asin_hr(t) / t;
}
/* d/dt (asin(t)/t) */
static real arc_ratio_deriv(real t) {
  if (absr(t) < (real)0.1) {
    const real t2 = t * t;
    real p = (real)0.22372159090909091;
    p = FMA(t2, p, (real)0.24305555555555555);
    p = FMA(t2, p, (real)0.26785714285714285);
    p = FMA(t2, p, (real)0.3);
    p = FMA(t2, p, (real)0.3333333333333333);
    return t * p;
  }
  return ((real)1 / SQRT((real)1 - t * t) - arc_ratio(t)) / t;
}

double ORACLE_SYM(asin)(double t) { return (double)asin_hr((real)t); }

/* the 16-bit storage round trip of one cluster's (y, w) */
void ORACLE_SYM(pack)(double* y, double* w) {
  real a = (real)*y, b = (real)*w;
  pack_roundtrip(&a, &b);
  *y = a;
  *w = b;
}

/* ------------------------------------------------------------------------------------------------
 * Small dense linear algebra (5x5), written out plainly. Every sum of products in the Kalman
 * filter accumulates with a fused multiply-add (one rounding per term), in index order.
 * ---------------------------------------------------------------------------------------------- */
static void mat_mul5(real A[5][5], real B[5][5], real O[5][5]) {
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) {
      real acc = 0;
      for (int j = 0; j < 5; ++j) acc = FMA(A[i][j], B[j][k], acc);
      O[i][k] = acc;
    }
}
static void mat_mul5_bt(real A[5][5], real B[5][5], real O[5][5]) { /* O = A * B^T */
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) {
      real acc = 0;
      for (int j = 0; j < 5; ++j) acc = FMA(A[i][j], B[k][j], acc);
      O[i][k] = acc;
    }
}
/* keep symmetric: the lower triangle (row >= column) is the value, mirrored to the upper */
static void mirror_lower(real C[5][5]) {
  for (int i = 0; i < 5; ++i)
    for (int k = i + 1; k < 5; ++k) C[i][k] = C[k][i];
}

/* ------------------------------------------------------------------------------------------------
 * Kalman filter pieces
 * ---------------------------------------------------------------------------------------------- */

/* Exact helix transport of (P, C) from x0 to x1 in the sector frame, with multiple-scattering
 * process noise. Returns 0 on success, 1 if |sin phi| would reach max_sin. */
static int kf_propagate(const ctx_t* cx, real P[5], real C[5][5], real x0, real x1, double* m,
                        real (*Jout)[5]) {
  const real dx = x1 - x0;
  const real k = cx->kq * P[4];
  const real s0 = P[2];
  const real s1 = s0 + k * dx;
  note_margin(m, absr(s1), cx->max_sin);
  if (!(absr(s1) < cx->max_sin)) return 1;
  const real c0 = SQRT((real)1 - s0 * s0);
  const real c1 = SQRT((real)1 - s1 * s1);
  const real N = s0 + s1, D = c0 + c1;
  const real iD = (real)1 / D;
  const real dy = dx * QUO(N, D, iD);           /* chord relation of a circle */
  const real l = SQRT(dx * dx + dy * dy);       /* chord length in the xy plane */
  const real t = l * k * (real)0.5;             /* sin of half the turning angle */
  real a = l * arc_ratio(t);                    /* arc length */
  if (dx < 0) a = -a;
  const real tw = P[3];
  const real ic0 = (real)1 / c0, ic1 = (real)1 / c1, il = (real)1 / l;
  /* Jacobian d(y1, w1, s1, t, q/pT) / d(y0, w0, s0, t, q/pT) */
  const real iDD = iD * iD;
  const real dy_ds0 = dx * (QUO((real)2, D, iD) + QUO(N * (QUO(s0, c0, ic0) + QUO(s1, c1, ic1)), D * D, iDD));
  const real dy_dk = dx * dx * (QUO((real)1, D, iD) + QUO(QUO(N * s1, c1, ic1), D * D, iDD));
  real da_dl = (real)1 / SQRT((real)1 - t * t);
  real da_dk = l * l * (real)0.5 * arc_ratio_deriv(t); /* at fixed chord */
  if (dx < 0) { da_dl = -da_dl; da_dk = -da_dk; }
  const real dl_ds0 = QUO(dy * dy_ds0, l, il);
  const real dl_dk = QUO(dy * dy_dk, l, il);
  real J[5][5];
  memset(J, 0, sizeof(J));
  for (int i = 0; i < 5; ++i) J[i][i] = 1;
  J[0][2] = dy_ds0;
  J[0][4] = dy_dk * cx->kq;
  J[1][2] = tw * (da_dl * dl_ds0);
  J[1][3] = a;
  J[1][4] = tw * (da_dl * dl_dk + da_dk) * cx->kq;
  J[2][4] = dx * cx->kq;
  if (Jout) memcpy(Jout, J, sizeof(J));
  /* state */
  P[0] = P[0] + dy;
  P[1] = P[1] + tw * a;
  P[2] = s1;
  /* covariance: J C J^T */
  real T[5][5], O[5][5];
  mat_mul5(J, C, T);
  mat_mul5_bt(T, J, O);
  mirror_lower(O);
  /* multiple scattering: theta0^2 on the direction; var(sin phi) = c^2 (1+t^2) th^2,
   * var(t) = (1+t^2)^2 th^2; with q2 = 1/p^2 = (q/pT)^2/(1+t^2), 1/(beta p)^2 = q2 (1 + m^2 q2) */
  if (cx->ms_on && P[4] != 0) {
    const real one_tw2 = (real)1 + tw * tw;
    const real pathf = QUO(SQRT(one_tw2), c1, ic1);
    const real xx0 = cx->x0_row * pathf;
    const real q2 = P[4] * P[4] / one_tw2;
    const real th2 = cx->ms_c * xx0 * q2 * ((real)1 + cx->mass2 * q2);
    O[2][2] = O[2][2] + th2 * (c1 * c1) * one_tw2;
    O[3][3] = O[3][3] + th2 * one_tw2 * one_tw2;
  }
  memcpy(C, O, sizeof(O));
  return 0;
}

/* The state part of kf_propagate alone (the same operations): step 8's predictions. */
static int propagate_state(const ctx_t* cx, real P[5], real x0, real x1) {
  const real dx = x1 - x0;
  const real k = cx->kq * P[4];
  const real s0 = P[2];
  const real s1 = s0 + k * dx;
  if (!(absr(s1) < cx->max_sin)) return 1;
  const real c0 = SQRT((real)1 - s0 * s0);
  const real c1 = SQRT((real)1 - s1 * s1);
  const real N = s0 + s1, D = c0 + c1;
  const real iD = (real)1 / D;
  const real dy = dx * QUO(N, D, iD);
  const real l = SQRT(dx * dx + dy * dy);
  const real t = l * k * (real)0.5;
  real a = l * arc_ratio(t);
  if (dx < 0) a = -a;
  P[0] = P[0] + dy;
  P[1] = P[1] + P[3] * a;
  P[2] = s1;
  return 0;
}

/* chi2 of a measurement (ym, wm) against the state; returns +inf if S is not positive definite */
static real kf_chi2(const ctx_t* cx, const real P[5], real C[5][5], real ym, real wm) {
  const real S00 = C[0][0] + cx->r00, S01 = C[0][1], S10 = C[1][0], S11 = C[1][1] + cx->r11;
  const real det = S00 * S11 - S01 * S10;
  if (!(det > 0)) return (real)INFINITY;
  const real idet = (real)1 / det;
  const real i00 = QUO(S11, det, idet), i01 = QUO(-S01, det, idet), i10 = QUO(-S10, det, idet),
             i11 = QUO(S00, det, idet);
  const real r0 = ym - P[0], r1 = wm - P[1];
  const real u0 = FMA(i01, r1, i00 * r0), u1 = FMA(i11, r1, i10 * r0); /* S^-1 r */
  return FMA(r1, u1, r0 * u0);
}

/* Kalman update with measurement (ym, wm): gain K = C H^T S^-1, Joseph form
 * C' = (I - K H) C (I - K H)^T + K R K^T, then symmetrised from the lower triangle. */
static void kf_update(const ctx_t* cx, real P[5], real C[5][5], real ym, real wm) {
  real S[2][2], Si[2][2];
  S[0][0] = C[0][0] + cx->r00; S[0][1] = C[0][1] + 0;
  S[1][0] = C[1][0] + 0;       S[1][1] = C[1][1] + cx->r11;
  const real det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
  const real idet = (real)1 / det;
  Si[0][0] = QUO(S[1][1], det, idet); Si[0][1] = QUO(-S[0][1], det, idet);
  Si[1][0] = QUO(-S[1][0], det, idet); Si[1][1] = QUO(S[0][0], det, idet);
  real K[5][2];
  for (int i = 0; i < 5; ++i)
    for (int l = 0; l < 2; ++l) {
      real acc = 0;
      for (int m = 0; m < 2; ++m) acc = FMA(C[i][m], Si[m][l], acc); /* (C H^T)[i][m] = C[i][m] */
      K[i][l] = acc;
    }
  const real r[2] = {ym - P[0], wm - P[1]};
  for (int i = 0; i < 5; ++i) {
    real acc = 0;
    for (int l = 0; l < 2; ++l) acc = FMA(K[i][l], r[l], acc);
    P[i] = P[i] + acc;
  }
  real A[5][5], T[5][5], O[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      real kh = 0;
      for (int l = 0; l < 2; ++l) kh = FMA(K[i][l], (real)(l == j ? 1 : 0), kh); /* (K H)[i][j] */
      A[i][j] = (real)(i == j ? 1 : 0) - kh;
    }
  mat_mul5(A, C, T);
  mat_mul5_bt(T, A, O);
  real KR[5][2];
  for (int i = 0; i < 5; ++i) {
    real acc0 = 0, acc1 = 0;
    acc0 = FMA(K[i][0], cx->r00, acc0); acc0 = FMA(K[i][1], (real)0, acc0);
    acc1 = FMA(K[i][0], (real)0, acc1); acc1 = FMA(K[i][1], cx->r11, acc1);
    KR[i][0] = acc0; KR[i][1] = acc1;
  }
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) {
      real acc = 0;
      for (int b = 0; b < 2; ++b) acc = FMA(KR[i][b], K[k][b], acc);
      O[i][k] = O[i][k] + acc;
    }
  mirror_lower(O);
  memcpy(C, O, sizeof(O));
}

/* Seed from three hits (x, y, w) of a chain: circle through them in (x, y), the state at the first
 * hit, w-slope from the end points over the arc. Returns 0 on success. */
static int kf_seed(const ctx_t* cx, const real h[3][3], real P[5], double* m) {
  const real ax = h[1][0] - h[0][0], ay = h[1][1] - h[0][1];
  const real bx = h[2][0] - h[0][0], by = h[2][1] - h[0][1];
  const real cx_ = h[2][0] - h[1][0], cy = h[2][1] - h[1][1];
  const real cross = ax * by - ay * bx;
  const real d01 = SQRT(ax * ax + ay * ay);
  const real d02 = SQRT(bx * bx + by * by);
  const real d12 = SQRT(cx_ * cx_ + cy * cy);
  const real k = (real)2 * cross / (d01 * d02 * d12);
  const real sg = k * d02 * (real)0.5;      /* sin of the angle between chord and tangent */
  note_margin(m, absr(sg), (real)1);
  if (!(absr(sg) < (real)1)) return 1;
  const real cg = SQRT((real)1 - sg * sg);
  const real sphi = (by * cg - bx * sg) / d02;
  note_margin(m, absr(sphi), cx->max_sin);
  if (!(absr(sphi) < cx->max_sin)) return 1;
  const real arc = d02 * arc_ratio(sg);
  P[0] = h[0][1];
  P[1] = h[0][2];
  P[2] = sphi;
  P[3] = (h[2][2] - h[0][2]) / arc;
  P[4] = cx->kq != 0 ? k / cx->kq : (real)0;
  return 0;
}

/* Step 7, beam line: the track's fit (P, C at x_ref) transported to x = 0 without scattering; out =
 * (y0, w0, var(w0), t0 = (w0 - L) / v_d, z_ref = +-(w0 - w_ref), + on side A); all NaN when the
 * transport fails (|sin phi| reaches max_sin on the way). */
static void beamline(const ctx_t* cx, const real P[5], real C[5][5], real x_ref, int sector, real out[5]) {
  ctx_t c0 = *cx;
  c0.ms_on = 0;
  real Pb[5], Cb[5][5];
  memcpy(Pb, P, sizeof(Pb));
  memcpy(Cb, C, sizeof(Cb));
  if (kf_propagate(&c0, Pb, Cb, x_ref, (real)0, NULL, NULL)) {
    for (int i = 0; i < 5; ++i) out[i] = (real)NAN;
    return;
  }
  const real w0 = Pb[1];
  const real dz = w0 - P[1];
  out[0] = Pb[0];
  out[1] = w0;
  out[2] = Cb[1][1];
  out[3] = (w0 - cx->drift_len) / cx->vdrift;
  out[4] = sector < NSEC / 2 ? dz : -dz;
}

/* ------------------------------------------------------------------------------------------------
 * Exported unit entry points (for the pins): one propagation, one update, one seed.
 * State/covariance exchange in double: P[5], C[25] (row-major full matrix).
 * ---------------------------------------------------------------------------------------------- */
int ORACLE_SYM(propagate)(const oracle_params* p, double* P, double* C, double x0, double x1,
                          double* J) {
  ctx_t cx;
  make_ctx(p, &cx);
  real Pr[5], Cr[5][5], Jr[5][5];
  for (int i = 0; i < 5; ++i) Pr[i] = (real)P[i];
  for (int i = 0; i < 25; ++i) Cr[i / 5][i % 5] = (real)C[i];
  memset(Jr, 0, sizeof(Jr));
  int rc = kf_propagate(&cx, Pr, Cr, (real)x0, (real)x1, NULL, Jr);
  for (int i = 0; i < 5; ++i) P[i] = Pr[i];
  for (int i = 0; i < 25; ++i) C[i] = Cr[i / 5][i % 5];
  if (J)
    for (int i = 0; i < 25; ++i) J[i] = Jr[i / 5][i % 5];
  return rc;
}
double ORACLE_SYM(update)(const oracle_params* p, double* P, double* C, double ym, double wm) {
  ctx_t cx;
  make_ctx(p, &cx);
  real Pr[5], Cr[5][5];
  for (int i = 0; i < 5; ++i) Pr[i] = (real)P[i];
  for (int i = 0; i < 25; ++i) Cr[i / 5][i % 5] = (real)C[i];
  real chi2 = kf_chi2(&cx, Pr, Cr, (real)ym, (real)wm);
  kf_update(&cx, Pr, Cr, (real)ym, (real)wm);
  for (int i = 0; i < 5; ++i) P[i] = Pr[i];
  for (int i = 0; i < 25; ++i) C[i] = Cr[i / 5][i % 5];
  return (double)chi2;
}
int ORACLE_SYM(seed)(const oracle_params* p, const double* h9, double* P) {
  ctx_t cx;
  make_ctx(p, &cx);
  real h[3][3], Pr[5];
  for (int i = 0; i < 9; ++i) h[i / 3][i % 3] = (real)h9[i];
  int rc = kf_seed(&cx, h, Pr, NULL);
  for (int i = 0; i < 5; ++i) P[i] = rc ? NAN : (double)Pr[i];
  return rc;
}
void ORACLE_SYM(beamline)(const oracle_params* p, const double* P, const double* C, double x_ref, int sector,
                          double* out) {
  ctx_t cx;
  make_ctx(p, &cx);
  real Pr[5], Cr[5][5], o[5];
  for (int i = 0; i < 5; ++i) Pr[i] = (real)P[i];
  for (int i = 0; i < 25; ++i) Cr[i / 5][i % 5] = (real)C[i];
  beamline(&cx, Pr, Cr, (real)x_ref, sector, o);
  for (int i = 0; i < 5; ++i) out[i] = (double)o[i];
}
double ORACLE_SYM(row_x)(int r) {
  ctx_t cx;
  oracle_params p;
  ORACLE_SYM(default_params)(&p);
  make_ctx(&p, &cx);
  return (r >= 0 && r < NROW) ? (double)cx.x[r] : NAN;
}

/* ------------------------------------------------------------------------------------------------
 * Whole-frame tracker
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  int64_t n_clusters;
  /* links in caller (original) index space, -1 = none */
  int32_t *up, *down, *up_c, *down_c;
  double* nb_margin;               /* per cluster: min relative margin of its neighbour decisions */
  /* start hits in canonical order (sector, rank) */
  int64_t n_start;
  int32_t* start;
  /* tracklets (one per start hit, same order) */
  int64_t n_tracklets;
  int32_t *tl_sector, *tl_start, *tl_nhits, *tl_ndf, *tl_row_ref, *tl_row_top, *tl_ok;
  double *tl_xref, *tl_param, *tl_cov, *tl_chi2, *tl_margin;
  int64_t* tl_hit_off;             /* [n_tracklets + 1] */
  int32_t* tl_hits;                /* original indices, ascending row */
  /* tracks in canonical order (sector, rank of the tracklet's start hit) */
  int64_t n_tracks;
  int32_t *tr_sector, *tr_ndf, *tr_nhits, *tr_tracklet;
  double *tr_xref, *tr_param, *tr_cov, *tr_chi2;
  double* tr_beam;                 /* [n_tracks][5] step 7: y0, w0, var(w0), t0, z_ref */
  int32_t* tr_res;                 /* [total track hits][2] step 8: residuals (or absolute) */
  int32_t* tr_npred;               /* [n_tracks] step 8: hits stored as residuals */
  uint8_t* keep;                   /* [n_clusters] step 8: strategy-B protection */
  int64_t* tr_hit_off;
  int32_t* tr_hits;                /* original indices, ascending row */
  struct merge_out* merged;        /* step 9 (ORACLE_MERGE), else NULL */
} oracle_result;

/* Step 9 output: merged tracks in canonical order (the canonical index of their innermost sector
 * track), each a chain of sector tracks (segments) inner to outer, refit over all their hits. */
typedef struct merge_out {
  int64_t n_tracks;                /* sector tracks the step read */
  int64_t n_merged;
  int32_t *mt_head, *mt_nseg, *mt_sector, *mt_ndf, *mt_nfit;
  double *mt_xref, *mt_param, *mt_cov, *mt_chi2;
  int64_t* mt_hit_off;             /* [n_merged + 1] */
  int32_t* mt_hits;                /* original indices: the segments' hits, inner segment first */
  int32_t* tr_next;                /* [n_tracks] the outer partner of each sector track, -1 if none */
  double* tr_merge_chi2;           /* [n_tracks] chi2 of that merge, NaN if none */
  double* tr_outer;                /* [n_tracks][5] the fit transported to the last hit's row, NaN if it fails */
} merge_out;

#define ORACLE_BRUTE_FORCE 1
#define ORACLE_PACKED 2
#define ORACLE_MERGE 4


typedef struct {
  int64_t n;                 /* clusters of this sector */
  int64_t row_start[NROW + 1];
  int32_t* orig;             /* sorted by (row, w, orig) */
  real *y, *w;
  int32_t *up, *dn, *upc, *dnc; /* local indices */
  double* nbm;
  /* tracklets */
  int64_t nt, cap_t;
  int32_t *t_start, *t_rank, *t_nhits, *t_ndf, *t_rref, *t_rtop, *t_ok;
  real *t_x, *t_p, *t_c, *t_chi2;
  double* t_m;
  int32_t* t_slots;          /* [nt][NROW] local hit per row, -1 */
  /* tracks */
  int64_t ntr;
  int32_t* tr_t;             /* tracklet index */
  int32_t* tr_nk;            /* kept hits */
  int32_t* tr_min;           /* smallest original index among kept hits */
  uint64_t* weight;          /* per local hit */
  uint8_t* is_start;         /* per local hit: 1 for the start hit of a tracklet */
} sector_t;

/* Each row is ordered by (w, y, original index). A hit's position in this order (its "rank") is
 * the tie-break of every arg-min below and of the selection key, so results do not depend on the
 * caller's cluster order unless two clusters of a row have identical coordinates. */
typedef struct { real w; int32_t orig; real y; } rowhit;
static int cmp_rowhit(const void* a, const void* b) {
  const rowhit* x = (const rowhit*)a;
  const rowhit* y = (const rowhit*)b;
  if (x->w < y->w) return -1;
  if (x->w > y->w) return 1;
  if (x->y < y->y) return -1;
  if (x->y > y->y) return 1;
  return x->orig < y->orig ? -1 : (x->orig > y->orig);
}

/* first local index in row r with w >= v (rows are sorted by w) */
static int64_t row_lower_bound(const sector_t* S, int r, real v) {
  int64_t lo = S->row_start[r], hi = S->row_start[r + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (S->w[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* Step 8 for track t (tracklet key `key`): residuals res[2 i], res[2 i + 1] of its i-th hit (ascending
 * rows), the number of predicted hits, and the protection of the clusters near a good track. */
static int32_t quant(real v) { return (int32_t)RINT(v * (real)512); }
static void compress_track(const ctx_t* cx, const sector_t* S, int64_t t, uint64_t key, int32_t* res,
                           int32_t* npred, uint8_t* keep) {
  real P[5];
  for (int i = 0; i < 5; ++i) P[i] = S->t_p[t * 5 + i];
  const int r0 = S->t_rref[t];
  int last = -1;
  for (int r = NROW - 1; r >= 0 && last < 0; --r) {
    const int32_t h = S->t_slots[t * NROW + r];
    if (h >= 0 && S->weight[h] == key) last = r;
  }
  const int good = absr(P[4]) <= cx->keep_qpt_max;
  int ok = 1, n = 0, np = 0;
  for (int r = r0; r <= last; ++r) {
    real Pr[5];
    for (int i = 0; i < 5; ++i) Pr[i] = P[i];
    if (ok && r > r0 && propagate_state(cx, Pr, cx->x[r0], cx->x[r])) ok = 0;
    if (ok && good) {
      /* the row's clusters within the vicinity (exact test; the w range searched is widened by
       * the rounding of w +- vw) */
      const real pad = absr(Pr[1]) * (real)1e-6 + cx->keep_vw * (real)1e-6 + (real)1e-6;
      const real lo = (Pr[1] - cx->keep_vw) - pad, hi = (Pr[1] + cx->keep_vw) + pad;
      for (int64_t i = row_lower_bound(S, r, lo); i < S->row_start[r + 1] && S->w[i] <= hi; ++i)
        if (absr(S->w[i] - Pr[1]) <= cx->keep_vw && absr(S->y[i] - Pr[0]) <= cx->keep_vy) keep[i] = 1;
    }
    const int32_t h = S->t_slots[t * NROW + r];
    if (h >= 0 && S->weight[h] == key) {
      if (good) keep[h] = 1;
      if (ok) {
        res[2 * n] = quant(S->y[h]) - quant(Pr[0]);
        res[2 * n + 1] = quant(S->w[h]) - quant(Pr[1]);
        ++np;
      } else {
        res[2 * n] = quant(S->y[h]);
        res[2 * n + 1] = quant(S->w[h]);
      }
      ++n;
    }
  }
  *npred = np;
}

/* candidates in row rr of hit (yi, wi) within |dy| <= wy, |dw| <= ww: index range to scan */
static void scan_range(const sector_t* S, int rr, real wi, real ww, int brute, int64_t* b, int64_t* e) {
  if (brute) { *b = S->row_start[rr]; *e = S->row_start[rr + 1]; return; }
  /* widen by a hair so that hits just outside the window are visited for the margin trace; the
   * exact window test below decides */
  real pad = ww * (real)1e-3 + (real)1e-3;
  *b = row_lower_bound(S, rr, wi - ww - pad);
  int64_t hi = row_lower_bound(S, rr, wi + ww + pad);
  while (hi < S->row_start[rr + 1] && !(S->w[hi] > wi + ww + pad)) ++hi;
  *e = hi;
}

static void find_neighbours(const ctx_t* cx, sector_t* S, int brute) {
  for (int64_t i = 0; i < S->n; ++i) { S->up[i] = -1; S->dn[i] = -1; S->nbm[i] = INFINITY; }
  for (int r = 1; r + 1 < NROW; ++r) {
    const real dxm = cx->x[r] - cx->x[r - 1];
    const real dxp = cx->x[r + 1] - cx->x[r];
    const real wy_dn = cx->ky * dxm + cx->eps, ww_dn = cx->kw * dxm + cx->eps;
    const real wy_up = cx->ky * dxp + cx->eps, ww_up = cx->kw * dxp + cx->eps;
    const real f = dxm / (dxm + dxp);
    for (int64_t i = S->row_start[r]; i < S->row_start[r + 1]; ++i) {
      const real yi = S->y[i], wi = S->w[i];
      double* m = &S->nbm[i];
      int64_t db, de, ub, ue;
      scan_range(S, r - 1, wi, ww_dn, brute, &db, &de);
      scan_range(S, r + 1, wi, ww_up, brute, &ub, &ue);
      real best = (real)INFINITY, second = (real)INFINITY;
      int64_t bd = -1, bu = -1;
      for (int64_t d = db; d < de; ++d) {
        const real ady = absr(S->y[d] - yi), adw = absr(S->w[d] - wi);
        note_margin(m, ady, wy_dn);
        note_margin(m, adw, ww_dn);
        if (!(ady <= wy_dn && adw <= ww_dn)) continue;
        for (int64_t u = ub; u < ue; ++u) {
          const real uy = absr(S->y[u] - yi), uw = absr(S->w[u] - wi);
          note_margin(m, uy, wy_up);
          note_margin(m, uw, ww_up);
          if (!(uy <= wy_up && uw <= ww_up)) continue;
          const real py = S->y[d] + (S->y[u] - S->y[d]) * f;
          const real pw = S->w[d] + (S->w[u] - S->w[d]) * f;
          const real ey = yi - py, ew = wi - pw;
          const real chi = ey * ey + ew * ew;
          /* lexicographic minimum of (chi_n, rank of d, rank of u) */
          int better;
          if (bd < 0 || chi < best) better = 1;
          else if (chi > best) better = 0;
          else if (d != bd) better = d < bd;
          else better = u < bu;
          if (better) { second = best; best = chi; bd = d; bu = u; }
          else if (chi < second) second = chi;
        }
      }
      if (bd >= 0) {
        note_margin(m, best, cx->chi_n_max);
        if (second < (real)INFINITY) note_margin(m, second, best);
        if (best <= cx->chi_n_max) { S->dn[i] = (int32_t)bd; S->up[i] = (int32_t)bu; }
      }
    }
  }
}

static void clean_links(sector_t* S) {
  for (int64_t i = 0; i < S->n; ++i) {
    int32_t u = S->up[i], d = S->dn[i];
    S->upc[i] = (u >= 0 && S->dn[u] == i) ? u : -1;
    S->dnc[i] = (d >= 0 && S->up[d] == i) ? d : -1;
  }
}

/* Search row r of the sector for the hit with the smallest chi2 inside the window around the
 * predicted (y, w). Returns the local index or -1, and its chi2. */
static int64_t search_row(const ctx_t* cx, const sector_t* S, int r, const real P[5], real C[5][5],
                          real* chi2_out, double* m) {
  const real wy = cx->win_nsig * SQRT(C[0][0]) + cx->win_add;
  const real ww = cx->win_nsig * SQRT(C[1][1]) + cx->win_add;
  int64_t b, e;
  scan_range(S, r, P[1], ww, 0, &b, &e);
  int64_t best = -1;
  real bchi = (real)INFINITY, second = (real)INFINITY;
  for (int64_t h = b; h < e; ++h) {
    const real ady = absr(S->y[h] - P[0]), adw = absr(S->w[h] - P[1]);
    note_margin(m, ady, wy);
    note_margin(m, adw, ww);
    if (!(ady <= wy && adw <= ww)) continue;
    const real chi = kf_chi2(cx, P, C, S->y[h], S->w[h]);
    /* lexicographic minimum of (chi2, rank) */
    int better;
    if (best < 0 || chi < bchi) better = 1;
    else if (chi > bchi) better = 0;
    else better = h < best;
    if (better) { second = bchi; bchi = chi; best = h; }
    else if (chi < second) second = chi;
  }
  if (best >= 0 && second < (real)INFINITY) note_margin(m, second, bchi);
  *chi2_out = bchi;
  return best;
}

static void add_tracklet_storage(sector_t* S) {
  if (S->nt < S->cap_t) return;
  int64_t nc = S->cap_t ? 2 * S->cap_t : 64;
  S->t_start = realloc(S->t_start, nc * sizeof(int32_t));
  S->t_rank = realloc(S->t_rank, nc * sizeof(int32_t));
  S->t_nhits = realloc(S->t_nhits, nc * sizeof(int32_t));
  S->t_ndf = realloc(S->t_ndf, nc * sizeof(int32_t));
  S->t_rref = realloc(S->t_rref, nc * sizeof(int32_t));
  S->t_rtop = realloc(S->t_rtop, nc * sizeof(int32_t));
  S->t_ok = realloc(S->t_ok, nc * sizeof(int32_t));
  S->t_x = realloc(S->t_x, nc * sizeof(real));
  S->t_p = realloc(S->t_p, nc * 5 * sizeof(real));
  S->t_c = realloc(S->t_c, nc * 15 * sizeof(real));
  S->t_chi2 = realloc(S->t_chi2, nc * sizeof(real));
  S->t_m = realloc(S->t_m, nc * sizeof(double));
  S->t_slots = realloc(S->t_slots, nc * NROW * sizeof(int32_t));
  S->cap_t = nc;
}

/* Build the tracklet of start hit h0 (local index) in row r0. */
static void build_tracklet(const ctx_t* cx, sector_t* S, int64_t h0, int r0) {
  add_tracklet_storage(S);
  const int64_t t = S->nt++;
  double mg = INFINITY;
  double* m = cx->want_margins ? &mg : NULL;
  int32_t* slotC = &S->t_slots[t * NROW];
  int32_t slotAB[NROW];
  for (int r = 0; r < NROW; ++r) { slotC[r] = -1; slotAB[r] = -1; }
  S->t_start[t] = S->orig[h0];
  S->t_rank[t] = (int32_t)h0;
  S->t_ok[t] = 0; S->t_nhits[t] = 0; S->t_ndf[t] = -5; S->t_rref[t] = -1; S->t_rtop[t] = -1;
  S->t_x[t] = 0; S->t_chi2[t] = 0;
  for (int i = 0; i < 5; ++i) S->t_p[t * 5 + i] = 0;
  for (int i = 0; i < 15; ++i) S->t_c[t * 15 + i] = 0;
  /* the chain */
  int64_t chain[NROW];
  int mlen = 0;
  for (int64_t h = h0; h >= 0 && mlen < NROW; h = S->upc[h]) chain[mlen++] = h;
  /* seed */
  real hh[3][3];
  const int64_t hs[3] = {chain[0], chain[mlen / 2], chain[mlen - 1]};
  const int rs[3] = {r0, r0 + mlen / 2, r0 + mlen - 1};
  for (int j = 0; j < 3; ++j) { hh[j][0] = cx->x[rs[j]]; hh[j][1] = S->y[hs[j]]; hh[j][2] = S->w[hs[j]]; }
  real P[5], C[5][5];
  if (kf_seed(cx, hh, P, m)) { S->t_m[t] = mg; return; }
  memset(C, 0, sizeof(C));
  for (int i = 0; i < 5; ++i) C[i][i] = cx->cov0[i];
  /* Phase A (chain) and B (outward extension) */
  real Ptop[5], Ctop[5][5];
  int top = -1, nmiss = 0;
  for (int r = r0; r < NROW; ++r) {
    if (r > r0) {
      if (kf_propagate(cx, P, C, cx->x[r - 1], cx->x[r], m, NULL)) break;
      const real lim = cx->x[r] * cx->tan10 + cx->y_margin;
      note_margin(m, absr(P[0]), lim);
      if (absr(P[0]) > lim) break;
    }
    int64_t hit;
    real chi;
    if (r < r0 + mlen) {
      hit = chain[r - r0];
      chi = kf_chi2(cx, P, C, S->y[hit], S->w[hit]);
    } else {
      hit = search_row(cx, S, r, P, C, &chi, m);
    }
    if (hit >= 0) note_margin(m, chi, cx->chi2_hit_max);
    if (hit >= 0 && chi <= cx->chi2_hit_max) {
      kf_update(cx, P, C, S->y[hit], S->w[hit]);
      slotAB[r] = (int32_t)hit;
      nmiss = 0;
      top = r;
      memcpy(Ptop, P, sizeof(Ptop));
      memcpy(Ctop, C, sizeof(Ctop));
      /* the extension reached another chain's start hit: that tracklet covers the rest outward */
      if (cx->ext_stop && r >= r0 + mlen && S->is_start[hit]) break;
    } else {
      ++nmiss;
      if (r >= r0 + mlen && nmiss >= cx->n_miss_max) break;
    }
  }
  if (top < 0) { S->t_m[t] = mg; return; }
  /* Phase C: inward refit from the outermost hit with the covariance reset, then inward extension */
  memcpy(P, Ptop, sizeof(P));
  memset(C, 0, sizeof(C));
  for (int i = 0; i < 5; ++i) C[i][i] = cx->cov0[i];
  real Pout[5], Cout[5][5];
  int ref = -1, nh = 0;
  real chi2sum = 0;
  nmiss = 0;
  for (int r = top; r >= 0; --r) {
    if (r < top) {
      if (kf_propagate(cx, P, C, cx->x[r + 1], cx->x[r], m, NULL)) break;
      const real lim = cx->x[r] * cx->tan10 + cx->y_margin;
      note_margin(m, absr(P[0]), lim);
      if (absr(P[0]) > lim) break;
    }
    int64_t hit;
    real chi = (real)INFINITY;
    if (r >= r0) {
      hit = slotAB[r];
      if (hit >= 0) chi = kf_chi2(cx, P, C, S->y[hit], S->w[hit]);
    } else {
      hit = search_row(cx, S, r, P, C, &chi, m);
    }
    if (hit >= 0) note_margin(m, chi, cx->chi2_hit_max);
    if (hit >= 0 && chi <= cx->chi2_hit_max) {
      kf_update(cx, P, C, S->y[hit], S->w[hit]);
      slotC[r] = (int32_t)hit;
      ++nh;
      chi2sum = chi2sum + chi;
      nmiss = 0;
      ref = r;
      memcpy(Pout, P, sizeof(Pout));
      memcpy(Cout, C, sizeof(Cout));
    } else {
      ++nmiss;
      if (r < r0 && nmiss >= cx->n_miss_max) break;
    }
  }
  S->t_m[t] = mg;
  if (ref < 0) return;
  S->t_ok[t] = 1;
  S->t_nhits[t] = nh;
  S->t_ndf[t] = 2 * nh - 5;
  S->t_rref[t] = ref;
  S->t_rtop[t] = top;
  S->t_x[t] = cx->x[ref];
  S->t_chi2[t] = chi2sum;
  for (int i = 0; i < 5; ++i) S->t_p[t * 5 + i] = Pout[i];
  for (int i = 0, o = 0; i < 5; ++i)
    for (int k = 0; k <= i; ++k, ++o) S->t_c[t * 15 + o] = Cout[i][k];
}

/* selection key: more hits first, then the smaller rank (position in the sector's row-ordered
 * hits) of the start hit; unique within a sector */
static uint64_t tracklet_key(const sector_t* S, int64_t t) {
  return ((uint64_t)(uint32_t)S->t_nhits[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)S->t_rank[t]);
}

static void select_tracks(const ctx_t* cx, sector_t* S) {
  S->weight = (uint64_t*)calloc(S->n > 0 ? S->n : 1, sizeof(uint64_t));
  for (int64_t t = 0; t < S->nt; ++t) {
    if (!S->t_ok[t] || S->t_nhits[t] < cx->nmin) continue;
    const uint64_t key = tracklet_key(S, t);
    for (int r = 0; r < NROW; ++r) {
      int32_t h = S->t_slots[t * NROW + r];
      if (h >= 0 && S->weight[h] < key) S->weight[h] = key;
    }
  }
  S->tr_t = (int32_t*)malloc(sizeof(int32_t) * (S->nt > 0 ? S->nt : 1));
  S->tr_nk = (int32_t*)malloc(sizeof(int32_t) * (S->nt > 0 ? S->nt : 1));
  S->tr_min = (int32_t*)malloc(sizeof(int32_t) * (S->nt > 0 ? S->nt : 1));
  S->ntr = 0;
  for (int64_t t = 0; t < S->nt; ++t) {
    if (!S->t_ok[t] || S->t_nhits[t] < cx->nmin) continue;
    const uint64_t key = tracklet_key(S, t);
    int kept = 0;
    int32_t mn = INT32_MAX;
    for (int r = 0; r < NROW; ++r) {
      int32_t h = S->t_slots[t * NROW + r];
      if (h >= 0 && S->weight[h] == key) {
        ++kept;
        if (S->orig[h] < mn) mn = S->orig[h];
      }
    }
    if (kept >= cx->nmin && 2 * kept >= S->t_nhits[t]) {
      S->tr_t[S->ntr] = (int32_t)t;
      S->tr_nk[S->ntr] = kept;
      S->tr_min[S->ntr] = mn;
      S->ntr++;
    }
  }
}

static void free_sector(sector_t* S);

/* Step 6 alone, on tracklets given by the caller (for the pins of the selection rule): nt tracklets
 * of one sector, tracklet t with start-hit rank rank[t] (unique) and hit slots[t * NROW + r] (a hit
 * index in [0, n_hits) or -1) in row r. Out: accepted[t] (0/1), kept[t] (hits it keeps, 0 if not
 * accepted) and weight[h] (the largest key of a voting tracklet holding hit h, 0 if none). Returns 0,
 * or -1 for a malformed input. */
int ORACLE_SYM(select)(int32_t nmin, int64_t n_hits, int64_t nt, const int32_t* rank, const int32_t* slots,
                       int32_t* accepted, int32_t* kept, uint64_t* weight) {
  if (n_hits < 0 || nt < 0 || n_hits >= INT32_MAX) return -1;
  for (int64_t i = 0; i < nt * NROW; ++i)
    if (slots[i] < -1 || slots[i] >= n_hits) return -1;
  ctx_t cx;
  memset(&cx, 0, sizeof(cx));
  cx.nmin = nmin;
  sector_t S;
  memset(&S, 0, sizeof(S));
  S.n = n_hits;
  S.nt = nt;
  const int64_t ta = nt > 0 ? nt : 1;
  S.t_rank = (int32_t*)malloc(ta * sizeof(int32_t));
  S.t_nhits = (int32_t*)malloc(ta * sizeof(int32_t));
  S.t_ok = (int32_t*)malloc(ta * sizeof(int32_t));
  S.t_slots = (int32_t*)malloc(ta * NROW * sizeof(int32_t));
  S.orig = (int32_t*)malloc((n_hits > 0 ? n_hits : 1) * sizeof(int32_t));
  for (int64_t h = 0; h < n_hits; ++h) S.orig[h] = (int32_t)h;
  for (int64_t t = 0; t < nt; ++t) {
    int c = 0;
    for (int r = 0; r < NROW; ++r) {
      S.t_slots[t * NROW + r] = slots[t * NROW + r];
      c += slots[t * NROW + r] >= 0;
    }
    S.t_rank[t] = rank[t];
    S.t_nhits[t] = c;
    S.t_ok[t] = 1;
  }
  select_tracks(&cx, &S);
  for (int64_t t = 0; t < nt; ++t) { accepted[t] = 0; kept[t] = 0; }
  for (int64_t k = 0; k < S.ntr; ++k) {
    accepted[S.tr_t[k]] = 1;
    kept[S.tr_t[k]] = S.tr_nk[k];
  }
  for (int64_t h = 0; h < n_hits; ++h) weight[h] = S.weight[h];
  free_sector(&S);
  return 0;
}

static void track_sector(const ctx_t* cx, sector_t* S, int brute) {
  find_neighbours(cx, S, brute);
  clean_links(S);
  /* start hits: head of a cleaned chain of at least lmin hits */
  S->is_start = (uint8_t*)calloc(S->n > 0 ? S->n : 1, 1);
  for (int r = 1; r + 1 < NROW; ++r)
    for (int64_t i = S->row_start[r]; i < S->row_start[r + 1]; ++i) {
      if (!(S->upc[i] >= 0 && S->dnc[i] < 0)) continue;
      int len = 1;
      for (int64_t h = S->upc[i]; h >= 0 && len < cx->lmin; h = S->upc[h]) ++len;
      S->is_start[i] = len >= cx->lmin;
    }
  /* tracklets in start-hit (row, w, y, orig) order; built independently of each other */
  for (int r = 1; r + 1 < NROW; ++r)
    for (int64_t i = S->row_start[r]; i < S->row_start[r + 1]; ++i)
      if (S->is_start[i]) build_tracklet(cx, S, i, r);
  select_tracks(cx, S);
}

/* ------------------------------------------------------------------------------------------------
 * Step 9: merging of sector tracks across sector boundaries and a global refit without corrections
 * (Sec. 6: after the standalone sector tracking the tracks are refit; Table 1 of Sec. 7.2 times the
 * refit with its sorts as "Track Fit").
 *
 *   outer state  each sector track's fit (at x_ref) transported row by row, with the scattering
 *                noise of each row, to the row of its last hit;
 *   candidates   a track B in a phi-neighbouring sector of the same drift side whose reference row
 *                lies 1 .. merge_gap_rows rows above the last hit row of A, with
 *                |w_B(x_ref) - w_A(outer)| <= merge_dw;
 *   chi2         A's outer state rotated into B's frame (rotate_state) and carried by one helix step
 *                (one row of scattering noise) to B's x_ref; chi2 = d^T (C_A + C_B)^-1 d over the 5
 *                parameters (Cholesky); a candidate needs chi2 <= merge_chi2_max;
 *   matching     A's best candidate and B's best candidate (smallest chi2, tie: smaller index); A and
 *                B merge when each is the other's best; merged pairs chain inner to outer;
 *   refit        each chain (a single sector track is a chain of one) is refit over all its hits by
 *                the Kalman filter of step 5 in refit_passes passes (3), inward, outward, inward, each
 *                starting at the end hit of the previous one (the first at the outermost segment's
 *                outer state) from the previous state, its covariance multiplied by refit_scale (100:
 *                the previous pass's information counts 1%, while the state keeps the linearisation
 *                point; a reset to cov0 would let the first updates move the slope far from it), and
 *                updating with every hit in turn: row by row within a segment, rotated into the next
 *                hit's frame at a segment change and carried by one step to its row; no hit is
 *                rejected; a failed step ends the refit at the last updated hit. The result is the
 *                last pass's fit at the innermost hit, in its segment's frame, with that pass's chi2
 *                and hits.
 * Tracks never cross the central membrane in the workloads here (primaries from z = 0), so no A/C
 * pair is formed.
 * ---------------------------------------------------------------------------------------------- */

/* The state at x in the frame of angle alpha, expressed in the frame of angle alpha + d (cd = cos d,
 * sd = sin d): the point keeps its place, x' = x cd + y sd, y' = y cd - x sd, and the direction
 * angle drops by d. The covariance is carried at fixed x' to first order: a change dy at fixed x
 * moves the point off the line x' = const by sd dy, and the state is moved back along the track to
 * it, so dy' = (cos phi / cos phi') dy, dw' = -t sd / cos phi' dy, d sin phi' = -k sd dy +
 * (cos phi' / cos phi) d sin phi. Returns 1 if cos phi' <= 0 or |sin phi'| >= max_sin. */
static int rotate_state(const ctx_t* cx, real P[5], real C[5][5], real* x, real cd, real sd) {
  const real s = P[2];
  const real c = SQRT((real)1 - s * s);
  const real s1 = s * cd - c * sd;
  const real c1 = c * cd + s * sd;
  if (!(c1 > 0) || !(absr(s1) < cx->max_sin)) return 1;
  const real x1 = *x * cd + P[0] * sd;
  const real y1 = P[0] * cd - *x * sd;
  const real k = cx->kq * P[4];
  const real ic = (real)1 / c, ic1 = (real)1 / c1;
  real J[5][5];
  memset(J, 0, sizeof(J));
  for (int i = 0; i < 5; ++i) J[i][i] = 1;
  J[0][0] = QUO(c, c1, ic1);
  J[1][0] = -QUO(P[3] * sd, c1, ic1);
  J[2][0] = -(k * sd);
  J[2][2] = QUO(c1, c, ic);
  real T[5][5], O[5][5];
  mat_mul5(J, C, T);
  mat_mul5_bt(T, J, O);
  mirror_lower(O);
  memcpy(C, O, sizeof(O));
  P[0] = y1;
  P[2] = s1;
  *x = x1;
  return 0;
}

/* chi2 = d^T S^-1 d for a symmetric positive definite S (lower triangle used), by Cholesky
 * S = L L^T and forward substitution; +inf if S is not positive definite. */
static real chi2_5(real S[5][5], const real d[5]) {
  real L[5][5], z[5];
  memset(L, 0, sizeof(L));
  for (int j = 0; j < 5; ++j) {
    real acc = S[j][j];
    for (int k = 0; k < j; ++k) acc = FMA(-L[j][k], L[j][k], acc);
    if (!(acc > 0)) return (real)INFINITY;
    L[j][j] = SQRT(acc);
    const real il = (real)1 / L[j][j];
    for (int i = j + 1; i < 5; ++i) {
      real a = S[i][j];
      for (int k = 0; k < j; ++k) a = FMA(-L[i][k], L[j][k], a);
      L[i][j] = QUO(a, L[j][j], il);
    }
  }
  for (int i = 0; i < 5; ++i) {
    real acc = d[i];
    for (int k = 0; k < i; ++k) acc = FMA(-L[i][k], z[k], acc);
    z[i] = QUO(acc, L[i][i], (real)1 / L[i][i]);
  }
  real q = 0;
  for (int i = 0; i < 5; ++i) q = FMA(z[i], z[i], q);
  return q;
}

static void unpack_cov(const real* c15, real C[5][5]) {
  for (int i = 0, o = 0; i < 5; ++i)
    for (int k = 0; k <= i; ++k, ++o) C[i][k] = C[k][i] = c15[o];
}

/* the rotation from sector a's frame to the frame of its phi neighbour b: +20 degrees if b follows a
 * in phi, else -20 degrees */
static real rot_sign(int sa, int sb) { return ((sa % 18) + 1) % 18 == sb % 18 ? (real)1 : (real)-1; }

typedef struct { real w; int32_t t; } wkey;
static int cmp_wkey(const void* a, const void* b) {
  const wkey* x = (const wkey*)a;
  const wkey* y = (const wkey*)b;
  if (x->w < y->w) return -1;
  if (x->w > y->w) return 1;
  return (x->t > y->t) - (x->t < y->t);
}

static merge_out* merge_tracks(const ctx_t* cx, int64_t nt, const int32_t* sec, const int32_t* row_ref,
                               const real* P0, const real* C0, const int64_t* hoff, const int32_t* hits,
                               const uint8_t* crow, const real* cy, const real* cw, int brute) {
  merge_out* M = (merge_out*)calloc(1, sizeof(merge_out));
  const int64_t na = nt > 0 ? nt : 1;
  M->n_tracks = nt;
  real* PO = (real*)malloc(na * 5 * sizeof(real));
  real* CO = (real*)malloc(na * 25 * sizeof(real));
  int* has_out = (int*)calloc(na, sizeof(int));
  int* last_row = (int*)malloc(na * sizeof(int));
  M->tr_outer = (double*)malloc(na * 5 * sizeof(double));
  /* outer states */
  for (int64_t t = 0; t < nt; ++t) {
    last_row[t] = hoff[t + 1] > hoff[t] ? crow[hits[hoff[t + 1] - 1]] : row_ref[t];
    real P[5], C[5][5];
    memcpy(P, P0 + 5 * t, sizeof(P));
    unpack_cov(C0 + 15 * t, C);
    int ok = 1;
    for (int r = row_ref[t] + 1; r <= last_row[t] && ok; ++r)
      if (kf_propagate(cx, P, C, cx->x[r - 1], cx->x[r], NULL, NULL)) ok = 0;
    has_out[t] = ok;
    memcpy(PO + 5 * t, P, sizeof(P));
    memcpy(CO + 25 * t, C, sizeof(C));
    for (int i = 0; i < 5; ++i) M->tr_outer[5 * t + i] = ok ? (double)P[i] : NAN;
  }
  /* each sector's tracks ordered by w at x_ref, for the candidates' w window */
  int64_t cnt[NSEC + 1];
  memset(cnt, 0, sizeof(cnt));
  for (int64_t t = 0; t < nt; ++t) cnt[sec[t] + 1]++;
  for (int q = 0; q < NSEC; ++q) cnt[q + 1] += cnt[q];
  wkey* keys = (wkey*)malloc(na * sizeof(wkey));
  {
    int64_t fill[NSEC];
    for (int q = 0; q < NSEC; ++q) fill[q] = cnt[q];
    for (int64_t t = 0; t < nt; ++t) {
      keys[fill[sec[t]]].w = P0[5 * t + 1];
      keys[fill[sec[t]]++].t = (int32_t)t;
    }
    for (int q = 0; q < NSEC; ++q) qsort(keys + cnt[q], cnt[q + 1] - cnt[q], sizeof(wkey), cmp_wkey);
  }
  int32_t* bestB = (int32_t*)malloc(na * sizeof(int32_t));
  int32_t* bestA = (int32_t*)malloc(na * sizeof(int32_t));
  real* chiB = (real*)malloc(na * sizeof(real));
  real* chiA = (real*)malloc(na * sizeof(real));
  for (int64_t t = 0; t < nt; ++t) { bestB[t] = bestA[t] = -1; chiB[t] = chiA[t] = (real)INFINITY; }
  for (int64_t a = 0; a < nt; ++a) {
    if (!has_out[a]) continue;
    const int side = sec[a] / 18, ka = sec[a] % 18;
    const real wa = PO[5 * a + 1];
    for (int dir = -1; dir <= 1; dir += 2) {
      const int sb = side * 18 + (ka + dir + 18) % 18;
      /* the sector's tracks with w inside the window (widened by a hair; the exact test decides) */
      const real pad = absr(wa) * (real)1e-6 + (real)1e-6;
      const real lo = (wa - cx->merge_dw) - pad;
      int64_t i0 = cnt[sb], i1 = cnt[sb + 1];
      while (!brute && i0 < i1) {
        const int64_t mid = i0 + (i1 - i0) / 2;
        if (keys[mid].w < lo) i0 = mid + 1; else i1 = mid;
      }
      if (brute) i0 = cnt[sb];
      for (int64_t i = i0; i < cnt[sb + 1] && (brute || keys[i].w <= (wa + cx->merge_dw) + pad); ++i) {
        const int64_t b = keys[i].t;
        const int g = row_ref[b] - last_row[a];
        if (g < 1 || g > cx->merge_gap_rows) continue;
        if (!(absr(P0[5 * b + 1] - wa) <= cx->merge_dw)) continue;
        real P[5], C[5][5], Cb[5][5], x = cx->x[last_row[a]];
        memcpy(P, PO + 5 * a, sizeof(P));
        memcpy(C, CO + 25 * a, sizeof(C));
        if (rotate_state(cx, P, C, &x, cx->rot_c, rot_sign(sec[a], sb) * cx->rot_s)) continue;
        if (kf_propagate(cx, P, C, x, cx->x[row_ref[b]], NULL, NULL)) continue;
        unpack_cov(C0 + 15 * b, Cb);
        real S[5][5], d[5];
        for (int r = 0; r < 5; ++r) {
          d[r] = P[r] - P0[5 * b + r];
          for (int q = 0; q < 5; ++q) S[r][q] = C[r][q] + Cb[r][q];
        }
        const real chi = chi2_5(S, d);
        if (!(chi <= cx->merge_chi2_max)) continue;
        if (chi < chiB[a] || (chi == chiB[a] && b < bestB[a])) { chiB[a] = chi; bestB[a] = (int32_t)b; }
        if (chi < chiA[b] || (chi == chiA[b] && a < bestA[b])) { chiA[b] = chi; bestA[b] = (int32_t)a; }
      }
    }
  }
  M->tr_next = (int32_t*)malloc(na * sizeof(int32_t));
  M->tr_merge_chi2 = (double*)malloc(na * sizeof(double));
  int32_t* prev = (int32_t*)malloc(na * sizeof(int32_t));
  for (int64_t t = 0; t < nt; ++t) { M->tr_next[t] = -1; prev[t] = -1; M->tr_merge_chi2[t] = NAN; }
  for (int64_t a = 0; a < nt; ++a) {
    const int32_t b = bestB[a];
    if (b >= 0 && bestA[b] == a) {
      M->tr_next[a] = b;
      prev[b] = (int32_t)a;
      M->tr_merge_chi2[a] = (double)chiB[a];
    }
  }
  /* chains and their refit */
  int64_t nm = 0, nh = 0;
  for (int64_t t = 0; t < nt; ++t)
    if (prev[t] < 0) ++nm;
  nh = nt > 0 ? hoff[nt] : 0;
  const int64_t ma = nm > 0 ? nm : 1;
  M->n_merged = nm;
  M->mt_head = (int32_t*)malloc(ma * sizeof(int32_t));
  M->mt_nseg = (int32_t*)malloc(ma * sizeof(int32_t));
  M->mt_sector = (int32_t*)malloc(ma * sizeof(int32_t));
  M->mt_ndf = (int32_t*)malloc(ma * sizeof(int32_t));
  M->mt_nfit = (int32_t*)malloc(ma * sizeof(int32_t));
  M->mt_xref = (double*)malloc(ma * sizeof(double));
  M->mt_param = (double*)malloc(ma * 5 * sizeof(double));
  M->mt_cov = (double*)malloc(ma * 15 * sizeof(double));
  M->mt_chi2 = (double*)malloc(ma * sizeof(double));
  M->mt_hit_off = (int64_t*)malloc((nm + 1) * sizeof(int64_t));
  M->mt_hits = (int32_t*)malloc((nh > 0 ? nh : 1) * sizeof(int32_t));
  M->mt_hit_off[0] = 0;
  int32_t* segs = (int32_t*)malloc(na * sizeof(int32_t));
  int64_t m = 0, oh = 0;
  for (int64_t h0 = 0; h0 < nt; ++h0) {
    if (prev[h0] >= 0) continue;
    int ns = 0;
    for (int32_t t = (int32_t)h0; t >= 0; t = M->tr_next[t]) {
      segs[ns++] = t;
      for (int64_t i = hoff[t]; i < hoff[t + 1]; ++i) M->mt_hits[oh++] = hits[i];
    }
    M->mt_head[m] = (int32_t)h0;
    M->mt_nseg[m] = ns;
    M->mt_hit_off[m + 1] = oh;
    /* refit: three passes over the chain's hits (inward, outward, inward), each from the previous
     * pass's end state with the covariance reset, starting from the outermost segment's outer state */
    const int32_t tm = segs[ns - 1];
    int nfit = 0;
    real chi2sum = 0, Pr[5], Cr[5][5], xr = 0;
    int sr = sec[h0];
    if (has_out[tm]) {
      int64_t nh_chain = 0;
      for (int j = 0; j < ns; ++j) nh_chain += hoff[segs[j] + 1] - hoff[segs[j]];
      int32_t* H = (int32_t*)malloc((nh_chain > 0 ? nh_chain : 1) * sizeof(int32_t));
      int32_t* Hs = (int32_t*)malloc((nh_chain > 0 ? nh_chain : 1) * sizeof(int32_t));
      int64_t q = 0;
      for (int j = 0; j < ns; ++j)
        for (int64_t i = hoff[segs[j]]; i < hoff[segs[j] + 1]; ++i) { H[q] = hits[i]; Hs[q++] = sec[segs[j]]; }
      real P[5], Cs[5][5];
      memcpy(P, PO + 5 * tm, sizeof(P));
      memcpy(Cs, CO + 25 * tm, sizeof(Cs));
      int ok = 1;
      for (int pass = 0; pass < cx->refit_passes && ok; ++pass) {
        const int inward = pass != 1;
        real C[5][5];
        for (int i = 0; i < 5; ++i)
          for (int k = 0; k < 5; ++k) C[i][k] = Cs[i][k] * cx->refit_scale;
        int cur_sec = inward ? Hs[nh_chain - 1] : Hs[0], cur_row = -2;
        real cur_x = 0;
        int n_pass = 0;
        real chi_pass = 0;
        for (int64_t k2 = 0; k2 < nh_chain; ++k2) {
          const int64_t i = inward ? nh_chain - 1 - k2 : k2;
          const int32_t hc = H[i];
          const int r = crow[hc];
          if (Hs[i] != cur_sec) {
            if (rotate_state(cx, P, C, &cur_x, cx->rot_c, rot_sign(cur_sec, Hs[i]) * cx->rot_s)) { ok = 0; break; }
            cur_sec = Hs[i];
            cur_row = -1;
          }
          if (cur_row == -1) {
            if (kf_propagate(cx, P, C, cur_x, cx->x[r], NULL, NULL)) { ok = 0; break; }
          } else if (cur_row >= 0) {
            int bad = 0;
            if (inward)
              for (int rr = cur_row - 1; rr >= r && !bad; --rr) bad = kf_propagate(cx, P, C, cx->x[rr + 1], cx->x[rr], NULL, NULL);
            else
              for (int rr = cur_row + 1; rr <= r && !bad; ++rr) bad = kf_propagate(cx, P, C, cx->x[rr - 1], cx->x[rr], NULL, NULL);
            if (bad) { ok = 0; break; }
          }
          cur_row = r;
          cur_x = cx->x[r];
          const real chi = kf_chi2(cx, P, C, cy[hc], cw[hc]);
          kf_update(cx, P, C, cy[hc], cw[hc]);
          chi_pass = chi_pass + chi;
          ++n_pass;
          memcpy(Pr, P, sizeof(Pr));
          memcpy(Cr, C, sizeof(Cr));
          xr = cur_x;
          sr = cur_sec;
        }
        nfit = n_pass;
        chi2sum = chi_pass;
        memcpy(Cs, Cr, sizeof(Cs));
      }
      free(H);
      free(Hs);
    }
    M->mt_nfit[m] = nfit;
    M->mt_ndf[m] = 2 * nfit - 5;
    M->mt_sector[m] = sr;
    M->mt_chi2[m] = nfit ? (double)chi2sum : NAN;
    M->mt_xref[m] = nfit ? (double)xr : NAN;
    for (int i = 0; i < 5; ++i) M->mt_param[5 * m + i] = nfit ? (double)Pr[i] : NAN;
    for (int i = 0, o = 0; i < 5; ++i)
      for (int k = 0; k <= i; ++k, ++o) M->mt_cov[15 * m + o] = nfit ? (double)Cr[i][k] : NAN;
    ++m;
  }
  free(PO); free(CO); free(has_out); free(last_row); free(keys); free(bestB); free(bestA); free(chiB);
  free(chiA); free(prev); free(segs);
  return M;
}

void ORACLE_SYM(free_merge)(merge_out* M) {
  if (!M) return;
  free(M->mt_head); free(M->mt_nseg); free(M->mt_sector); free(M->mt_ndf); free(M->mt_nfit); free(M->mt_xref);
  free(M->mt_param); free(M->mt_cov); free(M->mt_chi2); free(M->mt_hit_off); free(M->mt_hits); free(M->tr_next);
  free(M->tr_merge_chi2); free(M->tr_outer);
  free(M);
}

/* Step 9 alone on caller-given sector tracks (for the pins): nt tracks with sector, the row of
 * x_ref, the fit (param [nt][5], cov [nt][15]) and kept hits (hit_off, hits: cluster indices,
 * ascending row); the clusters' rows and (y, w), rounded to REAL on entry. brute = 1 tests every track of
 * a neighbouring sector instead of the w-ordered window. Returns 0 or -1. */
int ORACLE_SYM(merge)(const oracle_params* p, int64_t n, const uint8_t* row, const double* y, const double* w,
                      int64_t nt, const int32_t* sector, const int32_t* row_ref, const double* param,
                      const double* cov, const int64_t* hit_off, const int32_t* hits, int brute, merge_out** out) {
  *out = NULL;
  if (n < 0 || nt < 0) return -1;
  for (int64_t t = 0; t < nt; ++t) {
    if (sector[t] < 0 || sector[t] >= NSEC || row_ref[t] < 0 || row_ref[t] >= NROW || hit_off[t + 1] < hit_off[t])
      return -1;
    for (int64_t i = hit_off[t]; i < hit_off[t + 1]; ++i)
      if (hits[i] < 0 || hits[i] >= n) return -1;
  }
  ctx_t cx;
  make_ctx(p, &cx);
  const int64_t na = n > 0 ? n : 1, ta = nt > 0 ? nt : 1;
  real* cy = (real*)malloc(na * sizeof(real));
  real* cw = (real*)malloc(na * sizeof(real));
  real* P = (real*)malloc(ta * 5 * sizeof(real));
  real* C = (real*)malloc(ta * 15 * sizeof(real));
  for (int64_t i = 0; i < n; ++i) { cy[i] = (real)y[i]; cw[i] = (real)w[i]; }
  for (int64_t i = 0; i < nt * 5; ++i) P[i] = (real)param[i];
  for (int64_t i = 0; i < nt * 15; ++i) C[i] = (real)cov[i];
  *out = merge_tracks(&cx, nt, sector, row_ref, P, C, hit_off, hits, row, cy, cw, brute);
  free(cy); free(cw); free(P); free(C);
  return 0;
}

/* one rotation (for the pins): the state P, C (full 5x5) at x in sector sa's frame into the frame of
 * its phi neighbour sb; returns 0 and the new x, or 1 */
int ORACLE_SYM(rotate)(const oracle_params* p, double* P, double* C, double* x, int sa, int sb) {
  ctx_t cx;
  make_ctx(p, &cx);
  real Pr[5], Cr[5][5], xr = (real)*x;
  for (int i = 0; i < 5; ++i) Pr[i] = (real)P[i];
  for (int i = 0; i < 25; ++i) Cr[i / 5][i % 5] = (real)C[i];
  const int rc = rotate_state(&cx, Pr, Cr, &xr, cx.rot_c, rot_sign(sa, sb) * cx.rot_s);
  for (int i = 0; i < 5; ++i) P[i] = Pr[i];
  for (int i = 0; i < 25; ++i) C[i] = Cr[i / 5][i % 5];
  *x = xr;
  return rc;
}

void ORACLE_SYM(free_result)(oracle_result* R) {
  if (!R) return;
  free(R->up); free(R->down); free(R->up_c); free(R->down_c); free(R->nb_margin); free(R->start);
  free(R->tl_sector); free(R->tl_start); free(R->tl_nhits); free(R->tl_ndf); free(R->tl_row_ref);
  free(R->tl_row_top); free(R->tl_ok); free(R->tl_xref); free(R->tl_param); free(R->tl_cov);
  free(R->tl_chi2); free(R->tl_margin); free(R->tl_hit_off); free(R->tl_hits);
  free(R->tr_sector); free(R->tr_ndf); free(R->tr_nhits); free(R->tr_tracklet); free(R->tr_xref);
  free(R->tr_param); free(R->tr_cov); free(R->tr_chi2); free(R->tr_hit_off); free(R->tr_hits);
  free(R->tr_beam); free(R->tr_res); free(R->tr_npred); free(R->keep);
  ORACLE_SYM(free_merge)(R->merged);
  free(R);
}

static void free_sector(sector_t* S) {
  free(S->orig); free(S->y); free(S->w); free(S->up); free(S->dn); free(S->upc); free(S->dnc);
  free(S->nbm); free(S->t_start); free(S->t_rank); free(S->t_nhits); free(S->t_ndf); free(S->t_rref); free(S->t_rtop);
  free(S->t_ok); free(S->t_x); free(S->t_p); free(S->t_c); free(S->t_chi2); free(S->t_m);
  free(S->t_slots); free(S->tr_t); free(S->tr_nk); free(S->tr_min); free(S->weight); free(S->is_start);
}

/* Track one frame. Inputs: n clusters in caller order (sector, row, y, w); y and w are given in
 * double and rounded to REAL on entry. flags: ORACLE_PACKED reads them back through the 16-bit
 * storage format first; ORACLE_BRUTE_FORCE scans whole rows in the neighbour
 * search instead of the sorted-w index. n_threads > 0 runs sectors in parallel (sectors are
 * independent). Returns 0, or -1 for malformed input, -2 for allocation failure. */
int ORACLE_SYM(track)(const oracle_params* p, int64_t n, const uint8_t* sector, const uint8_t* row,
                      const double* y, const double* w, int flags, int n_threads,
                      oracle_result** out) {
  *out = NULL;
  if (n < 0 || n >= INT32_MAX) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (sector[i] >= NSEC || row[i] >= NROW || !isfinite(y[i]) || !isfinite(w[i])) return -1;
  ctx_t cx;
  make_ctx(p, &cx);
  sector_t* secs = (sector_t*)calloc(NSEC, sizeof(sector_t));
  /* group by sector and row; rows sorted by (w, orig) */
  int64_t cnt[NSEC][NROW];
  memset(cnt, 0, sizeof(cnt));
  for (int64_t i = 0; i < n; ++i) cnt[sector[i]][row[i]]++;
  for (int s = 0; s < NSEC; ++s) {
    sector_t* S = &secs[s];
    S->row_start[0] = 0;
    for (int r = 0; r < NROW; ++r) S->row_start[r + 1] = S->row_start[r] + cnt[s][r];
    S->n = S->row_start[NROW];
    int64_t na = S->n > 0 ? S->n : 1;
    S->orig = malloc(na * sizeof(int32_t));
    S->y = malloc(na * sizeof(real)); S->w = malloc(na * sizeof(real));
    S->up = malloc(na * sizeof(int32_t)); S->dn = malloc(na * sizeof(int32_t));
    S->upc = malloc(na * sizeof(int32_t)); S->dnc = malloc(na * sizeof(int32_t));
    S->nbm = malloc(na * sizeof(double));
  }
  {
    int64_t fill[NSEC][NROW];
    for (int s = 0; s < NSEC; ++s)
      for (int r = 0; r < NROW; ++r) fill[s][r] = secs[s].row_start[r];
    for (int64_t i = 0; i < n; ++i) {
      sector_t* S = &secs[sector[i]];
      int64_t o = fill[sector[i]][row[i]]++;
      S->orig[o] = (int32_t)i; S->y[o] = (real)y[i]; S->w[o] = (real)w[i];
      if (flags & ORACLE_PACKED) pack_roundtrip(&S->y[o], &S->w[o]);
    }
  }
  /* the tracker's view of every cluster, kept for step 9's refit */
  real *cy = NULL, *cw = NULL;
  if (flags & ORACLE_MERGE) {
    cy = (real*)malloc((n > 0 ? n : 1) * sizeof(real));
    cw = (real*)malloc((n > 0 ? n : 1) * sizeof(real));
    for (int64_t i = 0; i < n; ++i) {
      cy[i] = (real)y[i];
      cw[i] = (real)w[i];
      if (flags & ORACLE_PACKED) pack_roundtrip(&cy[i], &cw[i]);
    }
  }
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int s = 0; s < NSEC; ++s) {
    sector_t* S = &secs[s];
    for (int r = 0; r < NROW; ++r) {
      int64_t b = S->row_start[r], m = S->row_start[r + 1] - b;
      if (m < 2) continue;
      rowhit* tmp = (rowhit*)malloc(m * sizeof(rowhit));
      for (int64_t j = 0; j < m; ++j) { tmp[j].w = S->w[b + j]; tmp[j].orig = S->orig[b + j]; tmp[j].y = S->y[b + j]; }
      qsort(tmp, m, sizeof(rowhit), cmp_rowhit);
      for (int64_t j = 0; j < m; ++j) { S->w[b + j] = tmp[j].w; S->orig[b + j] = tmp[j].orig; S->y[b + j] = tmp[j].y; }
      free(tmp);
    }
    track_sector(&cx, S, flags & ORACLE_BRUTE_FORCE);
  }
  /* gather results */
  oracle_result* R = (oracle_result*)calloc(1, sizeof(oracle_result));
  int64_t na = n > 0 ? n : 1;
  R->n_clusters = n;
  R->up = malloc(na * sizeof(int32_t)); R->down = malloc(na * sizeof(int32_t));
  R->up_c = malloc(na * sizeof(int32_t)); R->down_c = malloc(na * sizeof(int32_t));
  R->nb_margin = malloc(na * sizeof(double));
  int64_t nt = 0, ntr = 0, nhl = 0, nhr = 0;
  for (int s = 0; s < NSEC; ++s) {
    sector_t* S = &secs[s];
    for (int64_t i = 0; i < S->n; ++i) {
      int32_t o = S->orig[i];
      R->up[o] = S->up[i] >= 0 ? S->orig[S->up[i]] : -1;
      R->down[o] = S->dn[i] >= 0 ? S->orig[S->dn[i]] : -1;
      R->up_c[o] = S->upc[i] >= 0 ? S->orig[S->upc[i]] : -1;
      R->down_c[o] = S->dnc[i] >= 0 ? S->orig[S->dnc[i]] : -1;
      R->nb_margin[o] = S->nbm[i];
    }
    nt += S->nt;
    ntr += S->ntr;
    for (int64_t t = 0; t < S->nt; ++t) nhl += S->t_ok[t] ? S->t_nhits[t] : 0;
    for (int64_t k = 0; k < S->ntr; ++k) nhr += S->tr_nk[k];
  }
  R->n_start = nt;
  R->n_tracklets = nt;
  int64_t ta = nt > 0 ? nt : 1, ra = ntr > 0 ? ntr : 1;
  R->start = malloc(ta * sizeof(int32_t));
  R->tl_sector = malloc(ta * sizeof(int32_t)); R->tl_start = malloc(ta * sizeof(int32_t));
  R->tl_nhits = malloc(ta * sizeof(int32_t)); R->tl_ndf = malloc(ta * sizeof(int32_t));
  R->tl_row_ref = malloc(ta * sizeof(int32_t)); R->tl_row_top = malloc(ta * sizeof(int32_t));
  R->tl_ok = malloc(ta * sizeof(int32_t));
  R->tl_xref = malloc(ta * sizeof(double)); R->tl_param = malloc(ta * 5 * sizeof(double));
  R->tl_cov = malloc(ta * 15 * sizeof(double)); R->tl_chi2 = malloc(ta * sizeof(double));
  R->tl_margin = malloc(ta * sizeof(double));
  R->tl_hit_off = malloc((nt + 1) * sizeof(int64_t));
  R->tl_hits = malloc((nhl > 0 ? nhl : 1) * sizeof(int32_t));
  R->n_tracks = ntr;
  R->tr_sector = malloc(ra * sizeof(int32_t)); R->tr_ndf = malloc(ra * sizeof(int32_t));
  R->tr_nhits = malloc(ra * sizeof(int32_t)); R->tr_tracklet = malloc(ra * sizeof(int32_t));
  R->tr_xref = malloc(ra * sizeof(double)); R->tr_param = malloc(ra * 5 * sizeof(double));
  R->tr_cov = malloc(ra * 15 * sizeof(double)); R->tr_chi2 = malloc(ra * sizeof(double));
  R->tr_beam = malloc(ra * 5 * sizeof(double));
  R->tr_npred = malloc(ra * sizeof(int32_t));
  R->tr_res = malloc((nhr > 0 ? nhr : 1) * 2 * sizeof(int32_t));
  R->keep = calloc(na, 1);
  R->tr_hit_off = malloc((ntr + 1) * sizeof(int64_t));
  R->tr_hits = malloc((nhr > 0 ? nhr : 1) * sizeof(int32_t));
  int64_t ot = 0, otr = 0, ohl = 0, ohr = 0;
  R->tl_hit_off[0] = 0;
  R->tr_hit_off[0] = 0;
  for (int s = 0; s < NSEC; ++s) {
    sector_t* S = &secs[s];
    /* tracklets and tracks are already in canonical order: the rank of the start hit (the
     * hit's position in the sector ordered by row, w, y, input index) */
    int32_t* ti = malloc((S->nt > 0 ? S->nt : 1) * sizeof(int32_t));
    for (int64_t t = 0; t < S->nt; ++t) ti[t] = (int32_t)t;
    int32_t* tpos = malloc((S->nt > 0 ? S->nt : 1) * sizeof(int32_t));
    for (int64_t j = 0; j < S->nt; ++j) {
      int64_t t = ti[j];
      tpos[t] = (int32_t)(ot);
      R->start[ot] = S->t_start[t];
      R->tl_sector[ot] = s; R->tl_start[ot] = S->t_start[t]; R->tl_nhits[ot] = S->t_nhits[t];
      R->tl_ndf[ot] = S->t_ndf[t]; R->tl_row_ref[ot] = S->t_rref[t]; R->tl_row_top[ot] = S->t_rtop[t];
      R->tl_ok[ot] = S->t_ok[t]; R->tl_xref[ot] = S->t_x[t]; R->tl_chi2[ot] = S->t_chi2[t];
      R->tl_margin[ot] = S->t_m[t];
      for (int i = 0; i < 5; ++i) R->tl_param[ot * 5 + i] = S->t_p[t * 5 + i];
      for (int i = 0; i < 15; ++i) R->tl_cov[ot * 15 + i] = S->t_c[t * 15 + i];
      if (S->t_ok[t])
        for (int r = 0; r < NROW; ++r) {
          int32_t h = S->t_slots[t * NROW + r];
          if (h >= 0) R->tl_hits[ohl++] = S->orig[h];
        }
      R->tl_hit_off[ot + 1] = ohl;
      ++ot;
    }
    int32_t* ki = malloc((S->ntr > 0 ? S->ntr : 1) * sizeof(int32_t));
    for (int64_t k = 0; k < S->ntr; ++k) ki[k] = (int32_t)k;
    uint8_t* keep_local = calloc(S->n > 0 ? S->n : 1, 1);
    for (int64_t j = 0; j < S->ntr; ++j) {
      int64_t k = ki[j], t = S->tr_t[k];
      const uint64_t key = tracklet_key(S, t);
      R->tr_sector[otr] = s; R->tr_ndf[otr] = S->t_ndf[t]; R->tr_nhits[otr] = S->tr_nk[k];
      R->tr_tracklet[otr] = tpos[t];
      R->tr_xref[otr] = S->t_x[t]; R->tr_chi2[otr] = S->t_chi2[t];
      for (int i = 0; i < 5; ++i) R->tr_param[otr * 5 + i] = S->t_p[t * 5 + i];
      for (int i = 0; i < 15; ++i) R->tr_cov[otr * 15 + i] = S->t_c[t * 15 + i];
      {
        real Pt[5], Ct[5][5], ob[5];
        for (int i = 0; i < 5; ++i) Pt[i] = S->t_p[t * 5 + i];
        for (int i = 0; i < 5; ++i)
          for (int k2 = 0; k2 <= i; ++k2) Ct[i][k2] = Ct[k2][i] = S->t_c[t * 15 + i * (i + 1) / 2 + k2];
        beamline(&cx, Pt, Ct, S->t_x[t], s, ob);
        for (int i = 0; i < 5; ++i) R->tr_beam[otr * 5 + i] = (double)ob[i];
      }
      compress_track(&cx, S, t, key, R->tr_res + 2 * ohr, &R->tr_npred[otr], keep_local);
      for (int r = 0; r < NROW; ++r) {
        int32_t h = S->t_slots[t * NROW + r];
        if (h >= 0 && S->weight[h] == key) R->tr_hits[ohr++] = S->orig[h];
      }
      R->tr_hit_off[otr + 1] = ohr;
      ++otr;
    }
    for (int64_t i = 0; i < S->n; ++i) R->keep[S->orig[i]] = keep_local[i];
    free(keep_local);
    free(ti); free(tpos); free(ki);
    free_sector(S);
  }
  free(secs);
  if (flags & ORACLE_MERGE) {
    const int64_t nt = R->n_tracks, ta = nt > 0 ? nt : 1;
    int32_t* rref = (int32_t*)malloc(ta * sizeof(int32_t));
    real* P = (real*)malloc(ta * 5 * sizeof(real));
    real* C = (real*)malloc(ta * 15 * sizeof(real));
    for (int64_t t = 0; t < nt; ++t) rref[t] = R->tl_row_ref[R->tr_tracklet[t]];
    for (int64_t i = 0; i < nt * 5; ++i) P[i] = (real)R->tr_param[i];
    for (int64_t i = 0; i < nt * 15; ++i) C[i] = (real)R->tr_cov[i];
    R->merged = merge_tracks(&cx, nt, R->tr_sector, rref, P, C, R->tr_hit_off, R->tr_hits, row, cy, cw,
                             flags & ORACLE_BRUTE_FORCE);
    free(rref); free(P); free(C); free(cy); free(cw);
  }
  *out = R;
  return 0;
}
