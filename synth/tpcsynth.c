/*
 * tpcsynth.c — seeded synthetic TPC time frames (input generator).
 *
 * This module produces inputs only. It holds none of the tracker's arithmetic and is shared by the
 * CPU oracle tests and the CUDA path alike. It models the workloads of the paper's synchronous
 * reconstruction (Sec. 2: continuous readout, clusters in native row/time coordinates; Sec. 7.1:
 * time frames of many overlapping collisions) with the detector layout of the Pb-Pb/pp configurations
 * used throughout this project: 36 sectors of 20 degrees (18 in phi x 2 drift sides), 152 pad rows
 * at radii 85-245 cm, 250 cm drift length, solenoid field Bz along +z.
 *
 * Physics model (all in double precision):
 *   - primaries from the origin; pT log-uniform, |eta| uniform below eta_max, phi uniform, q = +-1;
 *   - exact helix in the solenoid field: d(phi)/ds = k = -0.0029979246 * Bz * q / pT  [1/cm];
 *   - one cluster per crossed pad row on the first outgoing leg (loopers are not followed);
 *   - continuous readout: the cluster's drift coordinate is w = v_d * t_coll + (250 - |z|) with
 *     v_d = 250 cm / 90 us; clusters arriving after the frame end are lost (Sec. 2);
 *   - multiple scattering: Highland kick at every row with x/X0 = x0_total/152 per row (scaled by
 *     the path length through the row), log term at the nominal per-row thickness;
 *   - Gaussian smearing (sigma_y, sigma_w), row-crossing inefficiency, and uniform noise clusters.
 *
 * Random numbers: counter-based SplitMix64 streams keyed by (seed, frame, kind, id), so results do
 * not depend on thread count or scheduling.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SY_NSEC_PHI 18
#define SY_NSEC 36
#define SY_NROW 152
#define SY_PI 3.14159265358979323846
#define SY_VDRIFT (250.0 / 90.0) /* cm per microsecond */
#define SY_ZMAX 250.0
#define SY_PION_MASS 0.13957039
#define SY_CHUNK 512

typedef struct {
  uint64_t seed;
  uint64_t frame_id;
  int32_t n_collisions;  /* >= 0: fixed count; < 0: Poisson(poisson_mean) */
  double poisson_mean;
  int32_t mult_fixed;    /* > 0: fixed multiplicity per collision */
  double mult_mean;      /* otherwise exponential with this mean ... */
  int32_t mult_cap;      /* ... capped here */
  double pt_min, pt_max, eta_max;
  double bz;             /* tesla */
  double sigma_y, sigma_w;
  double dropout;        /* probability to lose a row crossing */
  double noise_frac;     /* noise clusters per signal cluster in each (sector,row) */
  double x0_total;       /* total X/X0 over the 152 rows; 0 disables scattering */
  double frame_us;       /* collision window: collision times uniform in [0, frame_us) */
  double tail_us;        /* readout continues this long after the window; later clusters are lost */
  int32_t t_zero;        /* 1: every collision at t = 0 */
  int32_t shuffle;       /* 1: emit clusters in a seeded random order */
  int32_t want_truth;    /* 1: fill per-cluster truth */
  int32_t n_threads;     /* 0: OpenMP default */
} synth_params;

typedef struct {
  int64_t n_clusters, n_tracks, n_collisions;
  uint8_t* sector;
  uint8_t* row;
  float* y;
  float* w;
  int32_t* truth_track;   /* -1 for noise; may be NULL */
  double* truth_state;    /* [n][5]: y, w, sin(phi_local), dw/ds, q/pT at the crossing; may be NULL */
  /* per track */
  int32_t* trk_coll;
  int8_t* trk_q;
  double* trk_pt;
  double* trk_eta;
  double* trk_phi0;
  double* trk_tc;          /* collision time, us */
  int32_t* trk_ncl;
  double* coll_tc;
} synth_frame;

/* ---------------------------------------------------------------- RNG (SplitMix64) */
static inline uint64_t sy_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
typedef struct { uint64_t s; } sy_rng;
enum { SY_K_EVENT = 1, SY_K_TRACK = 2, SY_K_NOISE = 3, SY_K_SHUFFLE = 4 };
static sy_rng sy_stream(const synth_params* p, uint64_t kind, uint64_t id) {
  sy_rng r;
  r.s = sy_mix(p->seed * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL) ^
        sy_mix(p->frame_id + 0xD1B54A32D192ED03ULL) ^ sy_mix((kind << 58) ^ (id + 1));
  return r;
}
static inline uint64_t sy_next(sy_rng* r) {
  r->s += 0x9E3779B97F4A7C15ULL;
  return sy_mix(r->s);
}
static inline double sy_u01(sy_rng* r) { return (double)(sy_next(r) >> 11) * 0x1.0p-53; }
static inline double sy_gauss(sy_rng* r) {
  double u1 = 1.0 - sy_u01(r); /* (0,1] */
  double u2 = sy_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * SY_PI * u2);
}
static int sy_poisson(sy_rng* r, double lam) {
  double L = exp(-lam), prod = sy_u01(r);
  int n = 0;
  while (prod > L) { ++n; prod *= sy_u01(r); }
  return n;
}

/* ---------------------------------------------------------------- geometry */
static inline double sy_row_x(int r) { return 85.0 + (double)r * (160.0 / 151.0); }
static inline double sy_alpha(int k) { return ((double)k + 0.5) * (SY_PI / 9.0); }
static inline double sy_wrap(double a) { /* into (-pi, pi] */
  a = fmod(a, 2.0 * SY_PI);
  if (a > SY_PI) a -= 2.0 * SY_PI;
  if (a <= -SY_PI) a += 2.0 * SY_PI;
  return a;
}

typedef struct {
  uint8_t sector, row;
  float y, w;
  int32_t track;
  double truth[5];
} sy_rec;

typedef struct {
  double phi0, eta, pt, tc;
  int q, coll;
} sy_track;

/* compact per-cluster record kept per chunk until the frame is assembled (truth kept apart) */
typedef struct {
  float y, w;
  int32_t track;
  uint8_t sector, row;
} sy_crec;

/* Propagate one primary and emit its clusters into out[] (<= SY_NROW records). */
static int sy_track_clusters(const synth_params* p, const sy_track* t, int64_t tid, sy_rec* out) {
  sy_rng rng = sy_stream(p, SY_K_TRACK, (uint64_t)tid);
  const double kappa = 0.0029979246 * p->bz;
  const double tan10 = tan(10.0 * SY_PI / 180.0);
  const double w_end = SY_VDRIFT * (p->frame_us + p->tail_us);
  const double xx0_row = p->x0_total / (double)SY_NROW;
  const double hl_log = xx0_row > 0 ? (1.0 + 0.038 * log(xx0_row)) : 1.0;
  double px = 0, py = 0, pz = 0, phi = t->phi0, tgl = sinh(t->eta), pt = t->pt;
  const double ptot = pt * sqrt(1.0 + tgl * tgl);
  const int q = t->q;
  const int side = t->eta >= 0 ? 0 : 1;
  double s_total = 0;
  int sec = -1, n = 0;
  for (int r = 0; r < SY_NROW; ++r) {
    const double X = sy_row_x(r);
    const double k = -kappa * (double)q / pt;
    double best_s = INFINITY;
    int best_k = -1;
    double bx = 0, by = 0, bphi = 0;
    int ncand = sec < 0 ? SY_NSEC_PHI : 3;
    for (int c = 0; c < ncand; ++c) {
      int kk = sec < 0 ? c : (sec + c - 1 + SY_NSEC_PHI) % SY_NSEC_PHI;
      double al = sy_alpha(kk), ux = cos(al), uy = sin(al);
      double d = X - (px * ux + py * uy);
      double psi = sy_wrap(phi - al);
      double s;
      if (fabs(k) < 1e-12) {
        double cp = cos(psi);
        if (cp <= 1e-12) continue;
        s = d / cp;
      } else {
        double sig = sin(psi) + k * d;
        if (fabs(sig) >= 1.0) continue;
        double ang = asin(sig) - psi; /* k*s must equal ang modulo 2 pi */
        if (k > 0) {
          while (ang <= 1e-13) ang += 2.0 * SY_PI;
          while (ang > 2.0 * SY_PI + 1e-13) ang -= 2.0 * SY_PI;
        } else {
          while (ang >= -1e-13) ang -= 2.0 * SY_PI;
          while (ang < -2.0 * SY_PI - 1e-13) ang += 2.0 * SY_PI;
        }
        s = ang / k;
        if ((s_total + s) * fabs(k) >= SY_PI) continue; /* beyond the first outgoing leg */
      }
      if (!(s > 1e-9) || s >= best_s) continue;
      double nx, ny, nphi;
      if (fabs(k) < 1e-12) {
        nx = px + s * cos(phi);
        ny = py + s * sin(phi);
        nphi = phi;
      } else {
        nphi = phi + k * s;
        nx = px + (sin(nphi) - sin(phi)) / k;
        ny = py - (cos(nphi) - cos(phi)) / k;
      }
      double yl = -nx * uy + ny * ux;
      if (fabs(yl) > X * tan10) continue;
      best_s = s; best_k = kk; bx = nx; by = ny; bphi = nphi;
    }
    if (best_k < 0) break;
    px = bx; py = by; phi = bphi;
    pz += tgl * best_s;
    s_total += best_s;
    sec = best_k;
    if (fabs(pz) > SY_ZMAX) break;
    if ((side == 0 && pz < 0) || (side == 1 && pz > 0)) break; /* crossed the central membrane */
    const double al = sy_alpha(sec), ux = cos(al), uy = sin(al);
    const double yl = -px * uy + py * ux;
    const double w_true = SY_VDRIFT * t->tc + (SY_ZMAX - fabs(pz));
    const double psi_loc = phi - al;
    const double tw = -fabs(tgl);
    const int lost = sy_u01(&rng) < p->dropout;
    const double gy = sy_gauss(&rng), gw = sy_gauss(&rng);
    if (!lost && w_true <= w_end) {
      sy_rec* o = &out[n++];
      o->sector = (uint8_t)(sec + SY_NSEC_PHI * side);
      o->row = (uint8_t)r;
      o->y = (float)(yl + p->sigma_y * gy);
      o->w = (float)(w_true + p->sigma_w * gw);
      o->track = (int32_t)tid;
      o->truth[0] = yl;
      o->truth[1] = w_true;
      o->truth[2] = sin(psi_loc);
      o->truth[3] = tw;
      o->truth[4] = (double)q / pt;
    }
    if (xx0_row > 0) {
      double lam = atan(tgl);
      double cosloc = cos(psi_loc) * cos(lam);
      if (cosloc < 0.05) cosloc = 0.05;
      double xx0 = xx0_row / cosloc;
      double beta = ptot / sqrt(ptot * ptot + SY_PION_MASS * SY_PION_MASS);
      double th0 = 0.0136 / (beta * ptot) * sqrt(xx0) * hl_log;
      double t1 = th0 * sy_gauss(&rng), t2 = th0 * sy_gauss(&rng);
      phi += t1 / cos(lam);
      lam += t2;
      if (fabs(lam) > 1.4) break;
      tgl = tan(lam);
      pt = ptot * cos(lam);
    }
  }
  return n;
}

static void sy_free_frame(synth_frame* f) {
  if (!f) return;
  free(f->sector); free(f->row); free(f->y); free(f->w); free(f->truth_track); free(f->truth_state);
  free(f->trk_coll); free(f->trk_q); free(f->trk_pt); free(f->trk_eta); free(f->trk_phi0);
  free(f->trk_tc); free(f->trk_ncl); free(f->coll_tc);
  free(f);
}

void synth_free(synth_frame* f) { sy_free_frame(f); }

/* Returns 0 and a frame in *out, or a negative value on allocation failure / bad parameters. */
int synth_generate(const synth_params* p, synth_frame** out) {
  *out = NULL;
  if (!p || p->pt_min <= 0 || p->pt_max < p->pt_min || p->frame_us < 0) return -1;
  synth_frame* f = (synth_frame*)calloc(1, sizeof(synth_frame));
  if (!f) return -2;
  /* collisions */
  sy_rng ev = sy_stream(p, SY_K_EVENT, 0);
  int ncoll = p->n_collisions >= 0 ? p->n_collisions : sy_poisson(&ev, p->poisson_mean);
  f->n_collisions = ncoll;
  f->coll_tc = (double*)malloc(sizeof(double) * (ncoll > 0 ? ncoll : 1));
  int* mult = (int*)malloc(sizeof(int) * (ncoll > 0 ? ncoll : 1));
  int64_t ntrk = 0;
  for (int c = 0; c < ncoll; ++c) {
    f->coll_tc[c] = p->t_zero ? 0.0 : sy_u01(&ev) * p->frame_us;
    int m;
    if (p->mult_fixed > 0) m = p->mult_fixed;
    else {
      double x = -p->mult_mean * log(1.0 - sy_u01(&ev));
      m = (int)ceil(x);
      if (m < 1) m = 1;
      if (m > p->mult_cap) m = p->mult_cap;
    }
    mult[c] = m;
    ntrk += m;
  }
  f->n_tracks = ntrk;
  sy_track* trk = (sy_track*)malloc(sizeof(sy_track) * (ntrk > 0 ? ntrk : 1));
  f->trk_coll = (int32_t*)malloc(sizeof(int32_t) * (ntrk > 0 ? ntrk : 1));
  f->trk_q = (int8_t*)malloc(ntrk > 0 ? ntrk : 1);
  f->trk_pt = (double*)malloc(sizeof(double) * (ntrk > 0 ? ntrk : 1));
  f->trk_eta = (double*)malloc(sizeof(double) * (ntrk > 0 ? ntrk : 1));
  f->trk_phi0 = (double*)malloc(sizeof(double) * (ntrk > 0 ? ntrk : 1));
  f->trk_tc = (double*)malloc(sizeof(double) * (ntrk > 0 ? ntrk : 1));
  f->trk_ncl = (int32_t*)calloc(ntrk > 0 ? ntrk : 1, sizeof(int32_t));
  {
    int64_t t = 0;
    const double lr = log(p->pt_max / p->pt_min);
    for (int c = 0; c < ncoll; ++c)
      for (int i = 0; i < mult[c]; ++i, ++t) {
        sy_rng tr = sy_stream(p, SY_K_TRACK + 16, (uint64_t)t);
        trk[t].phi0 = 2.0 * SY_PI * sy_u01(&tr);
        trk[t].eta = p->eta_max * (2.0 * sy_u01(&tr) - 1.0);
        trk[t].pt = p->pt_min * exp(lr * sy_u01(&tr));
        trk[t].q = sy_u01(&tr) < 0.5 ? -1 : 1;
        trk[t].tc = f->coll_tc[c];
        trk[t].coll = c;
        f->trk_coll[t] = c; f->trk_q[t] = (int8_t)trk[t].q; f->trk_pt[t] = trk[t].pt;
        f->trk_eta[t] = trk[t].eta; f->trk_phi0[t] = trk[t].phi0; f->trk_tc[t] = trk[t].tc;
      }
  }
  free(mult);
  /* signal clusters, in chunks of tracks (deterministic order) */
  int64_t nchunk = (ntrk + SY_CHUNK - 1) / SY_CHUNK;
  sy_crec** cbuf = (sy_crec**)calloc(nchunk > 0 ? nchunk : 1, sizeof(sy_crec*));
  double** tbuf = (double**)calloc(nchunk > 0 ? nchunk : 1, sizeof(double*));
  int64_t* ccnt = (int64_t*)calloc(nchunk + 1, sizeof(int64_t));
  int fail = 0;
  if (p->n_threads > 0) {
#ifdef _OPENMP
    omp_set_num_threads(p->n_threads);
#endif
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nchunk; ++c) {
    int64_t t0 = c * SY_CHUNK, t1 = t0 + SY_CHUNK < ntrk ? t0 + SY_CHUNK : ntrk;
    sy_rec* b = (sy_rec*)malloc(sizeof(sy_rec) * (size_t)(t1 - t0) * SY_NROW);
    if (!b) { fail = 1; continue; }
    int64_t n = 0;
    for (int64_t t = t0; t < t1; ++t) {
      int k = sy_track_clusters(p, &trk[t], t, b + n);
      f->trk_ncl[t] = k;
      n += k;
    }
    sy_crec* cb = (sy_crec*)malloc(sizeof(sy_crec) * (size_t)(n > 0 ? n : 1));
    double* tb = p->want_truth ? (double*)malloc(sizeof(double) * 5 * (size_t)(n > 0 ? n : 1)) : NULL;
    if (!cb || (p->want_truth && !tb)) { free(b); free(cb); free(tb); fail = 1; continue; }
    for (int64_t i = 0; i < n; ++i) {
      cb[i].y = b[i].y; cb[i].w = b[i].w; cb[i].track = b[i].track;
      cb[i].sector = b[i].sector; cb[i].row = b[i].row;
      if (tb) memcpy(&tb[5 * i], b[i].truth, 5 * sizeof(double));
    }
    free(b);
    cbuf[c] = cb;
    tbuf[c] = tb;
    ccnt[c] = n;
  }
  free(trk);
  if (fail) {
    for (int64_t c = 0; c < nchunk; ++c) { free(cbuf[c]); free(tbuf[c]); }
    free(cbuf); free(tbuf); free(ccnt); sy_free_frame(f); return -2;
  }
  int64_t nsig = 0;
  for (int64_t c = 0; c < nchunk; ++c) nsig += ccnt[c];
  /* per (sector,row) signal counts and the occupied w range for noise */
  int64_t cnt[SY_NSEC * SY_NROW];
  memset(cnt, 0, sizeof(cnt));
  double wlo = INFINITY, whi = -INFINITY;
  for (int64_t c = 0; c < nchunk; ++c)
    for (int64_t i = 0; i < ccnt[c]; ++i) {
      const sy_crec* r = &cbuf[c][i];
      cnt[r->sector * SY_NROW + r->row]++;
      if (r->w < wlo) wlo = r->w;
      if (r->w > whi) whi = r->w;
    }
  if (!(wlo <= whi)) { wlo = 0; whi = SY_ZMAX; }
  int64_t nnoise_sr[SY_NSEC * SY_NROW];
  int64_t nnoise = 0;
  for (int sr = 0; sr < SY_NSEC * SY_NROW; ++sr) {
    sy_rng nr = sy_stream(p, SY_K_NOISE, (uint64_t)sr);
    double x = p->noise_frac * (double)cnt[sr];
    int64_t k = (int64_t)floor(x);
    if (sy_u01(&nr) < x - (double)k) ++k;
    nnoise_sr[sr] = k;
    nnoise += k;
  }
  int64_t n = nsig + nnoise;
  f->n_clusters = n;
  size_t na = (size_t)(n > 0 ? n : 1);
  f->sector = (uint8_t*)malloc(na);
  f->row = (uint8_t*)malloc(na);
  f->y = (float*)malloc(na * sizeof(float));
  f->w = (float*)malloc(na * sizeof(float));
  f->truth_track = (int32_t*)malloc(na * sizeof(int32_t));
  if (p->want_truth) f->truth_state = (double*)malloc(na * 5 * sizeof(double));
  if (!f->sector || !f->row || !f->y || !f->w || !f->truth_track || (p->want_truth && !f->truth_state)) {
    for (int64_t c = 0; c < nchunk; ++c) { free(cbuf[c]); free(tbuf[c]); }
    free(cbuf); free(tbuf); free(ccnt); sy_free_frame(f); return -2;
  }
  {
    int64_t o = 0;
    for (int64_t c = 0; c < nchunk; ++c) {
      for (int64_t i = 0; i < ccnt[c]; ++i, ++o) {
        const sy_crec* r = &cbuf[c][i];
        f->sector[o] = r->sector; f->row[o] = r->row; f->y[o] = r->y; f->w[o] = r->w;
        f->truth_track[o] = r->track;
        if (p->want_truth) memcpy(&f->truth_state[5 * o], &tbuf[c][5 * i], 5 * sizeof(double));
      }
      free(cbuf[c]);
      free(tbuf[c]);
    }
    free(cbuf); free(tbuf); free(ccnt);
    for (int sr = 0; sr < SY_NSEC * SY_NROW; ++sr) {
      sy_rng nr = sy_stream(p, SY_K_NOISE, (uint64_t)sr);
      (void)sy_u01(&nr); /* the draw used for the count above */
      const int s = sr / SY_NROW, r = sr % SY_NROW;
      const double ymax = sy_row_x(r) * tan(10.0 * SY_PI / 180.0);
      for (int64_t j = 0; j < nnoise_sr[sr]; ++j, ++o) {
        double yy = ymax * (2.0 * sy_u01(&nr) - 1.0);
        double ww = wlo + (whi - wlo) * sy_u01(&nr);
        f->sector[o] = (uint8_t)s; f->row[o] = (uint8_t)r;
        f->y[o] = (float)yy; f->w[o] = (float)ww;
        f->truth_track[o] = -1;
        if (p->want_truth) {
          double* tt = &f->truth_state[5 * o];
          tt[0] = yy; tt[1] = ww; tt[2] = tt[3] = tt[4] = NAN;
        }
      }
    }
  }
  if (p->shuffle && n > 1) {
    sy_rng sh = sy_stream(p, SY_K_SHUFFLE, 0);
    for (int64_t i = n - 1; i > 0; --i) {
      int64_t j = (int64_t)(sy_next(&sh) % (uint64_t)(i + 1));
      uint8_t t8 = f->sector[i]; f->sector[i] = f->sector[j]; f->sector[j] = t8;
      t8 = f->row[i]; f->row[i] = f->row[j]; f->row[j] = t8;
      float tf = f->y[i]; f->y[i] = f->y[j]; f->y[j] = tf;
      tf = f->w[i]; f->w[i] = f->w[j]; f->w[j] = tf;
      int32_t ti = f->truth_track[i]; f->truth_track[i] = f->truth_track[j]; f->truth_track[j] = ti;
      if (p->want_truth) {
        double tmp[5];
        memcpy(tmp, &f->truth_state[5 * i], sizeof(tmp));
        memcpy(&f->truth_state[5 * i], &f->truth_state[5 * j], sizeof(tmp));
        memcpy(&f->truth_state[5 * j], tmp, sizeof(tmp));
      }
    }
  }
  *out = f;
  return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Digits: the pad-row readout a cluster finder starts from (Sec. 2: the TPC records, per pad, the
 * charge in 0.2 us time bins, zero-suppressed). Each cluster of a frame spreads a log-normal charge
 * over the pads and time bins of its (sector, row) with a Gaussian of widths (sigma_pad, sigma_time)
 * centred at its (y, w); charges of overlapping clusters add; a cell becomes a digit when its
 * rounded charge reaches adc_threshold, saturating at adc_max.
 *
 * Cell geometry: row r has n_pads(r) = 2 ceil(x_r tan(10 deg) / pad_pitch) pads; pad k spans
 * y in [(k - n/2) p, (k + 1 - n/2) p); time bin j spans w in [j dw, (j + 1) dw), dw = time_bin_w.
 * Digits come out grouped by (sector, row), each group in (time, pad) order (the order in which a
 * row's readout is assembled), or in a seeded random order (shuffle). truth_cluster names the
 * cluster with the largest deposit in the cell.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  uint64_t seed;
  double pad_pitch, time_bin_w;     /* cm */
  double sigma_pad, sigma_time;     /* cm */
  double q_median, q_log_sigma;     /* cluster charge: q_median * exp(q_log_sigma * N(0,1)), ADC */
  int32_t adc_threshold, adc_max;
  int32_t shuffle;
  int32_t n_threads;
} synth_digit_params;

typedef struct {
  int64_t n_digits;
  int32_t n_time;                   /* 1 + the largest time bin of any digit */
  uint8_t* sector;
  uint8_t* row;
  uint16_t* pad;
  uint16_t* time;
  uint16_t* adc;
  int32_t* truth_cluster;
} synth_digits;

enum { SY_K_CHARGE = 5, SY_K_DSHUFFLE = 6 };
#define SY_FOOT 3 /* cells deposited on each side of the cluster's own cell */
#define SY_TCHUNK 512  /* time bins of the digitizer's charge map per pass */

static sy_rng sy_dstream(uint64_t seed, uint64_t kind, uint64_t id) {
  sy_rng r;
  r.s = sy_mix(seed * 0x9E3779B97F4A7C15ULL + 0x2545F4914F6CDD1DULL) ^ sy_mix((kind << 58) ^ (id + 1));
  return r;
}

int synth_npads(double pitch, int r) {
  return 2 * (int)ceil(sy_row_x(r) * tan(10.0 * SY_PI / 180.0) / pitch);
}

/* fraction of a unit Gaussian charge at mean mu, width s, deposited in [a, b) */
static inline double sy_frac(double a, double b, double mu, double s) {
  const double k = 1.0 / (s * sqrt(2.0));
  return 0.5 * (erf((b - mu) * k) - erf((a - mu) * k));
}

void synth_free_digits(synth_digits* d) {
  if (!d) return;
  free(d->sector); free(d->row); free(d->pad); free(d->time); free(d->adc); free(d->truth_cluster);
  free(d);
}

typedef struct { uint16_t pad, time, adc; int32_t truth; } sy_drec;

int synth_digitize(const synth_digit_params* p, int64_t n, const uint8_t* sector, const uint8_t* row,
                   const float* y, const float* w, synth_digits** out) {
  const int G = SY_NSEC * SY_NROW;
  if (!p || !out || n < 0 || p->pad_pitch <= 0 || p->time_bin_w <= 0 || p->adc_threshold < 1 ||
      p->adc_max < p->adc_threshold || p->adc_max > 65535)
    return -1;
  *out = NULL;
  int64_t* gstart = (int64_t*)calloc((size_t)G + 1, sizeof(int64_t));
  int64_t* order = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  sy_drec** gbuf = (sy_drec**)calloc((size_t)G, sizeof(sy_drec*));
  int64_t* gcnt = (int64_t*)calloc((size_t)G, sizeof(int64_t));
  int32_t* gtmax = (int32_t*)calloc((size_t)G, sizeof(int32_t));
  if (!gstart || !order || !gbuf || !gcnt || !gtmax) {
    free(gstart); free(order); free(gbuf); free(gcnt); free(gtmax);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (sector[i] >= SY_NSEC || row[i] >= SY_NROW) { free(gstart); free(order); free(gbuf); free(gcnt); free(gtmax); return -1; }
    ++gstart[sector[i] * SY_NROW + row[i] + 1];
  }
  for (int g = 0; g < G; ++g) gstart[g + 1] += gstart[g];
  {
    int64_t* fill = (int64_t*)malloc((size_t)G * sizeof(int64_t));
    if (!fill) { free(gstart); free(order); free(gbuf); free(gcnt); free(gtmax); return -2; }
    memcpy(fill, gstart, (size_t)G * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) order[fill[sector[i] * SY_NROW + row[i]]++] = i;
    free(fill);
  }
  int failed = 0;
#ifdef _OPENMP
  if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : failed)
#endif
  for (int g = 0; g < G; ++g) {
    const int64_t b = gstart[g], e = gstart[g + 1];
    if (b == e) continue;
    const int r = g % SY_NROW;
    const int np = synth_npads(p->pad_pitch, r);
    const double half = 0.5 * (double)np;
    int64_t jlo = INT64_MAX, jhi = INT64_MIN;
    for (int64_t q = b; q < e; ++q) {
      const int64_t j = (int64_t)floor((double)w[order[q]] / p->time_bin_w);
      if (j < jlo) jlo = j;
      if (j > jhi) jhi = j;
    }
    jlo -= SY_FOOT; jhi += SY_FOOT;
    if (jlo < 0) jlo = 0;
    if (jhi > 65534) jhi = 65534;
    if (jhi < jlo) continue;
    /* the row's charge map in chunks of SY_TCHUNK time bins (a long frame's rows span tens of
     * thousands of bins at low occupancy): each chunk takes the deposits of the clusters whose
     * footprint reaches it, in the clusters' order, so every cell sums the same terms in the same
     * order as a map of the whole range, and the chunks emit their digits in (time, pad) order */
    const int64_t ncl = e - b;
    double* cq = (double*)malloc((size_t)(ncl > 0 ? ncl : 1) * sizeof(double));
    int64_t* cjc = (int64_t*)malloc((size_t)(ncl > 0 ? ncl : 1) * sizeof(int64_t));
    double* q = (double*)malloc((size_t)np * SY_TCHUNK * sizeof(double));
    double* qbest = (double*)malloc((size_t)np * SY_TCHUNK * sizeof(double));
    int32_t* who = (int32_t*)malloc((size_t)np * SY_TCHUNK * sizeof(int32_t));
    int64_t cap = 1024, cnt = 0;
    sy_drec* buf = (sy_drec*)malloc((size_t)cap * sizeof(sy_drec));
    if (!cq || !cjc || !q || !qbest || !who || !buf) {
      free(cq); free(cjc); free(q); free(qbest); free(who); free(buf);
      failed = 1;
      continue;
    }
    for (int64_t c = b; c < e; ++c) {
      const int64_t i = order[c];
      sy_rng rr = sy_dstream(p->seed, SY_K_CHARGE, (uint64_t)i);
      cq[c - b] = p->q_median * exp(p->q_log_sigma * sy_gauss(&rr));
      cjc[c - b] = (int64_t)floor((double)w[i] / p->time_bin_w);
    }
    /* chunks no cluster footprint reaches hold no digit */
    const int64_t nchunk = (jhi - jlo) / SY_TCHUNK + 1;
    unsigned char* used = (unsigned char*)calloc((size_t)nchunk, 1);
    if (!used) {
      free(cq); free(cjc); free(q); free(qbest); free(who); free(buf);
      failed = 1;
      continue;
    }
    for (int64_t c = 0; c < ncl; ++c) {
      int64_t lo = cjc[c] - SY_FOOT - jlo, hi = cjc[c] + SY_FOOT - jlo;
      if (lo < 0) lo = 0;
      if (hi > jhi - jlo) hi = jhi - jlo;
      for (int64_t u = lo / SY_TCHUNK; u <= hi / SY_TCHUNK && lo <= hi; ++u) used[u] = 1;
    }
    int32_t tmax = 0;
    for (int64_t t0 = jlo; t0 <= jhi && !failed; t0 += SY_TCHUNK) {
      if (!used[(t0 - jlo) / SY_TCHUNK]) continue;
      const int64_t t1 = t0 + SY_TCHUNK - 1 < jhi ? t0 + SY_TCHUNK - 1 : jhi;
      const int64_t nt = t1 - t0 + 1;
      memset(q, 0, (size_t)(np * nt) * sizeof(double));
      memset(qbest, 0, (size_t)(np * nt) * sizeof(double));
      for (int64_t c = b; c < e; ++c) {
        const int64_t jc = cjc[c - b];
        if (jc + SY_FOOT < t0 || jc - SY_FOOT > t1) continue;
        const int64_t i = order[c];
        const double Q = cq[c - b];
        const double yc = (double)y[i], wc = (double)w[i];
        const int64_t kc = (int64_t)floor(yc / p->pad_pitch + half);
        double fk[2 * SY_FOOT + 1], fj[2 * SY_FOOT + 1];
        for (int d = -SY_FOOT; d <= SY_FOOT; ++d) {
          const double k = (double)(kc + d), j = (double)(jc + d);
          fk[d + SY_FOOT] = sy_frac((k - half) * p->pad_pitch, (k + 1.0 - half) * p->pad_pitch, yc, p->sigma_pad);
          fj[d + SY_FOOT] = sy_frac(j * p->time_bin_w, (j + 1.0) * p->time_bin_w, wc, p->sigma_time);
        }
        for (int dj = -SY_FOOT; dj <= SY_FOOT; ++dj) {
          const int64_t j = jc + dj;
          if (j < t0 || j > t1) continue;
          for (int dk = -SY_FOOT; dk <= SY_FOOT; ++dk) {
            const int64_t k = kc + dk;
            if (k < 0 || k >= np) continue;
            const double dq = Q * fk[dk + SY_FOOT] * fj[dj + SY_FOOT];
            const int64_t cell = (j - t0) * np + k;
            q[cell] += dq;
            if (dq > qbest[cell]) { qbest[cell] = dq; who[cell] = (int32_t)i; }
          }
        }
      }
      for (int64_t cell = 0; cell < np * nt; ++cell) {
        int64_t a = (int64_t)floor(q[cell] + 0.5);
        if (a < p->adc_threshold) continue;
        if (a > p->adc_max) a = p->adc_max;
        if (cnt == cap) {
          sy_drec* nb = (sy_drec*)realloc(buf, (size_t)(2 * cap) * sizeof(sy_drec));
          if (!nb) { failed = 1; break; }
          buf = nb;
          cap *= 2;
        }
        const int64_t j = t0 + cell / np;
        buf[cnt].pad = (uint16_t)(cell % np);
        buf[cnt].time = (uint16_t)j;
        buf[cnt].adc = (uint16_t)a;
        buf[cnt].truth = who[cell];
        if ((int32_t)j > tmax) tmax = (int32_t)j;
        ++cnt;
      }
    }
    free(cq); free(cjc); free(q); free(qbest); free(who); free(used);
    if (failed) { free(buf); continue; }
    gbuf[g] = buf;
    gcnt[g] = cnt;
    gtmax[g] = cnt > 0 ? tmax + 1 : 0;
  }
  int64_t total = 0;
  int32_t ntime = 0;
  for (int g = 0; g < G; ++g) { total += gcnt[g]; if (gtmax[g] > ntime) ntime = gtmax[g]; }
  synth_digits* d = (synth_digits*)calloc(1, sizeof(synth_digits));
  const size_t na = (size_t)(total > 0 ? total : 1);
  if (d) {
    d->sector = (uint8_t*)malloc(na); d->row = (uint8_t*)malloc(na);
    d->pad = (uint16_t*)malloc(na * 2); d->time = (uint16_t*)malloc(na * 2); d->adc = (uint16_t*)malloc(na * 2);
    d->truth_cluster = (int32_t*)malloc(na * 4);
  }
  if (failed || !d || !d->sector || !d->row || !d->pad || !d->time || !d->adc || !d->truth_cluster) {
    for (int g = 0; g < G; ++g) free(gbuf[g]);
    free(gstart); free(order); free(gbuf); free(gcnt); free(gtmax); synth_free_digits(d);
    return -2;
  }
  d->n_digits = total;
  d->n_time = ntime;
  int64_t o = 0;
  for (int g = 0; g < G; ++g) {
    for (int64_t k = 0; k < gcnt[g]; ++k, ++o) {
      d->sector[o] = (uint8_t)(g / SY_NROW); d->row[o] = (uint8_t)(g % SY_NROW);
      d->pad[o] = gbuf[g][k].pad; d->time[o] = gbuf[g][k].time; d->adc[o] = gbuf[g][k].adc;
      d->truth_cluster[o] = gbuf[g][k].truth;
    }
    free(gbuf[g]);
  }
  free(gstart); free(order); free(gbuf); free(gcnt); free(gtmax);
  if (p->shuffle && total > 1) {
    sy_rng sh = sy_dstream(p->seed, SY_K_DSHUFFLE, 0);
    for (int64_t i = total - 1; i > 0; --i) {
      const int64_t j = (int64_t)(sy_next(&sh) % (uint64_t)(i + 1));
      uint8_t t8 = d->sector[i]; d->sector[i] = d->sector[j]; d->sector[j] = t8;
      t8 = d->row[i]; d->row[i] = d->row[j]; d->row[j] = t8;
      uint16_t t16 = d->pad[i]; d->pad[i] = d->pad[j]; d->pad[j] = t16;
      t16 = d->time[i]; d->time[i] = d->time[j]; d->time[j] = t16;
      t16 = d->adc[i]; d->adc[i] = d->adc[j]; d->adc[j] = t16;
      int32_t t32 = d->truth_cluster[i]; d->truth_cluster[i] = d->truth_cluster[j]; d->truth_cluster[j] = t32;
    }
  }
  *out = d;
  return 0;
}
