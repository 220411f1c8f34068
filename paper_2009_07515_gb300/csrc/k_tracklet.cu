// k_tracklet.cu — K5 tracklet construction (helix Kalman filter in the solenoid field).
//
// One lane builds one tracklet at a time; a lane that finishes takes the next start hit from a
// device work counter, so lanes stay busy while their neighbours are still extending long tracks
// (persistent kernel, grid = SMs x resident blocks). Every lane runs the same per-step code
// (propagate one row, pick the candidate, update), so the warp stays converged except in the
// candidate search. Steps of one tracklet:
//   walk    follow the cleaned up-links to find the chain's length, middle and last hit;
//   seed    circle through the first, middle and last chain hits, covariance diag(cov0);
//   A/B     outward: one row per step, candidate = the chain hit while the chain lasts, then the
//           hit of smallest chi2 in the row's grid window nsig*sqrt(C)+add; Joseph-form update
//           when chi2 <= chi2_max; stop after n_miss_max empty rows past the chain, on
//           |sin(phi)| >= max_sin, or when |y| leaves the row by more than y_margin;
//   C       inward from the outermost hit with the covariance reset: refit the A/B hits row by
//           row, then search below the chain start the same way; the state at the last accepted
//           hit is the tracklet's fit at x_ref.
// Output per tracklet: fit (P, C, chi2, x_ref), counts, and its hit in every row of
// [ref_row, top_row] in the row-major slab.
#include "tpc_dev.cuh"

namespace tpc {

enum : int { kIdle = 0, kWalk = 1, kOut = 2, kIn = 3 };

struct Lane {
  float P[5], C[15], SP[5], SC[15];
  float chi2sum;
  int t, phase, r, r0, top, ref, nmiss, nh, m;
  int head, mid, chain, gb;
};

__device__ __forceinline__ void snapshot(Lane& L) {
#pragma unroll
  for (int i = 0; i < 5; ++i) L.SP[i] = L.P[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) L.SC[i] = L.C[i];
}

__device__ __forceinline__ void reset_cov(const DevParams& Q, float* C) {
#pragma unroll
  for (int i = 0; i < 15; ++i) C[i] = 0.f;
  C[lt(0, 0)] = Q.cov0[0];
  C[lt(1, 1)] = Q.cov0[1];
  C[lt(2, 2)] = Q.cov0[2];
  C[lt(3, 3)] = Q.cov0[3];
  C[lt(4, 4)] = Q.cov0[4];
}

// smallest-chi2 hit of segment g inside the window around the predicted (y, w); kNoHit if none
__device__ __forceinline__ int search_row(const Work& W, const DevParams& Q, int g, const float* P, const float* C,
                                          float& chi_out) {
  const float wy = Q.win_nsig * sqrtf(C[lt(0, 0)]) + Q.win_add;
  const float ww = Q.win_nsig * sqrtf(C[lt(1, 1)]) + Q.win_add;
  const uint32_t bb = W.seg_bb[g];
  const int nb = (int)W.seg_nb[g];
  const float2 geo = W.seg_geo[g];
  const float pad = win_pad(P[1], ww);
  const int b0 = bin_of((P[1] - ww) - pad, geo.x, geo.y, nb);
  const int b1 = bin_of((P[1] + ww) + pad, geo.x, geo.y, nb);
  const int p0 = (int)W.bin_start[bb + b0], p1 = (int)W.bin_start[bb + b1 + 1];
  // chi2 pieces depend on C only
  const float S00 = C[0] + Q.r00, S01 = C[1], S10 = C[1], S11 = C[2] + Q.r11;
  const float det = S00 * S11 - S01 * S10;
  const bool pd = det > 0.f;
  const float i00 = S11 / det, i01 = -S01 / det, i10 = -S10 / det, i11 = S00 / det;
  int best = -1;
  float bchi = __int_as_float(0x7f800000);
  for (int h = p0; h < p1; ++h) {
    const float2 c = W.hyw[h];
    if (!(fabsf(c.x - P[0]) <= wy && fabsf(c.y - P[1]) <= ww)) continue;
    float chi;
    if (pd) {
      const float r0 = c.x - P[0], r1 = c.y - P[1];
      chi = r0 * (i00 * r0 + i01 * r1) + r1 * (i10 * r0 + i11 * r1);
    } else {
      chi = __int_as_float(0x7f800000);
    }
    bool better;
    if (best < 0 || chi < bchi) better = true;
    else if (chi > bchi) better = false;
    else {
      const float2 o = W.hyw[best];
      better = key_less(c.y, c.x, W.horig[h], o.y, o.x, W.horig[best]);
    }
    if (better) { best = h; bchi = chi; }
  }
  chi_out = bchi;
  return best;
}

__device__ __forceinline__ void finish(const Work& W, const DevParams& Q, Lane& L, bool ok) {
  const long long t = L.t;
  if (ok) {
    float* o = W.tl_state + t * 24;
#pragma unroll
    for (int i = 0; i < 5; ++i) o[i] = L.SP[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) o[5 + i] = L.SC[i];
    o[20] = L.chi2sum;
    o[21] = Q.x[L.ref];
    W.tl_info[t] = (uint32_t)L.nh | ((uint32_t)L.ref << 8) | ((uint32_t)L.top << 16) | (1u << 24);
  } else {
    W.tl_info[t] = 0u;
  }
  L.phase = kIdle;
}

__global__ void __launch_bounds__(128) k_tracklets(Work W, DevParams Q) {
  const uint32_t ntl = min(W.cnt->n_starts, (uint32_t)W.tcap);
  const long long tcap = W.tcap;
  Lane L;
  L.phase = kIdle;
  L.t = -1;
  for (;;) {
    if (L.phase == kIdle) {
      const uint32_t t = atomicAdd(&W.cnt->k5_next, 1u);
      if (t >= ntl) break;
      const uint4 st = W.starts[t];
      L.t = (int)t;
      const int g = (int)st.y;
      L.r0 = (g % kSegPerFrame) % kNRow;
      L.gb = g - L.r0;
      L.head = (int)st.x;
      L.mid = (int)st.x;
      L.m = 1;
      L.phase = kWalk;
      continue;
    }
    if (L.phase == kWalk) {
      // advance the head one link; keep mid = chain[m/2]
      const int nx = W.clinks[L.head].y;
      if (nx >= 0 && L.m < kNRow) {
        L.head = nx;
        L.m += 1;
        if ((L.m & 1) == 0) L.mid = W.clinks[L.mid].y;
        continue;
      }
      // seed from chain[0], chain[m/2], chain[m-1]
      const int h0 = (int)W.starts[L.t].x;
      const float2 a = W.hyw[h0], b = W.hyw[L.mid], c = W.hyw[L.head];
      float hh[3][3];
      hh[0][0] = Q.x[L.r0];               hh[0][1] = a.x; hh[0][2] = a.y;
      hh[1][0] = Q.x[L.r0 + L.m / 2];     hh[1][1] = b.x; hh[1][2] = b.y;
      hh[2][0] = Q.x[L.r0 + L.m - 1];     hh[2][1] = c.x; hh[2][2] = c.y;
      if (!kf_seed(Q, hh, L.P)) { finish(W, Q, L, false); continue; }
      reset_cov(Q, L.C);
      L.phase = kOut;
      L.r = L.r0;
      L.top = -1;
      L.nmiss = 0;
      L.chain = h0;
      continue;
    }
    if (L.phase == kOut) {
      const int r = L.r;
      bool stop = false;
      if (r > L.r0) {
        if (!kf_propagate(Q, L.P, L.C, Q.x[r - 1], Q.x[r])) stop = true;
        else {
          const float lim = Q.x[r] * Q.tan10 + Q.y_margin;
          if (fabsf(L.P[0]) > lim) stop = true;
        }
      }
      if (!stop) {
        int hit;
        float chi;
        const bool on_chain = L.chain >= 0;
        if (on_chain) {
          hit = L.chain;
          L.chain = W.clinks[hit].y;
          const float2 c = W.hyw[hit];
          chi = kf_chi2(Q, L.P, L.C, c.x, c.y);
        } else {
          hit = search_row(W, Q, L.gb + r, L.P, L.C, chi);
        }
        if (hit >= 0 && chi <= Q.chi2_max) {
          const float2 c = W.hyw[hit];
          kf_update(Q, L.P, L.C, c.x, c.y);
          W.slab[(long long)r * tcap + L.t] = (uint32_t)hit;
          L.nmiss = 0;
          L.top = r;
          snapshot(L);
        } else {
          W.slab[(long long)r * tcap + L.t] = kNoHit;
          L.nmiss += 1;
          if (!on_chain && L.nmiss >= Q.n_miss_max) stop = true;
        }
        L.r = r + 1;
        if (L.r >= kNRow) stop = true;
      }
      if (stop) {
        if (L.top < 0) { finish(W, Q, L, false); continue; }
        // phase C: from the outermost hit, covariance reset
#pragma unroll
        for (int i = 0; i < 5; ++i) L.P[i] = L.SP[i];
        reset_cov(Q, L.C);
        L.phase = kIn;
        L.r = L.top;
        L.nmiss = 0;
        L.nh = 0;
        L.ref = -1;
        L.chi2sum = 0.f;
      }
      continue;
    }
    // kIn
    {
      const int r = L.r;
      bool stop = false;
      if (r < L.top) {
        if (!kf_propagate(Q, L.P, L.C, Q.x[r + 1], Q.x[r])) stop = true;
        else {
          const float lim = Q.x[r] * Q.tan10 + Q.y_margin;
          if (fabsf(L.P[0]) > lim) stop = true;
        }
      }
      if (!stop) {
        int hit;
        float chi = __int_as_float(0x7f800000);
        if (r >= L.r0) {
          const uint32_t s = W.slab[(long long)r * tcap + L.t];
          hit = s == kNoHit ? -1 : (int)s;
          if (hit >= 0) {
            const float2 c = W.hyw[hit];
            chi = kf_chi2(Q, L.P, L.C, c.x, c.y);
          }
        } else {
          hit = search_row(W, Q, L.gb + r, L.P, L.C, chi);
        }
        if (hit >= 0 && chi <= Q.chi2_max) {
          const float2 c = W.hyw[hit];
          kf_update(Q, L.P, L.C, c.x, c.y);
          W.slab[(long long)r * tcap + L.t] = (uint32_t)hit;
          L.nh += 1;
          L.chi2sum = L.chi2sum + chi;
          L.nmiss = 0;
          L.ref = r;
          snapshot(L);
        } else {
          W.slab[(long long)r * tcap + L.t] = kNoHit;
          L.nmiss += 1;
          if (r < L.r0 && L.nmiss >= Q.n_miss_max) stop = true;
        }
        L.r = r - 1;
        if (L.r < 0) stop = true;
      }
      if (stop) finish(W, Q, L, L.ref >= 0);
    }
  }
}

}  // namespace tpc
