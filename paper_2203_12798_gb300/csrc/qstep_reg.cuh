// Register-resident Q-step of the ALS iterations (Alg. 3 first inner loop;
// Eq. q_k) for one warp: for every slice k of the warp's share
//   T_k = F~_k Psi S_k H^T  (R x R),  T_k = Z_k Sigma_k P_k^T  (one-sided Jacobi),
//   Upol_k = Z_k P_k^T,  Pi_k = Upol_k^T F~_k,
// plus the Lemma 1 partial sum  G1 += (Pi_k Psi) diag(W(k,:))  of each group.
//
// Layout: one problem per group of R lanes (floor(32 / R) problems per warp);
// lane c of a group holds column c of T and column c of the accumulated right
// rotations V in registers.  Each Jacobi step pairs columns by the cyclic
// round-robin ordering; the two lanes of a pair exchange their columns with
// shuffles and compute the same rotation from the same operands (the same
// products in the same order), so no shared state is needed.  Column norms
// are carried along with the rotations (a' = a - t g, b' = b + t g) and
// recomputed at every sweep start.  Small products go through per-group
// shared memory.  R is a compile-time constant; ranks that are not
// instantiated run padded with zero rows / columns (zero columns are never
// rotated and get zero singular values, so the padded problem's polar factor
// restricted to the first R_actual rows / columns is the actual one).
//
// Warm start: T_k changes little from one ALS iteration to the next, so the
// right rotations P_k of the previous Q-step (Prot) are an almost exact
// starting point: the sweeps start from T_k V0 with V0 = Prot_k after one
// Newton-Schulz step V0 <- V0 (3 I - V0^T V0) / 2 that restores its
// orthonormality to rounding level (the rotations are accumulated in FP32
// across iterations).  The polar factor does not depend on the start.
//
// Used by the Q-step kernel (k_qstep.cu) and the persistent ALS kernel
// (k_als_persist.cu).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace dp2 {

// Shared memory of one warp: G groups x 3 R^2 floats of scratch (F~_k, T, P)
// and G x R^2 floats of Lemma 1 slots.
template <int R>
__host__ __device__ constexpr int qreg_groups() { return 32 / R; }

// The slices of warp `warp` are groups first, first + step, ... of G
// consecutive slices.  ps, hs: Psi and H (R x R, zero padded past Ra) in
// shared memory.  gscr: this warp's G x 3 R^2 scratch; gslots: its G x R^2
// Lemma 1 slots (zeroed here, accumulated over the warp's slices).
template <int R>
__device__ __forceinline__ void qstep_warp(int K, int Ra, const float* __restrict__ Ft, const float* ps,
                                           const float* hs, const float* __restrict__ W, float* __restrict__ Upol,
                                           float* __restrict__ Pi, int* __restrict__ status, int want_g1,
                                           float* __restrict__ Prot, const int* __restrict__ rank, float* gscr,
                                           float* gslots, int64_t first, int64_t step) {
  constexpr int G = 32 / R;  // problems per warp
  constexpr int RR = R * R;
  constexpr int M = R + (R & 1);  // round-robin players (one dummy when R is odd)
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int g = lane / R, c = lane - g * R;
  const bool lane_act = g < G;
  float* gs = gscr + (size_t)(lane_act ? g : 0) * 3 * RR;
  float* Fs = gs;
  float* Ts = gs + RR;
  float* Ps = gs + 2 * RR;
  const float tol = fmaxf(1e-6f, (float)Ra * 1.2e-7f);
  // a sweep whose largest kept-pair ratio |g| / sqrt(a b) is r leaves ratios
  // of about sqrt(R) r^2 behind: below rstop that is below tol, and the
  // sweep that would only confirm it is skipped
  const float rstop = sqrtf(tol * rsqrtf((float)Ra));
  const int RaRa = Ra * Ra;
  // Lemma 1 partial of this group, column c owned by lane c (accumulated in
  // shared memory: no registers held across the sweeps)
  float* gslot = gslots + (size_t)(lane_act ? g : 0) * RR;
  if (lane_act) {
#pragma unroll
    for (int i = 0; i < R; ++i) gslot[i * R + c] = 0.f;
  }

  for (int64_t kb = first * G; kb < K; kb += step * G) {
    const int64_t k = kb + g;
    const bool act = lane_act && k < K;
    // F~_k, column c
    if (lane_act) {
#pragma unroll
      for (int i = 0; i < R; ++i) Fs[i * R + c] = (act && i < Ra && c < Ra) ? Ft[k * RaRa + i * Ra + c] : 0.f;
    }
    // W(k, c) of this lane's column, and the scaled H rows W(k, r) H(c, r) of
    // T's second factor in the group's P scratch (read back by column)
    const float wc = (act && c < Ra) ? W[k * Ra + c] : 0.f;
    if (lane_act) {
#pragma unroll
      for (int r = 0; r < R; ++r) Ps[r * R + c] = (act && r < Ra ? W[k * Ra + r] : 0.f) * hs[c * R + r];
    }
    __syncwarp();
    // A1 = F~_k Psi, column c
    float t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < R; ++m) s = fmaf(Fs[i * R + m], ps[m * R + c], s);
      t[i] = s;
    }
    if (lane_act) {
#pragma unroll
      for (int i = 0; i < R; ++i) Ts[i * R + c] = t[i];
    }
    __syncwarp();
    // T = A1 S_k H^T, column c:  T(i, c) = sum_r A1(i, r) W(k, r) H(c, r)
#pragma unroll
    for (int i = 0; i < R; ++i) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) s = fmaf(Ts[i * R + r], Ps[r * R + c], s);
      t[i] = s;
    }
    __syncwarp();  // P scratch is free again
    float v[R];
    if (Prot) {
      // V0 = Prot_k (padded with the identity), column c
#pragma unroll
      for (int i = 0; i < R; ++i)
        v[i] = (act && i < Ra && c < Ra) ? Prot[k * RaRa + i * Ra + c] : (i == c ? 1.f : 0.f);
      if (lane_act) {
#pragma unroll
        for (int i = 0; i < R; ++i) Ps[i * R + c] = v[i];
      }
      __syncwarp();
      // Newton-Schulz: v <- 1.5 v - 0.5 V (V^T v)
      float gc[R];
#pragma unroll
      for (int a = 0; a < R; ++a) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) s = fmaf(Ps[i * R + a], v[i], s);
        gc[a] = s;
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < R; ++a) s = fmaf(Ps[i * R + a], gc[a], s);
        v[i] = fmaf(1.5f, v[i], -0.5f * s);
      }
      // T V0, column c (T through the group scratch)
      if (lane_act) {
#pragma unroll
        for (int i = 0; i < R; ++i) Ts[i * R + c] = t[i];
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < R; ++i) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < R; ++m) s = fmaf(Ts[i * R + m], v[m], s);
        t[i] = s;
      }
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = (i == c) ? 1.f : 0.f;
    }

    // ---- one-sided Jacobi, parallel round-robin ordering.  Convergence (the
    // rstop rule of k_eig_reg) is judged on the r_k largest columns only (r_k = the slice's stage-1 rank
    // >= rank(T_k)): the other R - r_k columns shrink to rounding noise of a
    // zero singular value and keep rotating among themselves without ever
    // passing the orthogonality test; the polar factor leaves them out.
    // (r_k differs between the problems of a warp: the ranking below runs in
    // every lane, only its use depends on r_k)
    const int rk = (act && rank) ? min(rank[k], Ra) : Ra;
    int sweep = 0;
    for (; sweep < 30; ++sweep) {
      float na = 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) na = fmaf(t[i], t[i], na);
      int above = 0;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float nj = __shfl_sync(FULL, na, (g * R + j) & 31);
        above += (nj > na || (nj == na && j < c)) ? 1 : 0;
      }
      const bool top = rk >= R || above < rk;
      float rmax = 0.f;  // largest ratio over pairs of kept columns
#pragma unroll 1
      for (int rr = 0; rr < M - 1; ++rr) {
        int p;
        if (c == 0) {
          p = 1 + rr;
        } else {
          const int x = c - 1;
          p = (x == rr) ? 0 : 1 + ((2 * rr - x + 2 * (M - 1)) % (M - 1));
        }
        const bool pair = lane_act && p < R;
        const int src = pair ? g * R + p : lane;
        const bool lo = c < p;
        const float nb = __shfl_sync(FULL, na, src);
        const int ptop = __shfl_sync(FULL, top ? 1 : 0, src);  // every lane shuffles
        const bool both_top = top && ptop != 0;
        const float a = lo ? na : nb, b = lo ? nb : na;
        if constexpr (R <= 12) {
          // partner columns held in registers
          float tp[R], vp[R];
#pragma unroll
          for (int i = 0; i < R; ++i) {
            tp[i] = __shfl_sync(FULL, t[i], src);
            vp[i] = __shfl_sync(FULL, v[i], src);
          }
          float gm = 0.f;
#pragma unroll
          for (int i = 0; i < R; ++i) gm = fmaf(t[i], tp[i], gm);
          const float rel = (pair && a > 0.f && b > 0.f) ? fabsf(gm) * rsqrtf(a) * rsqrtf(b) : 0.f;
          if (both_top) rmax = fmaxf(rmax, rel);
          if (rel > tol) {
            const float zeta = (b - a) / (2.f * gm);
            const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
            const float sg = lo ? -sn : sn;
#pragma unroll
            for (int i = 0; i + 1 < R; i += 2) {
              rot2(t[i], t[i + 1], tp[i], tp[i + 1], cs, sg);
              rot2(v[i], v[i + 1], vp[i], vp[i + 1], cs, sg);
            }
            if (R & 1) {
              t[R - 1] = fmaf(cs, t[R - 1], sg * tp[R - 1]);
              v[R - 1] = fmaf(cs, v[R - 1], sg * vp[R - 1]);
            }
            na = lo ? fmaf(-tt, gm, na) : fmaf(tt, gm, na);
          }
        } else {
          // larger R: partner entries shuffled again where they are used (fewer registers)
          float gm = 0.f;
#pragma unroll
          for (int i = 0; i < R; ++i) gm = fmaf(t[i], __shfl_sync(FULL, t[i], src), gm);
          const float rel = (pair && a > 0.f && b > 0.f) ? fabsf(gm) * rsqrtf(a) * rsqrtf(b) : 0.f;
          if (both_top) rmax = fmaxf(rmax, rel);
          const bool rot = rel > tol;
          float cs = 1.f, sg = 0.f, tt = 0.f;
          if (rot) {
            const float zeta = (b - a) / (2.f * gm);
            tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            cs = rsqrtf(fmaf(tt, tt, 1.f));
            sg = lo ? -cs * tt : cs * tt;
            na = lo ? fmaf(-tt, gm, na) : fmaf(tt, gm, na);
          }
#pragma unroll
          for (int i = 0; i + 1 < R; i += 2) {
            const float tp0 = __shfl_sync(FULL, t[i], src), tp1 = __shfl_sync(FULL, t[i + 1], src);
            const float vp0 = __shfl_sync(FULL, v[i], src), vp1 = __shfl_sync(FULL, v[i + 1], src);
            if (rot) {
              rot2(t[i], t[i + 1], tp0, tp1, cs, sg);
              rot2(v[i], v[i + 1], vp0, vp1, cs, sg);
            }
          }
          if (R & 1) {
            const float tpi = __shfl_sync(FULL, t[R - 1], src);
            const float vpi = __shfl_sync(FULL, v[R - 1], src);
            if (rot) {
              t[R - 1] = fmaf(cs, t[R - 1], sg * tpi);
              v[R - 1] = fmaf(cs, v[R - 1], sg * vpi);
            }
          }
        }
      }
      if (warp_max(rmax) <= rstop) break;
    }
    if (sweep == 30 && lane == 0) set_status(status, ST_SWEEP_CAP);
    if (Prot && act && c < Ra) {
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (i < Ra) Prot[k * RaRa + i * Ra + c] = v[i];
    }

    // ---- polar factor Upol = sum_i z_i v_i^T over the rank(F~_k) largest
    // sigma_i > 0.  rank(T_k) <= rank(F~_k) = the slice's stage-1 rank r_k, so
    // the other R - r_k final columns are rounding noise of a zero singular
    // value (a slice with I_k < R) and are left out; of the r_k kept ones every
    // nonzero column counts, however small (the final columns are mutually
    // orthogonal, and an FP32-level cut would drop directions of ill-conditioned
    // T_k that an FP64 SVD resolves).  Padded columns are zero.
    float s2 = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) s2 = fmaf(t[i], t[i], s2);
    const float sg = sqrtf(s2);
    int above = 0;  // columns of this problem ahead of column c in sigma order
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float sj = __shfl_sync(FULL, sg, (g * R + j) & 31);
      above += (sj > sg || (sj == sg && j < c)) ? 1 : 0;
    }
    const float inv = (sg > 0.f && above < rk) ? 1.f / sg : 0.f;
    __syncwarp();
    if (lane_act) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        Ts[i * R + c] = t[i] * inv;  // Z column c
        Ps[i * R + c] = v[i];        // P column c
      }
    }
    __syncwarp();
    float up[R];  // Upol column c: Upol(a, c) = sum_i Z(a, i) P(c, i)
#pragma unroll
    for (int a = 0; a < R; ++a) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) s = fmaf(Ts[a * R + i], Ps[c * R + i], s);
      up[a] = s;
    }
    if (act && c < Ra) {
#pragma unroll
      for (int a = 0; a < R; ++a)
        if (a < Ra) Upol[k * RaRa + a * Ra + c] = up[a];
    }
    __syncwarp();
    if (lane_act) {
#pragma unroll
      for (int a = 0; a < R; ++a) Ts[a * R + c] = up[a];
    }
    __syncwarp();
    float pc[R];  // Pi column c: Pi(a, c) = sum_i Upol(i, a) F~(i, c)
#pragma unroll
    for (int a = 0; a < R; ++a) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) s = fmaf(Ts[i * R + a], Fs[i * R + c], s);
      pc[a] = s;
    }
    if (act && c < Ra) {
#pragma unroll
      for (int a = 0; a < R; ++a)
        if (a < Ra) Pi[k * RaRa + a * Ra + c] = pc[a];
    }
    if (want_g1) {
      __syncwarp();
      if (lane_act) {
#pragma unroll
        for (int a = 0; a < R; ++a) Ps[a * R + c] = pc[a];
      }
      __syncwarp();
      // Lemma 1: G1(i, c) += W(k, c) (Pi Psi)(i, c)
      if (lane_act) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          float s = 0.f;
#pragma unroll
          for (int m = 0; m < R; ++m) s = fmaf(Ps[i * R + m], ps[m * R + c], s);
          gslot[i * R + c] = fmaf(wc, s, gslot[i * R + c]);
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace dp2
