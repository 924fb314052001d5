// Phases of one ALS iteration on the compressed slices (Alg. 3 repeat loop;
// Lemmas 1-3), shared by the three-launch iteration (k_als3.cu) and the
// persistent ALS kernel (k_als_persist.cu).  Every block that forms an update
// computes it from the same partials in the same order, so all blocks hold
// identical H, CV and inverses.
//
// Slice lists: a warp visits slices u * per + j (j < per) for u = first,
// first + step, ... (per = 1: every step-th slice; per = G: the groups of G
// consecutive slices of the register Q-step).
#pragma once
#include "common.cuh"
#include "internal.h"
#include "small_solve.cuh"

namespace dp2 {

// FP64 dot product sum_m a[m * sa] b[m * sb] over m < n as two interleaved
// chains (even and odd m) added at the end: a dependent FP64 FMA takes tens
// of cycles on this part, so two independent chains halve the latency.
__device__ __forceinline__ double dot2(const double* a, int sa, const double* b, int sb, int n) {
  double s0 = 0.0, s1 = 0.0;
  int m = 0;
  for (; m + 1 < n; m += 2) {
    s0 = fma(a[m * sa], b[m * sb], s0);
    s1 = fma(a[(m + 1) * sa], b[(m + 1) * sb], s1);
  }
  if (m < n) s0 = fma(a[m * sa], b[m * sb], s0);
  return s0 + s1;
}

// ---------------------------------------------------------------- H update --
// Hs (float, shared) and HtH (double, shared) <- the H update of Lemma 1 from
// the Q-step's partials: G1 = sum of the partials (FP64 combine), H = G1 InvH
// (FP64), columns scaled to unit norm, rounded to FP32; H^T H from the
// rounded H.  Whole block; work areas G1, Hn: R^2 doubles each; red: T doubles.
// quad != 0: the partials are read as float4 quads (par_reduce4_*; red then
// holds 4 T doubles, pstride a multiple of 4).
__device__ inline void block_h_update(const float* __restrict__ part1, int nq, int pstride,
                                      const double* __restrict__ InvH, int R, double* red, double* G1, double* Hn,
                                      float* Hs, double* HtH, int* status, int quad = 0) {
  __shared__ double scl[kMaxR];
  const int RR = R * R, T = blockDim.x;
  if (quad) par_reduce4_load(part1, nq, pstride, RR, red);
  else par_reduce_load(part1, nq, pstride, RR, 0, T, red, G1);
  __syncthreads();
  if (quad) par_reduce4_combine(RR, nq, red, G1);
  else par_reduce_combine(RR, 0, T, red, G1);
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {
    const int i = e / R, r = e - i * R;
    Hn[e] = dot2(G1 + i * R, 1, InvH + r, R, R);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += T) scl[r] = inv_norm(dot2(Hn + r, R, Hn + r, R, R), status);
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {
    const float h = (float)(Hn[e] * scl[e % R]);
    Hs[e] = h;
    Hn[e] = (double)h;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {
    const int a = e / R, b = e - a * R;
    HtH[e] = dot2(Hn + a, R, Hn + b, R, R);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Lemma 2 --
// One warp: slot (2 R^2 floats, hi in [0, RR), lo in [RR, 2 RR)) += for its
// slices g(m, r) = W(k, r) sum_i Pi_k(i, m) H(i, r) as double-float sums (the
// V update's system has condition numbers up to ~1e8 on nearly collinear
// factors, where FP32 rounding of g that no perturbation of the Pi_k explains
// derails the iteration).  hs: H (float, shared); pks: R^2 floats of scratch.
__device__ inline void lemma2_warp(int K, int R, const float* __restrict__ Pi, const float* __restrict__ W,
                                   const float* hs, float* slot, float* pks, int64_t first, int64_t step, int per) {
  const int RR = R * R, lane = threadIdx.x & 31;
  for (int64_t u = first; u * per < K; u += step) {
    for (int j = 0; j < per; ++j) {
      const int64_t k = u * per + j;
      if (k >= K) break;
      for (int e = lane; e < RR; e += 32) pks[e] = Pi[k * RR + e];
      __syncwarp();
      const float* wk = W + k * R;
      for (int e = lane; e < RR; e += 32) {
        const int m = e / R, r = e % R;
        DF d = {0.f, 0.f};
        for (int i = 0; i < R; ++i) df_mac(d, pks[i * R + m], hs[i * R + r]);
        const float w = wk[r];
        const float p = d.hi * w;
        DF t;
        t.hi = p;
        t.lo = fmaf(d.hi, w, -p) + d.lo * w;
        const DF acc = df_add(DF{slot[e], slot[RR + e]}, t);
        slot[e] = acc.hi;
        slot[RR + e] = acc.lo;
      }
      __syncwarp();
    }
  }
}

// Whole block: dst[e] (hi) and dst[n + e] (lo) <- the double-float sum over
// the nw warps' slots (2 n floats each, stride sstride) in warp order.
__device__ inline void block_slots_df(const float* slots, int nw, int sstride, int n, float* __restrict__ dst) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    DF a = {0.f, 0.f};
    for (int w = 0; w < nw; ++w) a = df_add(a, DF{slots[w * sstride + e], slots[w * sstride + n + e]});
    dst[e] = a.hi;
    dst[n + e] = a.lo;
  }
}

// ---------------------------------------------------------------- V update --
// Whole block: g from the Lemma 2 partials (double-float halves combined in
// FP64), CV = g InvV (FP64), columns scaled to unit norm through D^T D and
// rounded to FP32 (cvs), Psi = D^T D CV (DC, FP64; ps, FP32) and
// Gm = V^T V * H^T H with V^T V = CV^T D^T D CV formed from the rounded CV.
// With vtv != null the block also writes V^T V there (and CV, Psi to cvg,
// psig).  Work areas: red T doubles (4 T with quad), Cb 2 R^2, C, DC, Gm R^2
// doubles.
__device__ inline void block_v_update(const float* __restrict__ part2, int nb2, int pstride,
                                      const double* __restrict__ InvV, const double* __restrict__ DtD, const double* HtH,
                                      int R, double* red, double* Cb, double* C, double* DC, double* Gm, float* cvs,
                                      float* ps, double* vtv, float* cvg, double* psig, int* status, int quad = 0) {
  __shared__ double scl[kMaxR];
  const int RR = R * R, T = blockDim.x;
  if (quad) par_reduce4_load(part2, nb2, pstride, 2 * RR, red);
  else par_reduce_load(part2, nb2, pstride, 2 * RR, 0, T, red, Cb);
  __syncthreads();
  if (quad) par_reduce4_combine(2 * RR, nb2, red, Cb);
  else par_reduce_combine(2 * RR, 0, T, red, Cb);
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) Cb[e] += Cb[RR + e];  // g = hi + lo
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {
    const int i = e / R, r = e - i * R;
    C[e] = dot2(Cb + i * R, 1, InvV + r, R, R);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {  // DC = DtD C
    const int i = e / R, r = e - i * R;
    DC[e] = dot2(DtD + i * R, 1, C + r, R, R);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += T)  // ||V(:, r)||^2 = C(:, r)^T DtD C(:, r)
    scl[r] = inv_norm(fmax(dot2(C + r, R, DC + r, R, R), 0.0), status);
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {
    const float c = (float)(C[e] * scl[e % R]);
    cvs[e] = c;
    C[e] = (double)c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {  // Psi = DtD CV (rounded CV)
    const int i = e / R, r = e - i * R;
    const double s = dot2(DtD + i * R, 1, C + r, R, R);
    DC[e] = s;
    ps[e] = (float)s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += T) {  // V^T V = CV^T DtD CV; Gm = V^T V * H^T H
    const int a = e / R, b = e - a * R;
    const double s = dot2(C + a, R, DC + b, R, R);
    Gm[e] = s * HtH[e];
    if (vtv) {
      vtv[e] = s;
      psig[e] = DC[e];
      cvg[e] = cvs[e];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Lemma 3 --
// One warp, for its slices: G3(k, r) = H(:, r)^T Pi_k Psi(:, r) (FP32,
// insensitive), W_k = G3_k Ginv (FP64 product, stored FP32), and partials of
// W^T W (double-float in slot: hi [0, RR), lo [RR, 2 RR), from the stored
// FP32 W) and of e_k = ||Pi_k - H S_k CV^T||^2 (ek, double-float).
// ps, hs, cvs: Psi, H, CV (float, shared); gi: Ginv (FP64); pks: R^2, g3 and
// wn: R floats of scratch.
__device__ inline void lemma3_warp(int K, int R, const float* __restrict__ Pi, const float* ps, const float* hs,
                                   const float* cvs, const double* gi, float* __restrict__ W, float* slot, float* pks,
                                   float* g3, float* wn, DF& ek, int64_t first, int64_t step, int per) {
  const int RR = R * R, lane = threadIdx.x & 31;
  for (int64_t u = first; u * per < K; u += step) {
    for (int j = 0; j < per; ++j) {
      const int64_t k = u * per + j;
      if (k >= K) break;
      for (int e = lane; e < RR; e += 32) pks[e] = Pi[k * RR + e];
      __syncwarp();
      for (int r = lane; r < R; r += 32) {
        float s = 0.f;
        for (int i = 0; i < R; ++i) {
          float t = 0.f;
          for (int m = 0; m < R; ++m) t = fmaf(pks[i * R + m], ps[m * R + r], t);
          s = fmaf(hs[i * R + r], t, s);
        }
        g3[r] = s;
      }
      __syncwarp();
      for (int r = lane; r < R; r += 32) {
        double s = 0.0;
        for (int m = 0; m < R; ++m) s = fma((double)g3[m], gi[m * R + r], s);
        wn[r] = (float)s;
        W[k * R + r] = (float)s;
      }
      __syncwarp();
      for (int e = lane; e < RR; e += 32) {
        const int a = e / R, b = e - a * R;
        float mdl = 0.f;  // (H S_k CV^T)(a, b)
        for (int r = 0; r < R; ++r) mdl = fmaf(hs[a * R + r] * wn[r], cvs[b * R + r], mdl);
        const float d = pks[e] - mdl;
        df_mac(ek, d, d);
        DF g = {slot[e], slot[RR + e]};
        df_mac(g, wn[a], wn[b]);
        slot[e] = g.hi;
        slot[RR + e] = g.lo;
      }
      __syncwarp();
    }
  }
}

// Whole block, after lemma3_warp and a barrier: dst[0, 2 RR) <- the W^T W
// partial (double-float), dst[2 RR], dst[2 RR + 1] <- the e partial; ered:
// 32 x 2 floats of shared scratch.
__device__ inline void block_lemma3_out(const float* slots, int nw, int sstride, int R, DF ek, float (*ered)[2],
                                        float* __restrict__ dst) {
  const int RR = R * R, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF other;
    other.hi = __shfl_xor_sync(0xffffffffu, ek.hi, o);
    other.lo = __shfl_xor_sync(0xffffffffu, ek.lo, o);
    ek = df_add(ek, other);
  }
  if (lane == 0) {
    ered[warp][0] = ek.hi;
    ered[warp][1] = ek.lo;
  }
  __syncthreads();
  block_slots_df(slots, nw, sstride, RR, dst);
  if (threadIdx.x == 0) {
    DF s = {0.f, 0.f};
    for (int w = 0; w < nw; ++w) s = df_add(s, DF{ered[w][0], ered[w][1]});
    dst[2 * RR] = s.hi;
    dst[2 * RR + 1] = s.lo;
  }
}


// Whole block: dst[e] (hi), dst[n + e] (lo) <- the double-float sum of the
// G group slots of each of nw warps (warp w's slots start at w * wstride +
// off, 2 n floats apart by gstride), in warp-then-group order.
__device__ inline void block_group_slots_df(const float* wreg, int nw, int wstride, int off, int G, int gstride,
                                            int n, float* __restrict__ dst) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    DF a = {0.f, 0.f};
    for (int w = 0; w < nw; ++w)
      for (int g = 0; g < G; ++g) {
        const float* sl = wreg + (size_t)w * wstride + off + (size_t)g * gstride;
        a = df_add(a, DF{sl[e], sl[n + e]});
      }
    dst[e] = a.hi;
    dst[n + e] = a.lo;
  }
}

// ------------------------------------------- Lemma 2 / 3, group layout ----
// The same per-entry arithmetic as lemma2_warp / lemma3_warp, laid out as the
// register Q-step: lane c of group g (G = 32 / RP groups of RP lanes) works on
// column c of slice u * G + g, so a warp handles G slices at once and every
// loop over R is unrolled (RP is a compile-time constant, Ra <= RP the actual
// rank; lanes and rows past Ra are idle / zero).  gscr: the warp's G x RP^2
// floats of scratch; hs, ps, cvs: H, Psi, CV (compact Ra x Ra, shared).
//
// Lemma 2: acc[m] (lane c) += W(k, c) sum_i Pi_k(i, m) H(i, c), double-float.
template <int RP>
__device__ __forceinline__ void lemma2_group(int K, int Ra, const float* __restrict__ Pi, const float* __restrict__ W,
                                             const float* hs, float* gscr, DF (&acc)[RP], int64_t first,
                                             int64_t step) {
  constexpr int G = 32 / RP;
  const int lane = threadIdx.x & 31, g = lane / RP, c = lane - g * RP;
  const bool lane_act = g < G && c < Ra;
  const int RaRa = Ra * Ra;
  float* Ps = gscr + (size_t)(g < G ? g : 0) * RP * RP;
  float hc[RP];  // H(:, c)
#pragma unroll
  for (int i = 0; i < RP; ++i) hc[i] = (lane_act && i < Ra) ? hs[i * Ra + c] : 0.f;
#pragma unroll
  for (int m = 0; m < RP; ++m) acc[m] = DF{0.f, 0.f};
  for (int64_t kb = first * G; kb < K; kb += step * G) {
    const int64_t k = kb + g;
    const bool act = lane_act && k < K;
    __syncwarp();
    if (g < G) {
#pragma unroll
      for (int i = 0; i < RP; ++i) Ps[i * RP + c] = (act && i < Ra) ? Pi[k * RaRa + i * Ra + c] : 0.f;
    }
    __syncwarp();
    const float w = act ? W[k * Ra + c] : 0.f;
#pragma unroll
    for (int m = 0; m < RP; ++m) {
      DF d = {0.f, 0.f};
#pragma unroll
      for (int i = 0; i < RP; ++i)
        if (i < Ra) df_mac(d, Ps[i * RP + m], hc[i]);
      const float p = d.hi * w;
      DF t;
      t.hi = p;
      t.lo = fmaf(d.hi, w, -p) + d.lo * w;
      if (act && m < Ra) acc[m] = df_add(acc[m], t);
    }
  }
}

// Lemma 3 and the W update: W_k(c) = sum_m G3(k, m) Ginv(m, c) (FP64) with
// G3(k, c) = H(:, c)^T Pi_k Psi(:, c); wtw[a] (lane c) += W(k, a) W(k, c) and
// ek += ||Pi_k(:, c) - (H S_k CV^T)(:, c)||^2, both double-float.  H, Psi, CV
// and Ginv are read from shared memory where they are used (no register
// copies: the kernels running this hold many registers already).
template <int RP>
__device__ __forceinline__ void lemma3_group(int K, int Ra, const float* __restrict__ Pi, const float* ps,
                                             const float* hs, const float* cvs, const double* gi,
                                             float* __restrict__ W, float* gscr, DF (&wtw)[RP], DF& ek,
                                             int64_t first, int64_t step) {
  constexpr int G = 32 / RP;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane / RP, c = lane - g * RP;
  const bool lane_act = g < G && c < Ra;
  const int cc = lane_act ? c : 0;
  const int RaRa = Ra * Ra;
  float* Ps = gscr + (size_t)(g < G ? g : 0) * RP * RP;
#pragma unroll
  for (int m = 0; m < RP; ++m) wtw[m] = DF{0.f, 0.f};
  ek = DF{0.f, 0.f};
  for (int64_t kb = first * G; kb < K; kb += step * G) {
    const int64_t k = kb + g;
    const bool act = lane_act && k < K;
    __syncwarp();
    if (g < G) {
#pragma unroll
      for (int i = 0; i < RP; ++i) Ps[i * RP + c] = (act && i < Ra) ? Pi[k * RaRa + i * Ra + c] : 0.f;
    }
    __syncwarp();
    // G3(k, c) = sum_i H(i, c) sum_m Pi(i, m) Psi(m, c)
    float g3 = 0.f;
#pragma unroll
    for (int i = 0; i < RP; ++i) {
      if (i < Ra) {
        float t = 0.f;
#pragma unroll
        for (int m = 0; m < RP; ++m)
          if (m < Ra) t = fmaf(Ps[i * RP + m], ps[m * Ra + cc], t);
        g3 = fmaf(hs[i * Ra + cc], t, g3);
      }
    }
    // W(k, c) = sum_m G3(k, m) Ginv(m, c) in FP64
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < RP; ++m) {
      const float gm = __shfl_sync(FULL, g3, (g * RP + m) & 31);
      if (m < Ra) s = fma((double)gm, gi[m * Ra + cc], s);
    }
    const float wc = lane_act ? (float)s : 0.f;
    if (act) W[k * Ra + c] = wc;
    // t_r = W(k, r) CV(c, r); the model column (H S_k CV^T)(:, c) = H t
    float tr[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const float wr = __shfl_sync(FULL, wc, (g * RP + r) & 31);
      tr[r] = (r < Ra) ? wr * cvs[cc * Ra + r] : 0.f;
      if (act && r < Ra) df_mac(wtw[r], wr, wc);
    }
    if (act) {
#pragma unroll
      for (int a = 0; a < RP; ++a) {
        if (a < Ra) {
          float mdl = 0.f;  // (H S_k CV^T)(a, c) = sum_r H(a, r) t_r
#pragma unroll
          for (int r = 0; r < RP; ++r)
            if (r < Ra) mdl = fmaf(hs[a * Ra + r], tr[r], mdl);
          const float d = Ps[a * RP + c] - mdl;
          df_mac(ek, d, d);
        }
      }
    }
  }
}

}  // namespace dp2
