// ALS iterations on the compressed slices (Alg. 3 repeat loop; Sec. III-C..E).
//
// Per iteration, with F~_k = F^(k) E (R x R), Psi = D^T V (R x R):
//   Q-step (Eq. q_k): T_k = F~_k Psi S_k H^T; one-sided Jacobi SVD
//     T_k = Z_k Sigma_k P_k^T; Upol_k = Z_k P_k^T; Pi_k = Upol_k^T F~_k
//     (= P_k Z_k^T F^(k) E, so Y_k = Pi_k D^T is never formed).
//   Lemma 1: G1(:, r) = (sum_k W(k,r) Pi_k) Psi(:, r);  H = G1 (W^T W * V^T V)^+,
//     columns normalised.
//   Lemma 2: G2(:, r) = D g_r, g_r = sum_k W(k,r) Pi_k^T H(:, r);
//     V = G2 (W^T W * H^T H)^+ = D CV, CV = [g_r] (.)^+, columns normalised.
//     V stays in span(D), so Psi = D^T D CV and V^T V = CV^T D^T D CV are
//     R x R products (D^T D from stage 2).
//   Lemma 3: G3(k, r) = H(:, r)^T Pi_k Psi(:, r);  W = G3 (V^T V * H^T H)^+.
//   Convergence value (Sec. III-E): e = sum_k ||Pi_k D^T - H S_k V^T||^2
//     = sum_k ||Pi_k - H S_k CV^T||^2 (D^T D = I), summed from the residual
//     entries themselves.
// Grid-wide sums are block partials reduced in a fixed order (deterministic).
// The R x R Gram-Hadamard solves are FP64: a Gauss-Jordan inverse by the
// whole block for R <= 32, otherwise (or when a pivot fails) a Cholesky
// factorisation with the pseudoinverse from an FP64 Jacobi eigendecomposition
// as the last resort, applied in FP64 to the right-hand sides: Lemma 1 and 3
// partials in FP32 (compensated block sums), Lemma 2 partials and W^T W as
// double-float sums of exact products.  For R <= 20 and a fixed iteration
// count the whole loop runs as one persistent launch (k_als_persist.cu).
#include "common.cuh"
#include "internal.h"
#include "small_solve.cuh"

namespace dp2 {

constexpr int ALS_WARPS = 16;

// out[e] = sum_b part[b * pstride + e] for e < n.  The whole block cooperates:
// every entry's partials are split over tpe threads (8 loads in flight per
// thread, compensated fp32 sums), then combined in a fixed order in FP64.
// Thread t takes entry e0 + t mod per and every tpe-th partial from t / per
// on, so that a warp reads consecutive entries of one partial (coalesced).
__device__ void block_reduce_parts(const float* __restrict__ part, int nblk, int pstride, int n, double* out) {
  __shared__ double red[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int tpe = max(1, T / n), per = T / tpe;
  for (int e0 = 0; e0 < n; e0 += per) {
    const int e = e0 + t % per, sub = t / per;
    const bool act = sub < tpe && e < n;
    float s = 0.f, c = 0.f;
    if (act) {
      int b = sub;
      for (; b + 7 * tpe < nblk; b += 8 * tpe) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = part[(int64_t)(b + u * tpe) * pstride + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) neumaier(s, c, v[u]);
      }
      for (; b < nblk; b += tpe) neumaier(s, c, part[(int64_t)b * pstride + e]);
    }
    red[t] = (double)s + (double)c;
    __syncthreads();
    if (act && sub == 0) {
      double a = 0.0;
      for (int q = 0; q < tpe; ++q) a += red[q * per + t];
      out[e] = a;
    }
    __syncthreads();
  }
}


// out (n x n, FP64) = A^T B for A, B (rows x n, fp32, row-major): every block
// stages tiles of ATB_ROWS rows of its row chunk in shared memory and
// accumulates up to 16 entries per thread; the block partials are summed in
// a fixed order in FP64 by k_atb_fin.
constexpr int ATB_ROWS = 32;
constexpr int ATB_THREADS = 256;

__global__ void __launch_bounds__(ATB_THREADS) k_atb_part(int64_t rows, int n, const float* __restrict__ A,
                                                          const float* __restrict__ B, int64_t chunk,
                                                          float* __restrict__ part) {
  __shared__ float as[ATB_ROWS * kMaxR], bs[ATB_ROWS * kMaxR];
  const int t = threadIdx.x, nn = n * n;
  int ea[16], eb[16];
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = t + q * ATB_THREADS;
    ea[q] = e < nn ? e / n : 0;
    eb[q] = e < nn ? e % n : 0;
    acc[q] = 0.f;
  }
  const int64_t r0 = blockIdx.x * chunk, r1 = min64(rows, r0 + chunk);
  for (int64_t i0 = r0; i0 < r1; i0 += ATB_ROWS) {
    const int nr = (int)min64(ATB_ROWS, r1 - i0);
    __syncthreads();
    for (int e = t; e < nr * n; e += ATB_THREADS) {
      as[e] = A[i0 * n + e];
      bs[e] = B[i0 * n + e];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (t + q * ATB_THREADS < nn) {
        float s = acc[q];
        for (int i = 0; i < nr; ++i) s = fmaf(as[i * n + ea[q]], bs[i * n + eb[q]], s);
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = t + q * ATB_THREADS;
    if (e < nn) part[(int64_t)blockIdx.x * nn + e] = acc[q];
  }
}

__global__ void k_atb_fin(int nb, int nn, const float* __restrict__ part, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += (double)part[(int64_t)b * nn + e];
    out[e] = s;
  }
}

// ----------------------------------------------------- one-sided Jacobi ----
// Columns of T (n x n, pitch ld) are orthogonalised by plane rotations from
// the right, accumulated into V (starts at I).  Parallel (round-robin)
// ordering; lane i < m/2 owns one column pair per step.  Returns sweeps used
// (> max_sweeps when not converged).
// Convergence is judged on the rk largest columns (by norm at the start of a
// sweep; n <= 64): with rank(T) <= rk the other columns shrink to rounding
// noise and keep rotating among themselves without passing the test.  cn:
// n floats of warp scratch.
__device__ int warp_onesided_jacobi(float* T, float* V, int n, int ld, float tol, int max_sweeps, int rk,
                                    float* cn) {
  const int lane = threadIdx.x & 31;
  const int m = n + (n & 1);
  for (int e = lane; e < n * n; e += 32) V[(e / n) * ld + e % n] = (e / n == e % n) ? 1.f : 0.f;
  __syncwarp();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float worst = 0.f;
    unsigned long long topm = ~0ull;  // columns in the rk largest
    if (rk < n) {
      for (int c = lane; c < n; c += 32) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s = fmaf(T[i * ld + c], T[i * ld + c], s);
        cn[c] = s;
      }
      __syncwarp();
      bool in0 = false, in1 = false;
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        bool in = false;
        if (c < n) {
          int above = 0;
          for (int j = 0; j < n; ++j) above += (cn[j] > cn[c] || (cn[j] == cn[c] && j < c)) ? 1 : 0;
          in = above < rk;
        }
        if (h == 0) in0 = in;
        else in1 = in;
      }
      topm = ((unsigned long long)__ballot_sync(0xffffffffu, in1) << 32) | __ballot_sync(0xffffffffu, in0);
      __syncwarp();
    }
    for (int r = 0; r < m - 1; ++r) {
      for (int pi = lane; pi < m / 2; pi += 32) {
        int p, q;
        if (pi == 0) {
          p = 0;
          q = 1 + (r % (m - 1));
        } else {
          p = 1 + ((r + pi) % (m - 1));
          q = 1 + ((r - pi + (m - 1)) % (m - 1));
        }
        if (p > q) { int t = p; p = q; q = t; }
        if (q >= n) continue;
        float a = 0.f, b = 0.f, g = 0.f;
        for (int i = 0; i < n; ++i) {
          const float tp = T[i * ld + p], tq = T[i * ld + q];
          a = fmaf(tp, tp, a);
          b = fmaf(tq, tq, b);
          g = fmaf(tp, tq, g);
        }
        if (a == 0.f || b == 0.f) continue;
        const float rel = fabsf(g) * rsqrtf(a) * rsqrtf(b);
        if ((topm >> p) & (topm >> q) & 1ull) worst = fmaxf(worst, rel);
        if (rel <= tol) continue;
        const float zeta = (b - a) / (2.f * g);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float c = rsqrtf(1.f + t * t), s = c * t;
        for (int i = 0; i < n; ++i) {
          const float tp = T[i * ld + p], tq = T[i * ld + q];
          T[i * ld + p] = c * tp - s * tq;
          T[i * ld + q] = s * tp + c * tq;
          const float vp = V[i * ld + p], vq = V[i * ld + q];
          V[i * ld + p] = c * vp - s * vq;
          V[i * ld + q] = s * vp + c * vq;
        }
      }
      __syncwarp();
    }
    worst = warp_max(worst);
    if (worst <= tol) return sweep + 1;
  }
  return max_sweeps + 1;
}

// ------------------------------------------------------------- Q-step ----
// One warp per slice.  Writes Upol_k, Pi_k and the block partial of Lemma 1's
// G1 (R x R) into part[blk * pstride].
__global__ void k_qstep(int K, int R, const float* __restrict__ Ft, const double* __restrict__ Psi,
                        const float* __restrict__ W, const float* __restrict__ H, float* __restrict__ Upol,
                        float* __restrict__ Pi, float* __restrict__ part, int pstride, int* __restrict__ status,
                        int want_g1, const int* __restrict__ rank) {
  extern __shared__ __align__(16) float sm[];
  const int ld = R + 1, RR = R * R;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ps = sm;             // Psi (R x R)
  float* hs = ps + RR;        // H
  float* slots = hs + RR;     // nw x RR
  float* mine = slots + nw * RR + warp * (2 * R * ld + 3 * RR);
  float* Tm = mine;           // R x ld
  float* Vm = Tm + R * ld;    // R x ld
  float* Fk = Vm + R * ld;    // R x R
  float* A1 = Fk + RR;        // R x R
  float* Up = A1 + RR;        // R x R
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    ps[e] = (float)Psi[e];
    hs[e] = H[e];
  }
  for (int e = threadIdx.x; e < nw * RR; e += blockDim.x) slots[e] = 0.f;
  __syncthreads();
  const float tol = fmaxf(1e-6f, (float)R * 1.2e-7f);
  for (int k = blockIdx.x * nw + warp; k < K; k += gridDim.x * nw) {
    const float* fk = Ft + (int64_t)k * RR;
    const float* wk = W + (int64_t)k * R;
    for (int e = lane; e < RR; e += 32) Fk[e] = fk[e];
    __syncwarp();
    for (int e = lane; e < RR; e += 32) {  // A1 = F~_k Psi
      const int i = e / R, r = e % R;
      float s = 0.f;
      for (int m = 0; m < R; ++m) s = fmaf(Fk[i * R + m], ps[m * R + r], s);
      A1[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < RR; e += 32) {  // T = A1 S_k H^T
      const int i = e / R, b = e % R;
      float s = 0.f;
      for (int r = 0; r < R; ++r) s = fmaf(A1[i * R + r] * wk[r], hs[b * R + r], s);
      Tm[i * ld + b] = s;
    }
    __syncwarp();
    const int rk = rank ? min(rank[k], R) : R;  // one slice per warp: uniform in the warp
    const int sw = warp_onesided_jacobi(Tm, Vm, R, ld, tol, 30, rk, A1);
    if (sw > 30 && lane == 0) set_status(status, ST_SWEEP_CAP);
    // sigma_i = ||T(:, i)||; Upol = sum T(:, i) V(:, i)^T / sigma_i over the
    // rank(F~_k) = r_k largest sigma_i > 0 (the rest are rounding noise of zero
    // singular values; the kept final columns are mutually orthogonal however
    // small).  Fk doubles as the kept-column factors 1 / sigma_i.
    for (int i = lane; i < R; i += 32) {
      float s = 0.f;
      for (int a = 0; a < R; ++a) s = fmaf(Tm[a * ld + i], Tm[a * ld + i], s);
      A1[i] = sqrtf(s);
    }
    __syncwarp();
    float* kinv = Up;  // R factors, overwritten below only after use
    for (int i = lane; i < R; i += 32) {
      const float sg = A1[i];
      int above = 0;
      for (int j = 0; j < R; ++j) above += (A1[j] > sg || (A1[j] == sg && j < i)) ? 1 : 0;
      kinv[i] = (sg > 0.f && above < rk) ? 1.f / sg : 0.f;
    }
    __syncwarp();
    for (int i = lane; i < R; i += 32) A1[i] = kinv[i];
    __syncwarp();
    for (int e = lane; e < RR; e += 32) {
      const int a = e / R, b = e % R;
      float s = 0.f;
      for (int i = 0; i < R; ++i) s = fmaf(Tm[a * ld + i] * A1[i], Vm[b * ld + i], s);
      Up[e] = s;
    }
    __syncwarp();
    float* up = Upol + (int64_t)k * RR;
    float* pk = Pi + (int64_t)k * RR;
    for (int e = lane; e < RR; e += 32) {  // Pi = Upol^T F~_k
      const int a = e / R, b = e % R;
      float s = 0.f;
      for (int i = 0; i < R; ++i) s = fmaf(Up[i * R + a], Fk[i * R + b], s);
      up[e] = Up[e];
      pk[e] = s;
      A1[e] = s;
    }
    __syncwarp();
    if (want_g1) {
      float* slot = slots + warp * RR;
      for (int e = lane; e < RR; e += 32) {  // slot += (Pi Psi) o W_k
        const int i = e / R, r = e % R;
        float s = 0.f;
        for (int m = 0; m < R; ++m) s = fmaf(A1[i * R + m], ps[m * R + r], s);
        slot[e] += wk[r] * s;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  if (want_g1)
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
      float s = 0.f;
      for (int w = 0; w < nw; ++w) s += slots[w * RR + e];
      part[(int64_t)blockIdx.x * pstride + e] = s;
    }
}

// --------------------------------------------------------- Lemma 2 partial --
// part[blk] (R x R): g(m, r) += W(k, r) sum_i Pi_k(i, m) H(i, r), as
// double-float sums: exact products (TwoProduct) added with TwoSum, the hi
// floats in entries [0, R^2) of the partial and the lo floats in [R^2, 2 R^2).
// The V update solves with (W^T W * H^T H), whose condition number reaches
// 1e8 and more when H's columns become nearly parallel (the spectrogram
// workload: 4e8); there a relative error of 2e-7 in g that no perturbation
// of the Pi_k explains already derails the iteration, while FP32 dot products
// of length R carry several 1e-7.  With double-float sums the right-hand side
// is exact for the FP32 Pi_k, H and W it is formed from.
// With pre_on the grid's last block runs pre_solve (the V update's factor).
__global__ void k_g2(int K, int R, const float* __restrict__ Pi, const float* __restrict__ W,
                     const float* __restrict__ H, float* __restrict__ part, int pstride, PreSolve pre, int pre_on) {
  extern __shared__ __align__(16) float sm[];
  if (pre_on && blockIdx.x == gridDim.x - 1) {
    pre_solve(pre, reinterpret_cast<double*>(sm));
    return;
  }
  const int nb = gridDim.x - pre_on;
  const int RR = R * R;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* hs = sm;
  float* slots = hs + RR;                              // nw x 2 RR: hi then lo
  float* pks = slots + 2 * nw * RR + warp * RR;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) hs[e] = H[e];
  for (int e = threadIdx.x; e < 2 * nw * RR; e += blockDim.x) slots[e] = 0.f;
  __syncthreads();
  float* slot = slots + warp * 2 * RR;
  for (int k = blockIdx.x * nw + warp; k < K; k += nb * nw) {
    for (int e = lane; e < RR; e += 32) pks[e] = Pi[(int64_t)k * RR + e];
    __syncwarp();
    const float* wk = W + (int64_t)k * R;
    for (int e = lane; e < RR; e += 32) {
      const int m = e / R, r = e % R;
      DF d = {0.f, 0.f};
      for (int i = 0; i < R; ++i) df_mac(d, pks[i * R + m], hs[i * R + r]);
      // (d.hi + d.lo) * w as a double-float, added to the slot
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
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    DF a = {0.f, 0.f};
    for (int w = 0; w < nw; ++w) a = df_add(a, DF{slots[w * 2 * RR + e], slots[w * 2 * RR + RR + e]});
    part[(int64_t)blockIdx.x * pstride + e] = a.hi;
    part[(int64_t)blockIdx.x * pstride + RR + e] = a.lo;
  }
}

// --------------------------------------------------- Lemma 3 and W update --
// W_k = G3_k Ginv with G3(k, r) = H(:, r)^T Pi_k Psi(:, r) (G3 in FP32, the
// product with the FP64 inverse in FP64); also the block partials of W^T W
// and of the convergence value e, both double-float sums: W^T W's hi floats
// in entries [0, R^2), its lo floats in [R^2, 2 R^2), e's in 2 R^2 and
// 2 R^2 + 1.  W^T W is summed from exact products of the stored FP32 W (the
// H and V updates solve with W^T W * V^T V and W^T W * H^T H, whose
// condition numbers reach 1e6..1e8 on nearly collinear factors: a Gram
// matrix that disagrees with the stored W by FP32 rounding already makes
// those systems indefinite).  e is summed as the residual itself:
// Y_k - H S_k V^T = (Pi_k - H S_k CV^T) D^T with V = D CV, and D^T D = I to
// FP32 rounding, so e_k = ||Pi_k - H S_k CV^T||_F^2 (an R x R residual whose
// entries are formed before squaring; the expanded form ||Pi_k||^2 -
// 2 tr(...) + ... subtracts terms thousands of times larger than e when the
// model explains most of the compressed slices).
__global__ void k_g3w(int K, int R, const float* __restrict__ Pi, const double* __restrict__ Psi,
                      const float* __restrict__ H, const double* __restrict__ Ginv, const float* __restrict__ CV,
                      float* __restrict__ W, float* __restrict__ part, int pstride) {
  extern __shared__ __align__(16) double smd[];
  __shared__ float ered[32][2];
  const int RR = R * R;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* gi = smd;  // Ginv
  float* ps = reinterpret_cast<float*>(gi + RR);
  float* hs = ps + RR;
  float* cvs = hs + RR;
  float* slots = cvs + RR;          // nw x 2 RR (hi, lo)
  float* pks = slots + nw * 2 * RR + warp * (RR + 2 * R);
  float* g3 = pks + RR;
  float* wn = g3 + R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    ps[e] = (float)Psi[e];
    hs[e] = H[e];
    gi[e] = Ginv[e];
    cvs[e] = CV[e];
  }
  for (int e = threadIdx.x; e < nw * 2 * RR; e += blockDim.x) slots[e] = 0.f;
  __syncthreads();
  float* slot = slots + warp * 2 * RR;
  // e_k accumulated per lane as a double-float sum of exact squares
  DF ek;
  ek.hi = 0.f;
  ek.lo = 0.f;
  for (int k = blockIdx.x * nw + warp; k < K; k += gridDim.x * nw) {
    for (int e = lane; e < RR; e += 32) pks[e] = Pi[(int64_t)k * RR + e];
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
      W[(int64_t)k * R + r] = (float)s;
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
  // lane sums -> warp -> block, as double-float sums in a fixed order (FP32 pipes)
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
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    DF a = {0.f, 0.f};
    for (int w = 0; w < nw; ++w) a = df_add(a, DF{slots[w * 2 * RR + e], slots[w * 2 * RR + RR + e]});
    part[(int64_t)blockIdx.x * pstride + e] = a.hi;
    part[(int64_t)blockIdx.x * pstride + RR + e] = a.lo;
  }
  if (threadIdx.x == 0) {
    DF s = {0.f, 0.f};
    for (int w = 0; w < nw; ++w) s = df_add(s, DF{ered[w][0], ered[w][1]});
    part[(int64_t)blockIdx.x * pstride + 2 * RR] = s.hi;
    part[(int64_t)blockIdx.x * pstride + 2 * RR + 1] = s.lo;
  }
}

// shared memory of the H / V updates: the pseudoinverse workspace plus 5 R^2 + 2
// doubles of intermediates and W^T W's double-float partial sums when that
// fits in 160 KB, else the workspace only
inline size_t update_smem(int R, int* inshared) {
  const size_t full = (spd_pinv_words(R) + 6 * (size_t)R * R + 4) * sizeof(double);
  *inshared = full <= 160 * 1024;
  return *inshared ? full : spd_pinv_smem(R);
}

// --------------------------------------------------------------- H update --
// H = G1 (W^T W * V^T V)^+, columns normalised; HtH = H^T H.
// When it > 0 it first closes the previous iteration: W^T W and its e from the
// partials of the W update (part3; e as a (hi, lo) float pair).
__global__ void __launch_bounds__(1024) k_update_h(int R, const float* __restrict__ part, int nq,
                                                  const float* __restrict__ part3, int nblk, int pstride, int it,
                                                  double* __restrict__ WtW, const double* __restrict__ VtV,
                                                  float* __restrict__ H, double* __restrict__ HtH,
                                                  double* __restrict__ loss, double* __restrict__ scratch,
                                                  int* __restrict__ status, int inshared,
                                                  const double* __restrict__ InvPre) {
  extern __shared__ __align__(16) double ush[];
  __shared__ double scl[kMaxR];
  const int RR = R * R;
  // R x R intermediates in shared memory (global scratch for large R); L, V:
  // work arrays of the pseudoinverse fallback
  double* L = scratch;
  double* V = L + RR;
  double* G1 = inshared ? ush + spd_pinv_words(R) : scratch + 2 * RR;
  double* Gm = G1 + RR;
  double* Inv = Gm + RR;
  double* Hn = Inv + RR;
  double* W3 = Hn + RR;  // 2 RR + 2: W^T W (hi, lo), e (hi, lo)
  __shared__ int ok;
  __shared__ double red[kRedMax];
  const int T = blockDim.x;
  if (InvPre) {
    // W^T W, the loss and (W^T W * V^T V)^+ come from the Q-step's extra block
    par_reduce_load(part, nq, pstride, RR, 0, T, red, G1);
    __syncthreads();
    par_reduce_combine(RR, 0, T, red, G1);
    __syncthreads();
  } else {
    if (it > 0) {
      // W-update partials: W^T W as (hi, lo) in [0, 2 RR), e as (hi, lo) after them
      par_reduce_load(part3, nblk, pstride, 2 * RR + 2, 0, T, red, W3);
      __syncthreads();
      par_reduce_combine(2 * RR + 2, 0, T, red, W3);
      __syncthreads();
      for (int e = threadIdx.x; e < RR; e += blockDim.x) W3[e] += W3[RR + e];
      __syncthreads();
      for (int e = threadIdx.x; e < RR + 1; e += blockDim.x) {
        if (e < RR) WtW[e] = W3[e];
        else {
          const double v = W3[2 * RR] + W3[2 * RR + 1];
          loss[it - 1] = v;
          if (!isfinite(v)) set_status(status, ST_NONFINITE);
        }
      }
    }
    for (int e = threadIdx.x; e < RR; e += blockDim.x) Gm[e] = (it > 0 ? W3[e] : WtW[e]) * VtV[e];
    __syncthreads();
    // warp 0 factors (W^T W * V^T V) while the other threads reduce the Lemma 1 partials
    if (threadIdx.x < 32) {
      const bool f = warp_spd_factor<double>(Gm, R, ush);
      if (threadIdx.x == 0) ok = f;
    }
    par_reduce_load(part, nq, pstride, RR, 32, T - 32, red, G1);
    __syncthreads();
    par_reduce_combine(RR, 32, T - 32, red, G1);
    __syncthreads();
    block_spd_finish<double, double>(ok != 0, Gm, Inv, L, V, R, ush, status);
  }
  const double* Iv = InvPre ? InvPre : Inv;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int i = e / R, r = e - i * R;
    double s = 0.0;
    for (int m = 0; m < R; ++m) s = fma(G1[i * R + m], Iv[m * R + r], s);
    Hn[e] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double n2 = 0.0;
    for (int i = 0; i < R; ++i) n2 = fma(Hn[i * R + r], Hn[i * R + r], n2);
    scl[r] = inv_norm(n2, status);
  }
  __syncthreads();
  // H is stored in FP32: H^T H is formed from the rounded values, so that it
  // agrees exactly with the H the next right-hand sides are formed from
  for (int e = threadIdx.x; e < RR; e += blockDim.x) Hn[e] = (double)(float)(Hn[e] * scl[e % R]);
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    H[e] = (float)Hn[e];
    const int a = e / R, b = e - a * R;
    double s = 0.0;
    for (int i = 0; i < R; ++i) s = fma(Hn[i * R + a], Hn[i * R + b], s);
    HtH[e] = s;
  }
}

// --------------------------------------------------------------- V update --
// CV = g (W^T W * H^T H)^+ with columns normalised through D^T D; then
// Psi = D^T D CV, V^T V = CV^T D^T D CV and Ginv = (V^T V * H^T H)^+ for the W update.
__global__ void __launch_bounds__(1024) k_update_v(int R, const float* __restrict__ part, int nblk, int pstride,
                                                  const double* __restrict__ WtW, const double* __restrict__ HtH,
                                                  const double* __restrict__ DtD, float* __restrict__ CV,
                                                  double* __restrict__ Psi, double* __restrict__ VtV,
                                                  double* __restrict__ Ginv, double* __restrict__ scratch,
                                                  int* __restrict__ status, int inshared,
                                                  const double* __restrict__ InvPre) {
  extern __shared__ __align__(16) double ush[];
  __shared__ double scl[kMaxR];
  const int RR = R * R;
  double* L = scratch;
  double* V = L + RR;
  double* g = inshared ? ush + spd_pinv_words(R) : scratch + 2 * RR;
  double* Gm = g + RR;
  double* Inv = Gm + RR;
  double* C = Inv + RR;
  double* DC = C + RR;
  __shared__ int ok;
  __shared__ double red[kRedMax];
  const int T = blockDim.x;
  // the Lemma 2 partials are double-float (hi in [0, RR), lo in [RR, 2 RR)):
  // both halves reduced (into C and DC, free until later), then added
  if (InvPre) {
    // (W^T W * H^T H)^+ comes from the Lemma 2 grid's extra block
    par_reduce_load(part, nblk, pstride, 2 * RR, 0, T, red, C);
    __syncthreads();
    par_reduce_combine(2 * RR, 0, T, red, C);
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < RR; e += blockDim.x) Gm[e] = WtW[e] * HtH[e];
    __syncthreads();
    // warp 0 factors (W^T W * H^T H) while the other threads reduce the Lemma 2 partials
    if (threadIdx.x < 32) {
      const bool f = warp_spd_factor<double>(Gm, R, ush);
      if (threadIdx.x == 0) ok = f;
    }
    par_reduce_load(part, nblk, pstride, 2 * RR, 32, T - 32, red, C);
    __syncthreads();
    par_reduce_combine(2 * RR, 32, T - 32, red, C);
    __syncthreads();
    block_spd_finish<double, double>(ok != 0, Gm, Inv, L, V, R, ush, status);
  }
  for (int e = threadIdx.x; e < RR; e += blockDim.x) g[e] = C[e] + C[RR + e];
  __syncthreads();
  const double* Iv = InvPre ? InvPre : Inv;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int i = e / R, r = e - i * R;
    double s = 0.0;
    for (int m = 0; m < R; ++m) s = fma(g[i * R + m], Iv[m * R + r], s);
    C[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {  // DC = DtD C
    const int i = e / R, r = e - i * R;
    double s = 0.0;
    for (int m = 0; m < R; ++m) s = fma(DtD[i * R + m], C[m * R + r], s);
    DC[e] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {  // ||V(:, r)||^2 = C(:, r)^T DtD C(:, r)
    double n2 = 0.0;
    for (int i = 0; i < R; ++i) n2 = fma(C[i * R + r], DC[i * R + r], n2);
    scl[r] = inv_norm(fmax(n2, 0.0), status);
  }
  __syncthreads();
  // CV is stored in FP32: Psi = D^T D CV and V^T V = CV^T D^T D CV are formed
  // from the rounded CV, so that they agree exactly with the V = D CV the
  // next Q-step and right-hand sides use
  for (int e = threadIdx.x; e < RR; e += blockDim.x) C[e] = (double)(float)(C[e] * scl[e % R]);
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {  // DC = DtD C
    const int i = e / R, r = e - i * R;
    double s = 0.0;
    for (int m = 0; m < R; ++m) s = fma(DtD[i * R + m], C[m * R + r], s);
    DC[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e - a * R;
    CV[e] = (float)C[e];
    Psi[e] = DC[e];
    double s = 0.0;
    for (int i = 0; i < R; ++i) s = fma(C[i * R + a], DC[i * R + b], s);
    VtV[e] = s;
    Gm[e] = s * HtH[e];
  }
  __syncthreads();
  // Ginv = (V^T V * H^T H)^-1 in FP64 (the W update applies it in FP64)
  block_spd_pinv<double, double>(Gm, Ginv, L, V, R, ush, status);
}

// ----------------------------------------------------- iteration epilogue --
__global__ void k_finish(int R, const float* __restrict__ part, int nblk, int pstride, double* __restrict__ WtW,
                         double* __restrict__ loss, int it, double* __restrict__ scratch, int* __restrict__ status) {
  const int RR = R * R;
  block_reduce_parts(part, nblk, pstride, 2 * RR + 2, scratch);
  for (int e = threadIdx.x; e < RR + 1; e += blockDim.x) {
    if (e < RR) WtW[e] = scratch[e] + scratch[RR + e];
    else {
      const double v = scratch[2 * RR] + scratch[2 * RR + 1];
      loss[it] = v;
      if (!isfinite(v)) set_status(status, ST_NONFINITE);
    }
  }
}

// ---------------------------------------------------------------- init ----
// H = I, W = 1, W^T W = K, H^T H = I, Psi = D^T V0, V^T V = V0^T V0.
// Prot_k = I (the Q-step's first right rotations).
__global__ void k_als_init(int K, int J, int R, const float* __restrict__ D, const float* __restrict__ V0,
                           float* __restrict__ H, float* __restrict__ W, double* __restrict__ WtW,
                           double* __restrict__ HtH, double* __restrict__ Psi, double* __restrict__ VtV,
                           float* __restrict__ Prot) {
  const int RR = R * R;
  if (blockIdx.x > 0) {
    const int64_t nt = (int64_t)(gridDim.x - 1) * blockDim.x;
    const int64_t t0 = (blockIdx.x - 1) * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < (int64_t)K * R; i += nt) W[i] = 1.f;
    if (Prot)
      for (int64_t i = t0; i < (int64_t)K * RR; i += nt) {
        const int e = (int)(i % RR);
        Prot[i] = (e / R == e % R) ? 1.f : 0.f;
      }
    return;
  }
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e % R;
    H[e] = a == b ? 1.f : 0.f;
    HtH[e] = a == b ? 1.0 : 0.0;
    WtW[e] = (double)K;
  }
}

// ------------------------------------------------------- output helpers ----
// Tk (K x R x R) = Upol_k H.
__global__ void k_upol_h(int K, int R, const float* __restrict__ Upol, const float* __restrict__ H,
                         float* __restrict__ Tk) {
  const int RR = R * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)K * RR;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / RR;
    const int a = (int)(i % RR) / R, b = (int)(i % RR) % R;
    const float* u = Upol + k * RR;
    float s = 0.f;
    for (int m = 0; m < R; ++m) s = fmaf(u[a * R + m], H[m * R + b], s);
    Tk[i] = s;
  }
}

// Squared error through the exact stage-1 identity, one warp per slice:
//   ||X_k||^2 - 2 tr(P_k Upol_k H S_k) + ||A_k Upol_k H S_k V^T||^2,
// P_k = V^T M_k (R x R) with M_k = X_k^T A_k.  The last term is
// sum_ab (S Y1^T G_k Y1 S)_ab (V^T V)_ab, Y1 = Upol_k H, with G_k = A_k^T A_k
// (FP64, pitch ldg) when AtA is given, else G_k = I (A_k orthonormal).
// Y1, G_k Y1 and the sums are FP64 (products of the stored FP32 factors):
// with nearly collinear columns of H the quadratic form in S_k cancels terms
// far larger than its value, which FP32 products would not resolve.
// Writes block partials (FP64) of the sum.
__global__ void k_fitness(int K, int R, const float* __restrict__ P, const float* __restrict__ Upol,
                          const float* __restrict__ H, const float* __restrict__ W, const double* __restrict__ VtV,
                          const double* __restrict__ xnorm2, const double* __restrict__ AtA, int ldg,
                          double* __restrict__ part) {
  extern __shared__ __align__(16) double fsm[];
  const int RR = R * R;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* hs = fsm;
  double* vv = hs + RR;
  double* my = vv + RR + warp * 3 * RR;
  double* Y1 = my;          // Upol H
  double* Pk = my + RR;
  double* GY = my + 2 * RR;  // G_k Y1 (when AtA is given)
  __shared__ double red[32];
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    hs[e] = (double)H[e];
    vv[e] = VtV[e];
  }
  __syncthreads();
  double acc = 0.0;
  for (int k = blockIdx.x * nw + warp; k < K; k += gridDim.x * nw) {
    const float* u = Upol + (int64_t)k * RR;
    const float* wk = W + (int64_t)k * R;
    for (int e = lane; e < RR; e += 32) {
      const int a = e / R, b = e % R;
      double s = 0.0;
      for (int m = 0; m < R; ++m) s = fma((double)u[a * R + m], hs[m * R + b], s);
      Y1[e] = s;
      Pk[e] = (double)P[(int64_t)k * RR + e];
    }
    __syncwarp();
    const double* Z = Y1;
    if (AtA) {
      const double* g = AtA + (int64_t)k * ldg * ldg;
      for (int e = lane; e < RR; e += 32) {
        const int i = e / R, b = e % R;
        double t = 0.0;
        for (int m = 0; m < R; ++m) t = fma(g[i * ldg + m], Y1[m * R + b], t);
        GY[e] = t;
      }
      __syncwarp();
      Z = GY;
    }
    double cross = 0.0, model = 0.0;
    for (int e = lane; e < RR; e += 32) {
      const int a = e / R, b = e % R;
      // tr(P Y1 S) = sum_{a,b} P[a][b] Y1[b][a] W[a]
      cross = fma(Pk[e] * Y1[b * R + a], (double)wk[a], cross);
      // (S Y1^T G Y1 S)[a][b] VtV[a][b]
      double g = 0.0;
      for (int i = 0; i < R; ++i) g = fma(Y1[i * R + a], Z[i * R + b], g);
      model = fma((double)wk[a] * (double)wk[b] * g, vv[e], model);
    }
    cross = warp_sum(cross);
    model = warp_sum(model);
    if (lane == 0) acc += xnorm2[k] - 2.0 * cross + model;
    __syncwarp();
  }
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// P_k (R x R) = CV^T F~_k^T for V = D CV (then V^T M_k = CV^T D^T M_k and D^T M_k = F~_k^T).
__global__ void k_p_from_cv(int K, int R, const float* __restrict__ CV, const float* __restrict__ Ft,
                            float* __restrict__ P) {
  const int RR = R * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)K * RR;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / RR;
    const int a = (int)(i % RR) / R, b = (int)(i % RR) % R;
    const float* f = Ft + k * RR;
    float s = 0.f;
    for (int m = 0; m < R; ++m) s = fmaf(CV[m * R + a], f[b * R + m], s);
    P[i] = s;
  }
}

// P_k (R x R) = V^T M_k for an arbitrary V (J x R), one block per slice; M_k
// from the three BF16 parts of M^T (column b of M_k is row k R + b of each
// part, part p at Ms + p pstride).
__global__ void k_vtm(int J, int R, const float* __restrict__ V, const __nv_bfloat16* __restrict__ Ms,
                      int64_t pstride, int Jq, float* __restrict__ P) {
  const int k = blockIdx.x, RR = R * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e % R;
    const __nv_bfloat16* m = Ms + ((int64_t)k * R + b) * Jq;
    float s = 0.f, c = 0.f;
    for (int j = 0; j < J; ++j) {
      const float mv =
          (__bfloat162float(m[j + 2 * pstride]) + __bfloat162float(m[j + pstride])) + __bfloat162float(m[j]);
      const float x = V[(int64_t)j * R + a] * mv;
      const float t = s + x;
      c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    P[(int64_t)k * RR + e] = s + c;
  }
}

// P_k (R x R) = V^T (A_k^T X_k)^T from the projection of X onto A_k, stored
// as B[k] (rows c < R of pitch Jp over j): P[a][b] = sum_j V[j][a] B[k][b][j].
// One block per slice, compensated sums over j.
__global__ void k_p_stream(int J, int Jp, int R, int LP, const float* __restrict__ V, const float* __restrict__ B,
                           float* __restrict__ P) {
  const int k = blockIdx.x, RR = R * R;
  const float* bk = B + (int64_t)k * LP * Jp;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e % R;
    float s = 0.f, c = 0.f;
    for (int j = 0; j < J; ++j) {
      const float x = V[(int64_t)j * R + a] * bk[(int64_t)b * Jp + j];
      const float t = s + x;
      c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    P[(int64_t)k * RR + e] = s + c;
  }
}

__global__ void k_reduce_f64(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    out[0] = s;
  }
}

// ---------------------------------------------------------------- launchers --
static int als_warps(int R) {
  const int per = (2 * R * (R + 1) + 4 * R * R) * 4;
  int w = (160 * 1024) / per;
  return w < 1 ? 1 : (w > ALS_WARPS ? ALS_WARPS : w);
}

int als_blocks(int K, int R, int num_sms) {
  const int nw = als_warps(R);
  const int want = (K + nw - 1) / nw;
  return std::max(1, std::min(want, 2 * num_sms));
}
static size_t qstep_smem(int R, int nw) {
  return (size_t)(2 * R * R + nw * R * R + nw * (2 * R * (R + 1) + 3 * R * R)) * sizeof(float);
}

void als_set_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_qstep, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_g2, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_g3w, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_fitness, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_update_h, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  cudaFuncSetAttribute(k_update_v, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  done = true;
}

void launch_als_init(AlsBufs& b, const float* V0, cudaStream_t s) {
  als_set_attrs();
  DP2_COUNTED(k_als_init<<<1 + 64, 256, 0, s>>>(b.K, b.J, b.R, b.D, V0, b.H, b.W, b.WtW, b.HtH, b.Psi, b.VtV, b.Prot));
  launch_atb(b.J, b.R, b.D, V0, b.Psi, b.atb, s);
  launch_atb(b.J, b.R, V0, V0, b.VtV, b.atb, s);
}

void launch_qstep_only(AlsBufs& b, cudaStream_t s) {
  const int R = b.R, nw = als_warps(R);
  if (launch_qstep_reg(b, b.part, 2 * R * R + 2, 0, s)) return;
  DP2_COUNTED(k_qstep<<<b.nblk, nw * 32, qstep_smem(R, nw), s>>>(b.K, R, b.Ft, b.Psi, b.W, b.H, b.Upol, b.Pi, b.part,
                                                     2 * R * R + 2, b.status, 0, b.rank));
}

// One iteration = 5 launches: Q-step (+ Lemma 1 partials; its extra block
// closes the previous iteration's W^T W and e and factors the H update's
// matrix), H update, Lemma 2 partials (extra block: the V update's factor),
// V update, Lemma 3 + W update (+ W^T W and e partials).  Partials use three
// separate regions.
void launch_als_iteration(AlsBufs& b, int it, cudaStream_t s) {
  const int R = b.R, RR = R * R, nw = als_warps(R);
  const int ps = 2 * RR + 2;
  float* p1 = b.part;
  float* p2 = b.part + (size_t)b.pr * ps;
  float* p3 = b.part + (size_t)2 * b.pr * ps;
  // the H update's factor (closing the previous iteration's W^T W and loss)
  // in the Q-step's extra block, the V update's in the Lemma 2 grid's
  const bool pre = b.InvH && b.InvV;
  PreSolve ph, pv;
  ph.R = pv.R = R;
  ph.part3 = it > 0 ? p3 : nullptr;
  ph.nparts = b.nblk;
  ph.pstride = ps;
  ph.it = it;
  ph.WtW = pv.WtW = b.WtW;
  ph.B = b.VtV;
  pv.B = b.HtH;
  ph.loss = b.loss;
  ph.Inv = b.InvH;
  pv.Inv = b.InvV;
  ph.L = pv.L = b.small;
  ph.V = pv.V = b.small + RR;
  ph.status = pv.status = b.status;
  bool preh = pre;
  if (!launch_qstep_reg(b, p1, ps, 1, s, pre ? &ph : nullptr)) {
    DP2_COUNTED(k_qstep<<<b.nblk, nw * 32, qstep_smem(R, nw), s>>>(b.K, R, b.Ft, b.Psi, b.W, b.H, b.Upol, b.Pi, p1, ps,
                                                       b.status, 1, b.rank));
    preh = false;
  }
  int insh = 0;
  const size_t psm = update_smem(R, &insh);
  DP2_COUNTED(k_update_h<<<1, 1024, psm, s>>>(R, p1, b.nq, p3, b.nblk, ps, it, b.WtW, b.VtV, b.H, b.HtH, b.loss, b.small,
                                 b.status, insh, preh ? b.InvH : nullptr));
  size_t g2sm = (size_t)(RR + 2 * nw * RR + nw * RR) * 4;
  if (pre) g2sm = std::max(g2sm, pre_solve_words(R, nw * 32) * sizeof(double));
  DP2_COUNTED(k_g2<<<b.nblk + (pre ? 1 : 0), nw * 32, g2sm, s>>>(b.K, R, b.Pi, b.W, b.H, p2, ps, pv, pre ? 1 : 0));
  DP2_COUNTED(k_update_v<<<1, 1024, psm, s>>>(R, p2, b.nblk, ps, b.WtW, b.HtH, b.DtD, b.CV, b.Psi, b.VtV, b.Ginv, b.small,
                               b.status, insh, pre ? b.InvV : nullptr));
  DP2_COUNTED(k_g3w<<<b.nblk, nw * 32, (size_t)RR * 8 + (size_t)(3 * RR + nw * 2 * RR + nw * (RR + 2 * R)) * 4, s>>>(
      b.K, R, b.Pi, b.Psi, b.H, b.Ginv, b.CV, b.W, p3, ps));
}

// Closes the last iteration `it`: W^T W and loss[it] from the W-update partials.
void launch_als_finish(AlsBufs& b, int it, cudaStream_t s) {
  const int R = b.R, RR = R * R, ps = b.pstride ? b.pstride : 2 * RR + 2;
  DP2_COUNTED(k_finish<<<1, 512, 0, s>>>(R, b.part + (size_t)2 * b.pr * ps, b.nblk, ps, b.WtW, b.loss, it, b.small,
                             b.status));
}

void launch_upol_h(int K, int R, const float* Upol, const float* H, float* Tk, cudaStream_t s) {
  const int64_t n = (int64_t)K * R * R;
  DP2_COUNTED(k_upol_h<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, s>>>(K, R, Upol, H, Tk));
}

void launch_p_from_cv(int K, int R, const float* CV, const float* Ft, float* P, cudaStream_t s) {
  const int64_t n = (int64_t)K * R * R;
  DP2_COUNTED(k_p_from_cv<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, s>>>(K, R, CV, Ft, P));
}

void launch_vtm(int K, int J, int R, const float* V, const void* Ms, int64_t pstride, int Jq, float* P,
                cudaStream_t s) {
  DP2_COUNTED(k_vtm<<<K, 128, 0, s>>>(J, R, V, static_cast<const __nv_bfloat16*>(Ms), pstride, Jq, P));
}

void launch_psi_vtv(int J, int R, const float* D, const float* V, double* Psi, double* VtV, float* part,
                    cudaStream_t s) {
  launch_atb(J, R, D, V, Psi, part, s);
  launch_atb(J, R, V, V, VtV, part, s);
}

void launch_atb(int64_t rows, int n, const float* A, const float* B, double* out, float* part, cudaStream_t s) {
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kAtbBlocks, (rows + ATB_ROWS - 1) / ATB_ROWS));
  const int64_t chunk = (rows + nb - 1) / nb;
  DP2_COUNTED(k_atb_part<<<nb, ATB_THREADS, 0, s>>>(rows, n, A, B, chunk, part));
  DP2_COUNTED(k_atb_fin<<<(n * n + 255) / 256, 256, 0, s>>>(nb, n * n, part, out));
}

void launch_fitness(int K, int R, const float* P, const float* Upol, const float* H, const float* W,
                    const double* VtV, const double* xnorm2, double* part, int nblk, double* out, cudaStream_t s,
                    const double* AtA, int ldg) {
  als_set_attrs();
  const int nw = R > 40 ? 1 : (R > 32 ? 2 : 4);  // (2 + 3 nw) R^2 doubles of shared memory <= 200 KB
  DP2_COUNTED(k_fitness<<<nblk, nw * 32, (size_t)(2 * R * R + nw * 3 * R * R) * 8, s>>>(K, R, P, Upol, H, W, VtV, xnorm2, AtA,
                                                                           ldg, part));
  DP2_COUNTED(k_reduce_f64<<<1, 32, 0, s>>>(part, nblk, out));
}

void launch_p_stream(int K, int J, int Jp, int R, int LP, const float* V, const float* B, float* P, cudaStream_t s) {
  DP2_COUNTED(k_p_stream<<<K, 128, 0, s>>>(J, Jp, R, LP, V, B, P));
}

}  // namespace dp2
