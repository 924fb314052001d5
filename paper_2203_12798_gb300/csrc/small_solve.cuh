// Small FP64 solves shared by the ALS kernels: partial-sum reductions, the
// pseudoinverse of the R x R Gram-Hadamard matrices of the H, V and W updates
// (Alg. 3, the normal equations of each CP-ALS step; block Gauss-Jordan, with
// Cholesky and eigen fallbacks), and
// pre_solve, which factors the matrix of the next H or V update in an extra
// block of a grid whose work it does not depend on.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace dp2 {

__device__ inline void neumaier(float& s, float& c, float v) {
  const float t = s + v;
  c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
  s = t;
}

// Two-phase reduction out[e] = sum_b part[b * pstride + e] (e < n) by the
// threads [t0, t0 + T) of the block: for n <= T every entry's partials are
// split over tpe = T / n threads, each of which keeps 16 loads in flight and
// sums them with compensation in FP32 (phase 1, into red); after a barrier the
// tpe sub-sums of an entry are added in a fixed order in FP64 (phase 2).  For
// n > T each thread sums whole entries in phase 1 (large R).
constexpr int kRedMax = 1024;
__device__ inline void par_reduce_load(const float* __restrict__ part, int nparts, int pstride, int n, int t0, int T,
                                       double* red, double* out) {
  const int t = threadIdx.x - t0;
  if (t < 0 || t >= T) return;
  if (n > T) {
    // more entries than threads: thread t sums entries t, t + T, ... over all
    // partials itself (same order for every entry) and writes them to out
    // (16 loads in flight per thread)
    for (int e = t; e < n; e += T) {
      float s = 0.f, c = 0.f;
      int b = 0;
      for (; b + 15 < nparts; b += 16) {
        float x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = part[(int64_t)(b + u) * pstride + e];
#pragma unroll
        for (int u = 0; u < 16; ++u) neumaier(s, c, x[u]);
      }
      for (; b < nparts; ++b) neumaier(s, c, part[(int64_t)b * pstride + e]);
      out[e] = (double)s + (double)c;
    }
    return;
  }
  // thread t: entry t mod n, partials t / n, t / n + tpe, ... (a warp reads
  // consecutive entries of one partial)
  const int tpe = max(1, T / n);
  const int e = t % n, sub = t / n;
  double v = 0.0;
  if (sub < tpe) {
    float s = 0.f, c = 0.f;
    int b = sub;
    for (; b + 15 * tpe < nparts; b += 16 * tpe) {
      float x[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) x[u] = part[(int64_t)(b + u * tpe) * pstride + e];
#pragma unroll
      for (int u = 0; u < 16; ++u) neumaier(s, c, x[u]);
    }
    for (; b < nparts; b += tpe) neumaier(s, c, part[(int64_t)b * pstride + e]);
    v = (double)s + (double)c;
  }
  red[t] = v;
}
// Second phase (after a barrier): entry t = sum of its threads' partial sums.
// Nothing to do when n > T (the first phase wrote out directly).
__device__ inline void par_reduce_combine(int n, int t0, int T, const double* red, double* out) {
  const int t = threadIdx.x - t0;
  if (t < 0 || t >= T || n > T) return;
  const int tpe = max(1, T / n);
  if (t >= n) return;  // thread t combines entry t
  const double* r = red + t;
  double a = 0.0, b = 0.0;
  int q = 0;
  for (; q + 1 < tpe; q += 2) {
    a += r[q * n];
    b += r[(q + 1) * n];
  }
  if (q < tpe) a += r[q * n];
  out[t] = a + b;
}

// The same two-phase reduction reading the partials as float4 quads (pstride
// a multiple of 4, part 16-byte aligned, entries n .. round_up(n, 4) - 1 of a
// partial readable): item t = (quad q = t mod nq, sub-sum s = t / nq) adds
// partials s, s + S, ... with compensation in FP32 (S = min(T / nq, nparts)
// sub-sums per quad, 8 loads in flight), so that a thread meets one or two
// rounds of L2 latency where a scalar walk over the partials meets several;
// phase 2 adds each entry's S sub-sums in order in FP64.  red4: 4 T doubles.
__device__ inline int red4_subs(int n, int nparts, int T) {
  const int nq = (n + 3) / 4;
  return max(1, min(T / nq, nparts));
}
__device__ inline void neumaier4(float4& s, float4& c, float4 v) {
  neumaier(s.x, c.x, v.x);
  neumaier(s.y, c.y, v.y);
  neumaier(s.z, c.z, v.z);
  neumaier(s.w, c.w, v.w);
}
__device__ inline void par_reduce4_load(const float* __restrict__ part, int nparts, int pstride, int n, double* red4) {
  const int T = blockDim.x, nq = (n + 3) / 4, S = red4_subs(n, nparts, T);
  for (int t = threadIdx.x; t < nq * S; t += T) {
    const int q = t % nq, s0 = t / nq;
    const float4* p4 = reinterpret_cast<const float4*>(part) + q;
    const int ps4 = pstride >> 2;
    float4 sm = make_float4(0.f, 0.f, 0.f, 0.f), cm = sm;
    // chunks of 8 partials, loads predicated, so that a thread's loads are in
    // flight together whatever nparts / S is
    for (int b = s0; b < nparts; b += 8 * S) {
      float4 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int bb = b + u * S;
        x[u] = bb < nparts ? p4[(int64_t)bb * ps4] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (b + u * S < nparts) neumaier4(sm, cm, x[u]);
    }
    double* r = red4 + 4 * (size_t)t;
    r[0] = (double)sm.x + (double)cm.x;
    r[1] = (double)sm.y + (double)cm.y;
    r[2] = (double)sm.z + (double)cm.z;
    r[3] = (double)sm.w + (double)cm.w;
  }
}
__device__ inline void par_reduce4_combine(int n, int nparts, const double* red4, double* out) {
  const int T = blockDim.x, nq = (n + 3) / 4, S = red4_subs(n, nparts, T);
  for (int e = threadIdx.x; e < n; e += T) {
    const int q = e >> 2, c = e & 3;
    double a = 0.0, b = 0.0;
    int s = 0;
    for (; s + 1 < S; s += 2) {
      a += red4[4 * (size_t)(s * nq + q) + c];
      b += red4[4 * (size_t)((s + 1) * nq + q) + c];
    }
    if (s < S) a += red4[4 * (size_t)(s * nq + q) + c];
    out[e] = a + b;
  }
}

// -------------------------------------------------------- FP64 small solves --
// Symmetric FP64 Jacobi eigendecomposition (cyclic, one thread) for the
// pseudoinverse fallback: A <- diag, V eigenvectors.
__device__ inline void jacobi_eig_f64(double* A, double* V, int n) {
  for (int i = 0; i < n * n; ++i) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-30 * tot) return;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// Inv <- A^+ for symmetric PSD A (n x n, FP64), computed by the whole block:
// Cholesky A = R^T R by warp 0 and Inv = R^-1 R^-T, or the eigen
// pseudoinverse (MATLAB tolerance n eps ||A||) when a pivot is not above
// 1e-300.  sh: shared workspace of spd_pinv_smem(n) bytes; L, V: n x n work
// arrays of the fallback.
__host__ __device__ inline size_t spd_pinv_smem(int n) {
  return (size_t)(2 * n * n + n) * sizeof(double) + (size_t)(n * (n + 1) / 2) * sizeof(unsigned short);
}
// the same in doubles, rounded up
__host__ __device__ inline size_t spd_pinv_words(int n) { return (spd_pinv_smem(n) + 7) / 8; }


// Warp 0: Cholesky A = R^T R and R^-1 (in T precision) into the workspace sh;
// returns (in warp 0) whether every pivot was above 1e-300 (FP64) / the FP32
// rounding level of A's diagonal (FP32).
template <typename T>
__device__ bool warp_spd_factor(const double* A, int n, T* sh) {
  T* Rm = sh;
  T* Mi = Rm + n * n;
  T* rinv = Mi + n * n;
  unsigned short* pairs = reinterpret_cast<unsigned short*>(rinv + n);
  T md = T(0);
  for (int e = threadIdx.x; e < n * n; e += 32) {
    Rm[e] = (T)A[e];
    Mi[e] = T(0);
    if (e / n == e % n) md = fmax(md, Rm[e]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
  warp_pair_table(pairs, n);
  const T thr = sizeof(T) == 8 ? T(1e-300) : T(64 * 1.2e-7) * md;
  const int nd = warp_chol_upper<T>(Rm, n, thr, false, rinv, pairs);
  if (nd == 0) warp_tri_inv<T>(Rm, n, rinv, Mi);
  return nd == 0;
}

// Whole block, after warp_spd_factor and a barrier: Inv = R^-1 R^-T, or (ok
// false) the eigen pseudoinverse (MATLAB tolerance n eps ||A||) of A.
template <typename T, typename OutT>
__device__ void block_spd_finish(bool ok, const double* A, OutT* Inv, double* L, double* V, int n, const T* sh,
                                 int* status) {
  const T* Mi = sh + n * n;
  if (ok) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int a = e / n, b = e - a * n;
      T s = T(0);
      for (int i = max(a, b); i < n; ++i) s = fma(Mi[a * n + i], Mi[b * n + i], s);
      Inv[e] = (OutT)s;
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    set_status(status, ST_PINV);
    for (int e = 0; e < n * n; ++e) L[e] = A[e];
    jacobi_eig_f64(L, V, n);
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(L[i * n + i]));
    const double tol = n * 2.220446049250313e-16 * mx;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
          const double l = L[i * n + i];
          if (l > tol) s += V[a * n + i] * V[b * n + i] / l;
        }
        Inv[a * n + b] = (OutT)s;
      }
  }
  __syncthreads();
}

// Inv <- A^-1 for symmetric positive definite A (n x n, n <= 32, FP64) by the
// whole block: in-place Gauss-Jordan elimination without pivoting (stable
// for SPD A) on a shared copy S (n^2 doubles).  Pivot step p maps every
// entry independently,
//   S(p, p) <- 1 / d,  S(p, j) <- S(p, j) / d,  S(i, p) <- -S(i, p) / d,
//   S(i, j) <- S(i, j) - S(i, p) S(p, j) / d      (d = S(p, p), i, j != p).
// FP64 instructions issue at a small fraction of the FP32 rate on this part
// (one warp instruction per 16 SM cycles), so the FP64 work is kept to the
// threads that own entries (entry e by thread e mod T, spread over the SM's
// sub-partitions), and the reciprocal of the next pivot (the __drcp_rn
// intrinsic) is computed once, by the thread that produces that pivot, one
// step ahead.  Returns (in every thread) whether every pivot exceeded
// 1e-300 max diag; only then is Inv (symmetrised) written.
template <int EMAX>  // entries per thread: n^2 <= EMAX blockDim.x
__device__ inline bool block_spd_inv_gj_t(const double* A, double* Inv, int n, double* S) {
  __shared__ double g_r, g_md;
  __shared__ int g_ok;
  const int nn = n * n, T = blockDim.x;
  if (T * EMAX < nn) return false;
  int ei[EMAX], ej[EMAX];  // this thread's entries (e = threadIdx.x + u T)
#pragma unroll
  for (int u = 0; u < EMAX; ++u) {
    const int e = threadIdx.x + u * T;
    ei[u] = e < nn ? e / n : -1;
    ej[u] = e < nn ? e - ei[u] * n : -1;
    if (e < nn) S[e] = A[e];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double md = 0.0;
    for (int i = 0; i < n; ++i) md = fmax(md, S[i * n + i]);
    g_md = md;
    g_ok = md > 0.0 && S[0] > 1e-300 * md;
    g_r = __drcp_rn(S[0]);
  }
  __syncthreads();
  for (int p = 0; p < n; ++p) {
    if (!g_ok) break;  // the same decision in every thread (all read the same flag)
    double nv[EMAX];
    double rn = 0.0;
    int okn = 1;
    const double r = g_r;
#pragma unroll
    for (int u = 0; u < EMAX; ++u) {
      const int i = ei[u], j = ej[u];
      if (i >= 0) {
        const double sij = S[i * n + j];
        if (i == p) nv[u] = (j == p) ? r : sij * r;
        else if (j == p) nv[u] = -sij * r;
        else nv[u] = fma(-S[i * n + p], S[p * n + j] * r, sij);
        if (i == p + 1 && j == p + 1) {  // the next pivot: its reciprocal one step ahead
          rn = __drcp_rn(nv[u]);
          okn = nv[u] > 1e-300 * g_md;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < EMAX; ++u) {
      const int i = ei[u], j = ej[u];
      if (i >= 0) {
        S[i * n + j] = nv[u];
        if (i == p + 1 && j == p + 1) {
          g_r = rn;
          g_ok = okn;
        }
      }
    }
    __syncthreads();
  }
  const bool ok = g_ok != 0;
  if (ok)
    for (int e = threadIdx.x; e < nn; e += T) {
      const int i = e / n, j = e - i * n;
      Inv[e] = 0.5 * (S[e] + S[j * n + i]);
    }
  __syncthreads();
  return ok;
}

__device__ inline bool block_spd_inv_gj(const double* A, double* Inv, int n, double* S) {
  if (n * n <= (int)blockDim.x) return block_spd_inv_gj_t<1>(A, Inv, n, S);
  if (n * n <= 2 * (int)blockDim.x) return block_spd_inv_gj_t<2>(A, Inv, n, S);
  return block_spd_inv_gj_t<8>(A, Inv, n, S);
}

// Inv <- A^+ for symmetric PSD A (n x n), computed by the whole block.
// FP64 with n <= 32: the block Gauss-Jordan inverse above; the Cholesky path
// (and its eigen pseudoinverse fallback) for larger n or when a pivot fails.
template <typename T, typename OutT>
__device__ void block_spd_pinv(const double* A, OutT* Inv, double* L, double* V, int n, T* sh, int* status) {
  __shared__ int ok;
  if constexpr (sizeof(T) == 8 && sizeof(OutT) == 8) {
    if (n <= 32 && blockDim.x * 8 >= n * n) {
      if (block_spd_inv_gj(A, reinterpret_cast<double*>(Inv), n, reinterpret_cast<double*>(sh))) return;
    }
  }
  if (threadIdx.x < 32) {
    const bool f = warp_spd_factor<T>(A, n, sh);
    if (threadIdx.x == 0) ok = f;
  }
  __syncthreads();
  block_spd_finish<T, OutT>(ok != 0, A, Inv, L, V, n, sh, status);
}

// Scale factors 1 / ||column r|| for the R columns whose squared norms are
// n2[r] (1 for a zero column); flags a non-finite norm.
__device__ inline double inv_norm(double n2, int* status) {
  if (!isfinite(n2)) set_status(status, ST_NONFINITE);
  return n2 > 0.0 ? rsqrt_nr(n2) : 1.0;
}

// Factor for the next H or V update, by the whole block: Gm = A o B with A =
// W^T W (first reduced from the W-update partials when p.part3 is given,
// together with the previous iteration's loss), Inv = Gm^+ in FP64.  The
// block runs as the extra block of the Q-step grid (H update: B = V^T V) or
// of the Lemma 2 grid (V update: B = H^T H); neither grid's other blocks read
// what it writes, so the factorisation leaves the iteration's critical path.
// sh: pre_solve_words(R, blockDim.x) doubles of shared memory.
__host__ __device__ inline size_t pre_solve_words(int R, int T) {
  return spd_pinv_words(R) + 3 * (size_t)R * R + 2 + T;
}
__device__ inline void pre_solve(const PreSolve& p, double* sh) {
  const int R = p.R, RR = R * R, T = blockDim.x;
  double* fac = sh;
  double* Gm = sh + spd_pinv_words(R);
  double* W3 = Gm + RR;
  double* red = W3 + 2 * RR + 2;  // W3: W^T W (hi, lo) and e (hi, lo)
  __shared__ int ok;
  const double* A = p.WtW;
  if (p.part3 && p.it > 0) {
    par_reduce_load(p.part3, p.nparts, p.pstride, 2 * RR + 2, 0, T, red, W3);
    __syncthreads();
    par_reduce_combine(2 * RR + 2, 0, T, red, W3);
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += T) W3[e] += W3[RR + e];
    __syncthreads();
    for (int e = threadIdx.x; e < RR + 1; e += T) {
      if (e < RR) p.WtW[e] = W3[e];
      else {
        const double v = W3[2 * RR] + W3[2 * RR + 1];
        p.loss[p.it - 1] = v;
        if (!isfinite(v)) set_status(p.status, ST_NONFINITE);
      }
    }
    A = W3;
  }
  for (int e = threadIdx.x; e < RR; e += T) Gm[e] = A[e] * p.B[e];
  __syncthreads();
  block_spd_pinv<double, double>(Gm, p.Inv, p.L, p.V, R, fac, p.status);
}

}  // namespace dp2
