// Small FP64 solves shared by the ALS kernels: partial-sum reductions, the
// Cholesky-based pseudoinverse of the R x R Gram-Hadamard matrices of the H,
// V and W updates (Alg. 3, the normal equations of each CP-ALS step), and
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

// Inv <- A^+ for symmetric PSD A (n x n), computed by the whole block.
template <typename T, typename OutT>
__device__ void block_spd_pinv(const double* A, OutT* Inv, double* L, double* V, int n, T* sh, int* status) {
  __shared__ int ok;
  if (threadIdx.x < 32) {
    const bool f = warp_spd_factor<T>(A, n, sh);
    if (threadIdx.x == 0) ok = f;
  }
  __syncthreads();
  block_spd_finish<T, OutT>(ok != 0, A, Inv, L, V, n, sh, status);
}

// Inv <- A^-1 for symmetric positive definite A (n x n, FP64), to FP64
// accuracy, by the whole block.  Warp 0 factors A in FP32 (Cholesky and
// triangular inverse, fast on the FP32 pipes); X0 = R^-1 R^-T then takes
// Newton steps X <- X + X (I - A X), the residual E = I - A X formed in FP64
// and the correction X E in FP32 (E is small, so X E needs only a few
// digits).  Each step squares the residual: from max|E0| <= 0.1 (condition
// numbers up to ~1e5 for n ~ 10) at most five steps reach max|E| <= 1e-12 or
// the FP64 rounding floor (~n kappa 1e-16), and the result is accepted when
// max|E| <= 1e-9.  Otherwise -- an FP32 pivot failed, the start was too far
// off, or the steps stalled -- the FP64 Cholesky path (block_spd_finish) runs
// instead.  Worth it for small n: the Newton products cost 2 n^3 FP64
// operations per step against the factorisation's n^3 / 3, but their FP64
// chains are n long where the Cholesky's are n rsqrt-and-update steps long.
// sh: spd_pinv_words(n) doubles (the factorisations), work:
// refined_work_words(n) doubles, both shared memory; L, V: n x n global work
// arrays of the pseudoinverse fallback.
__host__ __device__ inline size_t refined_work_words(int n) { return 2 * (size_t)n * n + 40; }

__device__ inline void block_spd_inv_refined(const double* A, double* Inv, double* L, double* V, int n, double* sh,
                                             double* work, int* status) {
  float* fsh = reinterpret_cast<float*>(sh);
  double* E = work;
  double* X = E + n * n;
  double* red = X + n * n;  // one maximum per warp
  __shared__ int ok;
  const int T = blockDim.x, nn = n * n, nwarp = (T + 31) / 32;
  if (threadIdx.x < 32) {
    const bool f = warp_spd_factor<float>(A, n, fsh);
    if (threadIdx.x == 0) ok = f;
  }
  __syncthreads();
  bool good = ok != 0 && nn <= 4 * T;
  if (good) {
    const float* Mi = fsh + nn;
    for (int e = threadIdx.x; e < nn; e += T) {  // X0 = Mi Mi^T
      const int a = e / n, b = e - a * n;
      float s = 0.f;
      for (int i = max(a, b); i < n; ++i) s = fmaf(Mi[a * n + i], Mi[b * n + i], s);
      X[e] = (double)s;
    }
    __syncthreads();
    for (int step = 0;; ++step) {
      double m = 0.0;
      for (int e = threadIdx.x; e < nn; e += T) {  // E = I - A X (FP64)
        const int a = e / n, b = e - a * n;
        double s = (a == b) ? 1.0 : 0.0;
        for (int i = 0; i < n; ++i) s = fma(-A[a * n + i], X[i * n + b], s);
        E[e] = s;
        m = fmax(m, fabs(s));
      }
      m = warp_max(m);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
      __syncthreads();
      double mm = 0.0;
      for (int w = 0; w < nwarp; ++w) mm = fmax(mm, red[w]);
      if (step == 0 && !(mm <= 0.1)) {
        good = false;
        break;
      }
      if (mm <= 1e-12 || step == 5) {
        good = mm <= 1e-9;
        break;
      }
      double xn[4];  // X + X E for this thread's entries (n^2 <= 4 T)
      int q = 0;
      for (int e = threadIdx.x; e < nn; e += T, ++q) {
        const int a = e / n, b = e - a * n;
        float s = 0.f;
        for (int i = 0; i < n; ++i) s = fmaf((float)X[a * n + i], (float)E[i * n + b], s);
        xn[q] = X[e] + (double)s;
      }
      __syncthreads();  // every thread has read X, E and red
      q = 0;
      for (int e = threadIdx.x; e < nn; e += T, ++q) X[e] = xn[q];
      __syncthreads();
    }
  }
  __syncthreads();
  if (good) {
    for (int e = threadIdx.x; e < nn; e += T) {  // symmetric part
      const int a = e / n, b = e - a * n;
      Inv[e] = 0.5 * (X[a * n + b] + X[b * n + a]);
    }
    __syncthreads();
    return;
  }
  // FP64 Cholesky (or the eigen pseudoinverse) on the same shared workspace
  if (threadIdx.x < 32) {
    const bool f = warp_spd_factor<double>(A, n, sh);
    if (threadIdx.x == 0) ok = f;
  }
  __syncthreads();
  block_spd_finish<double, double>(ok != 0, A, Inv, L, V, n, sh, status);
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
  if (threadIdx.x < 32) {
    const bool f = warp_spd_factor<double>(Gm, R, fac);
    if (threadIdx.x == 0) ok = f;
  }
  __syncthreads();
  block_spd_finish<double, double>(ok != 0, Gm, p.Inv, p.L, p.V, R, fac, p.status);
}

}  // namespace dp2
