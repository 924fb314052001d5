// Per-slice small dense linear algebra of the randomized SVDs (Alg. 1) and
// the stage-2 compression (Sec. III-B, Eq. matricization_svd):
//   * FP64 Gram matrices of the sketches (double-float accumulation of exact
//     FMA products, converted to FP64),
//   * CholeskyQR2 steps: FP64 Cholesky with dropping of numerically dependent
//     columns and the inverse of the triangular factor,
//   * the small SVD of B = Q^T X through the l x l Gram B B^T (one-warp
//     Jacobi eigensolver, parallel ordering) and the blocks C_k B_k of M,
//   * the stage-2 sketch / projection / factor kernels.
#include "common.cuh"
#include "internal.h"

namespace dp2 {

__device__ inline double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ----------------------------------------------------------------- Gram ----
// G_k (ell x ell, pitch LP, FP64) = Y_k^T Y_k over the rows of slice k.
constexpr int GR_THREADS = 256;
constexpr int GR_ROWS = 64;
constexpr int GR_MAXP = 9;  // ceil(64*65/2 / 256)

__global__ void __launch_bounds__(GR_THREADS) k_gram_dd(const float* __restrict__ Y, int LP,
                                                        const int64_t* __restrict__ off, int ell,
                                                        double* __restrict__ G, int nsplit) {
  extern __shared__ __align__(16) float ys[];
  const int k = blockIdx.x, tid = threadIdx.x, split = blockIdx.y;
  const int P = ell * (ell + 1) / 2;
  int pa[GR_MAXP], pb[GR_MAXP];
  DF acc[GR_MAXP];
#pragma unroll
  for (int i = 0; i < GR_MAXP; ++i) {
    int p = tid + i * GR_THREADS;
    int a = 0, b = 0;
    if (p < P) {
      while (p >= ell - a) { p -= ell - a; ++a; }
      b = a + p;
    }
    pa[i] = a;
    pb[i] = b;
    acc[i].hi = 0.f;
    acc[i].lo = 0.f;
  }
  // rows of slice k, split in nsplit contiguous ranges (one per blockIdx.y)
  const int64_t s0 = off[k], s1 = off[k + 1];
  const int64_t chunk = round_up64((s1 - s0 + nsplit - 1) / nsplit, GR_ROWS);
  const int64_t r0 = min64(s1, s0 + split * chunk), r1 = min64(s1, r0 + chunk);
  for (int64_t rs = r0; rs < r1; rs += GR_ROWS) {
    const int nr = (int)min64(GR_ROWS, r1 - rs);
    __syncthreads();
    for (int p = tid; p < nr * LP / 4; p += GR_THREADS)
      reinterpret_cast<float4*>(ys)[p] = reinterpret_cast<const float4*>(Y + rs * LP)[p];
    __syncthreads();
    for (int i = 0; i < nr; ++i) {
      const float* yr = ys + i * LP;
#pragma unroll
      for (int q = 0; q < GR_MAXP; ++q)
        if (tid + q * GR_THREADS < P) df_mac(acc[q], yr[pa[q]], yr[pb[q]]);
    }
  }
  double* g = G + ((int64_t)k * nsplit + split) * LP * LP;
#pragma unroll
  for (int q = 0; q < GR_MAXP; ++q) {
    if (tid + q * GR_THREADS < P) {
      const double v = df_value(acc[q]);
      g[pa[q] * LP + pb[q]] = v;
      g[pb[q] * LP + pa[q]] = v;
    }
  }
}

// ------------------------------------------------------- Cholesky (drop) ----
// G = R^T R column by column (R upper triangular, FP64).  A pivot
// d_j = G_jj - sum_i R_ij^2 <= tau * max_i G_ii marks column j as numerically
// dependent on the columns before it: its row of R is zero and it is left
// out of Q.  Output Minv (LP x LP float) = pseudo-inverse of R (zero rows and
// columns at dropped indices), so that Q = Y Minv has orthonormal columns on
// the kept index set and zero columns elsewhere.
__global__ void __launch_bounds__(32) k_chol_drop(const double* __restrict__ G, int ell, int LP, double tau,
                                                  float* __restrict__ Minv, int* __restrict__ rank,
                                                  int* __restrict__ status) {
  extern __shared__ __align__(16) double sh[];
  double* Rm = sh;              // ell x ell
  double* Mi = sh + ell * ell;  // ell x ell
  __shared__ int dropped[kMaxEll];
  const int k = blockIdx.x, lane = threadIdx.x;
  const double* g = G + (int64_t)k * LP * LP;
  double md = 0.0;
  bool bad = false;
  for (int i = lane; i < ell; i += 32) {
    const double v = g[i * LP + i];
    if (!isfinite(v)) bad = true;
    md = fmax(md, v);
  }
  md = warp_max_d(md);
  bad = __any_sync(0xffffffffu, bad);
  for (int j = 0; j < ell; ++j) {
    double s = 0.0;
    for (int i = lane; i < j; i += 32) s += Rm[i * ell + j] * Rm[i * ell + j];
    s = warp_sum(s);
    const double d = g[j * LP + j] - s;
    const bool drop = !(d > tau * md) || bad;
    const double rjj = drop ? 0.0 : sqrt(d);
    if (lane == 0) {
      dropped[j] = drop;
      Rm[j * ell + j] = rjj;
    }
    for (int c = j + 1 + lane; c < ell; c += 32) {
      double t = 0.0;
      if (!drop) {
        t = g[j * LP + c];
        for (int i = 0; i < j; ++i) t -= Rm[i * ell + j] * Rm[i * ell + c];
        t /= rjj;
      }
      Rm[j * ell + c] = t;
    }
    __syncwarp();
  }
  for (int c = lane; c < ell; c += 32) {
    for (int i = ell - 1; i >= 0; --i) {
      double v = 0.0;
      if (i <= c && !dropped[c] && !dropped[i]) {
        v = (i == c) ? 1.0 : 0.0;
        for (int m = i + 1; m <= c; ++m) v -= Rm[i * ell + m] * Mi[m * ell + c];
        v /= Rm[i * ell + i];
      }
      Mi[i * ell + c] = v;
    }
  }
  __syncwarp();
  float* out = Minv + (int64_t)k * LP * LP;
  for (int e = lane; e < LP * LP; e += 32) {
    const int i = e / LP, c = e % LP;
    out[e] = (i < ell && c < ell) ? (float)Mi[i * ell + c] : 0.f;
  }
  int nd = 0;
  for (int j = lane; j < ell; j += 32) nd += dropped[j];
  nd = __reduce_add_sync(0xffffffffu, nd);
  if (lane == 0) {
    if (rank) rank[k] = ell - nd;
    if (nd) set_status(status, ST_RANK_DROP);
    if (bad) set_status(status, ST_NONFINITE);
  }
}

// ------------------------------------------------------------- Q = Y Minv ----
template <int LP>
__global__ void __launch_bounds__(128) k_formq(float* __restrict__ Y, const int64_t* __restrict__ off,
                                               const float* __restrict__ Minv) {
  __shared__ __align__(16) float ms[LP * LP];
  const int k = blockIdx.y;
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) ms[e] = Minv[(int64_t)k * LP * LP + e];
  __syncthreads();
  const int64_t row = off[k] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= off[k + 1]) return;
  float y[LP], q[LP];
#pragma unroll
  for (int c4 = 0; c4 < LP / 4; ++c4) {
    float4 v = reinterpret_cast<const float4*>(Y + row * LP)[c4];
    y[4 * c4] = v.x; y[4 * c4 + 1] = v.y; y[4 * c4 + 2] = v.z; y[4 * c4 + 3] = v.w;
  }
#pragma unroll
  for (int c = 0; c < LP; ++c) q[c] = 0.f;
#pragma unroll
  for (int i = 0; i < LP; ++i)
#pragma unroll
    for (int c = 0; c < LP; ++c) q[c] = fmaf(y[i], ms[i * LP + c], q[c]);
#pragma unroll
  for (int c4 = 0; c4 < LP / 4; ++c4)
    reinterpret_cast<float4*>(Y + row * LP)[c4] = make_float4(q[4 * c4], q[4 * c4 + 1], q[4 * c4 + 2], q[4 * c4 + 3]);
}

// out[k] = sum_i part[k * n + i] in a fixed order.
__global__ void k_reduce_rows_f64(const double* __restrict__ part, int K, int n, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[(int64_t)k * n + i];
  out[k] = s;
}

// -------------------------------------------------------- Gram of B1 rows ----
// G_k (LP x LP, FP64) = B1_k B1_k^T over columns j < J; B1_k is LP x Jp.
// Threads own 4x4 tiles of the upper triangle; thread groups split the columns.
constexpr int GB_THREADS = 256;
constexpr int GB_CJ = 64;

template <int LP>
__global__ void __launch_bounds__(GB_THREADS) k_gram_b1(const float* __restrict__ B1, int Jp, int J,
                                                        double* __restrict__ G) {
  constexpr int T = LP / 4;
  constexpr int NT = T * (T + 1) / 2;
  constexpr int NG = GB_THREADS / NT > 0 ? GB_THREADS / NT : 1;
  __shared__ __align__(16) float bs[GB_CJ][LP + 4];
  __shared__ float red[NG > 1 ? NG : 1][LP][LP + 1];
  const int k = blockIdx.x, tid = threadIdx.x;
  const int grp = tid / NT, tt = tid % NT;
  int ta = 0, tb = 0;
  {
    int p = tt;
    while (p >= T - ta) { p -= T - ta; ++ta; }
    tb = ta + p;
  }
  const bool act = grp < NG;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  const float* src = B1 + (int64_t)k * LP * Jp;
  for (int j0 = 0; j0 < J; j0 += GB_CJ) {
    __syncthreads();
    for (int e = tid; e < LP * GB_CJ; e += GB_THREADS) {
      const int c = e / GB_CJ, jj = e % GB_CJ;
      bs[jj][c] = (j0 + jj < J) ? src[(int64_t)c * Jp + j0 + jj] : 0.f;
    }
    __syncthreads();
    if (act) {
      for (int jj = grp; jj < GB_CJ; jj += NG) {
        const float4 va = *reinterpret_cast<const float4*>(&bs[jj][4 * ta]);
        const float4 vb = *reinterpret_cast<const float4*>(&bs[jj][4 * tb]);
        const float xa[4] = {va.x, va.y, va.z, va.w};
        const float xb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], xb[b], acc[a][b]);
      }
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) red[NG > 1 ? grp : 0][4 * ta + a][4 * tb + b] = acc[a][b];
  }
  __syncthreads();
  double* g = G + (int64_t)k * LP * LP;
  for (int e = tid; e < LP * LP; e += GB_THREADS) {
    const int a = e / LP, b = e % LP;
    const int ua = min(a, b), ub = max(a, b);
    if ((ua / 4) > (ub / 4)) continue;
    double s = 0.0;
    for (int q = 0; q < NG; ++q) s += (double)red[q][ua][ub];
    // tiles on the diagonal hold both orders; off-diagonal tiles only ua < ub rows
    if ((ua / 4) == (ub / 4)) {
      s = 0.0;
      for (int q = 0; q < NG; ++q) s += (double)red[q][a][b];
    }
    g[a * LP + b] = s;
  }
}

// ------------------------------------------------------ Jacobi eigensolver ----
// Symmetric n x n matrix A (smem, pitch n+1, overwritten by its eigenvalues on
// the diagonal) and eigenvectors V (smem, pitch n+1), computed by one warp
// with the cyclic parallel ordering (round-robin pairs, n padded to even).
// Stops when the off-diagonal Frobenius norm is <= tol * ||A||_F or after
// max_sweeps sweeps (then returns false).
__device__ bool warp_jacobi_eig(float* A, float* V, int n, float tol, int max_sweeps) {
  const int lane = threadIdx.x & 31;
  const int ld = n + 1;
  const int m = n + (n & 1);  // players (one dummy when n is odd)
  for (int e = lane; e < n * n; e += 32) V[(e / n) * ld + e % n] = (e / n == e % n) ? 1.f : 0.f;
  __syncwarp();
  float fro = 0.f;
  for (int e = lane; e < n * n; e += 32) fro += A[(e / n) * ld + e % n] * A[(e / n) * ld + e % n];
  fro = warp_sum(fro);
  const float thr = tol * tol * fro;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float off = 0.f;
    for (int e = lane; e < n * n; e += 32) {
      const int i = e / n, j = e % n;
      if (i != j) off += A[i * ld + j] * A[i * ld + j];
    }
    off = warp_sum(off);
    if (off <= thr || fro == 0.f) return true;
    for (int r = 0; r < m - 1; ++r) {
      // pair of this lane (lanes >= m/2 idle in the parameter phase)
      int p = -1, q = -1;
      float c = 1.f, s = 0.f;
      if (lane < m / 2) {
        if (lane == 0) {
          p = 0;
          q = 1 + (r % (m - 1));
        } else {
          p = 1 + ((r + lane) % (m - 1));
          q = 1 + ((r - lane + (m - 1)) % (m - 1));
        }
        if (p > q) { int t = p; p = q; q = t; }
        if (q < n) {
          const float apq = A[p * ld + q];
          if (apq != 0.f) {
            const float app = A[p * ld + p], aqq = A[q * ld + q];
            const float th = (aqq - app) / (2.f * apq);
            const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(1.f + th * th));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        } else {
          p = q = -1;
        }
      }
      // rows: A <- J^T A
      __syncwarp();
      for (int pi = 0; pi < m / 2; ++pi) {
        const int pp = __shfl_sync(0xffffffffu, p, pi), qq = __shfl_sync(0xffffffffu, q, pi);
        const float cc = __shfl_sync(0xffffffffu, c, pi), ss = __shfl_sync(0xffffffffu, s, pi);
        if (pp < 0 || ss == 0.f) continue;
        for (int col = lane; col < n; col += 32) {
          const float ap = A[pp * ld + col], aq = A[qq * ld + col];
          A[pp * ld + col] = cc * ap - ss * aq;
          A[qq * ld + col] = ss * ap + cc * aq;
        }
      }
      __syncwarp();
      // columns: A <- A J, V <- V J
      for (int pi = 0; pi < m / 2; ++pi) {
        const int pp = __shfl_sync(0xffffffffu, p, pi), qq = __shfl_sync(0xffffffffu, q, pi);
        const float cc = __shfl_sync(0xffffffffu, c, pi), ss = __shfl_sync(0xffffffffu, s, pi);
        if (pp < 0 || ss == 0.f) continue;
        for (int row = lane; row < n; row += 32) {
          const float ap = A[row * ld + pp], aq = A[row * ld + qq];
          A[row * ld + pp] = cc * ap - ss * aq;
          A[row * ld + qq] = ss * ap + cc * aq;
          const float vp = V[row * ld + pp], vq = V[row * ld + qq];
          V[row * ld + pp] = cc * vp - ss * vq;
          V[row * ld + qq] = ss * vp + cc * vq;
        }
      }
      __syncwarp();
    }
  }
  return false;
}

// --------------------------------------------------------- top eigenpairs ----
// For slice k: Gt = M2^T G M2 (ell x ell), eigen-decomposed; T_k (LP x R) =
// M2 U~_R with U~_R the eigenvectors of the R largest eigenvalues.  (B = M2^T
// B1 is the projected sketch Q^T X, B B^T = Gt, and A_k = Q1 T_k.)
__global__ void __launch_bounds__(32) k_eig_top(const double* __restrict__ G, const float* __restrict__ M2,
                                                int ell, int LP, int R, float* __restrict__ T,
                                                float* __restrict__ lam, int* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  const int n = ell, ld = n + 1;
  float* A = sm;               // n x ld
  float* V = A + n * ld;       // n x ld
  float* Ms = V + n * ld;      // n x n  (M2 restricted)
  float* Wt = Ms + n * n;      // n x n
  __shared__ int order[kMaxEll];
  const int k = blockIdx.x, lane = threadIdx.x;
  const double* g = G + (int64_t)k * LP * LP;
  const float* m2 = M2 + (int64_t)k * LP * LP;
  for (int e = lane; e < n * n; e += 32) Ms[e] = m2[(e / n) * LP + e % n];
  __syncwarp();
  // Wt = G M2
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, c = e % n;
    double s = 0.0;
    for (int m = 0; m < n; ++m) s += g[i * LP + m] * (double)Ms[m * n + c];
    Wt[e] = (float)s;
  }
  __syncwarp();
  // A = M2^T Wt
  for (int e = lane; e < n * n; e += 32) {
    const int a = e / n, c = e % n;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s = fmaf(Ms[i * n + a], Wt[i * n + c], s);
    A[a * ld + c] = s;
  }
  __syncwarp();
  // symmetrise
  for (int e = lane; e < n * n; e += 32) {
    const int a = e / n, c = e % n;
    if (a < c) {
      const float v = 0.5f * (A[a * ld + c] + A[c * ld + a]);
      A[a * ld + c] = v;
      A[c * ld + a] = v;
    }
  }
  __syncwarp();
  const bool ok = warp_jacobi_eig(A, V, n, 1e-7f, 40);
  if (!ok && lane == 0) set_status(status, ST_SWEEP_CAP);
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 0; i < n; ++i) {
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (A[order[j] * ld + order[j]] > A[order[best] * ld + order[best]]) best = j;
      const int t = order[i];
      order[i] = order[best];
      order[best] = t;
    }
  }
  __syncwarp();
  float* t = T + (int64_t)k * LP * R;
  for (int e = lane; e < LP * R; e += 32) {
    const int c = e / R, r = e % R;
    float s = 0.f;
    if (c < n && r < n) {
      const int col = order[r];
      for (int i = 0; i < n; ++i) s = fmaf(Ms[c * n + i], V[i * ld + col], s);
    }
    t[e] = s;
  }
  if (lam)
    for (int r = lane; r < R; r += 32) lam[(int64_t)k * R + r] = r < n ? A[order[r] * ld + order[r]] : 0.f;
}

// -------------------------------------------------------- M blocks C_k B_k ----
// M_k (J x R) = B1_k^T T_k; sigma_r = ||M_k(:, r)|| (the stage-1 singular
// values B_k); columns with sigma_r <= tau * max sigma are zeroed in M_k and
// T_k (numerical rank rule).
constexpr int MB_THREADS = 256;

template <int RB>
__global__ void __launch_bounds__(MB_THREADS) k_mblock(const float* __restrict__ B1, int Jp, int J, int ell,
                                                       int LP, int R, float* __restrict__ T,
                                                       float* __restrict__ Bk, float* __restrict__ Mblk,
                                                       int* __restrict__ rank, float tau) {
  __shared__ __align__(16) float ts[kMaxEll * RB];
  __shared__ double red[MB_THREADS / 32][RB];
  __shared__ double red2[MB_THREADS / 32][RB];
  __shared__ float keep[RB];  // 0 (dropped) or the sign +-1 of a kept component
  const int k = blockIdx.x, tid = threadIdx.x;
  float* t = T + (int64_t)k * LP * R;
  for (int e = tid; e < ell * RB; e += MB_THREADS) {
    const int c = e / RB, r = e % RB;
    ts[e] = r < R ? t[c * R + r] : 0.f;
  }
  __syncthreads();
  const float* b1 = B1 + (int64_t)k * LP * Jp;
  float nrm[RB], csum[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) nrm[r] = csum[r] = 0.f;
  for (int j = tid; j < J; j += MB_THREADS) {
    float o[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) o[r] = 0.f;
    for (int c = 0; c < ell; ++c) {
      const float b = b1[(int64_t)c * Jp + j];
#pragma unroll
      for (int r = 0; r < RB; ++r) o[r] = fmaf(b, ts[c * RB + r], o[r]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      nrm[r] = fmaf(o[r], o[r], nrm[r]);
      csum[r] += o[r];
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const float v = warp_sum(nrm[r]);
    const float c = warp_sum(csum[r]);
    if ((tid & 31) == 0) {
      red[tid >> 5][r] = v;
      red2[tid >> 5][r] = c;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double smax = 0.0;
    double sg[RB];
    for (int r = 0; r < RB; ++r) {
      double s = 0.0;
      for (int w = 0; w < MB_THREADS / 32; ++w) s += red[w][r];
      sg[r] = sqrt(s);
      if (r < R) smax = fmax(smax, sg[r]);
    }
    int rk = 0;
    for (int r = 0; r < RB; ++r) {
      // sign rule: the right singular vector (column of C_k) has a non-negative sum
      double cs = 0.0;
      for (int w = 0; w < MB_THREADS / 32; ++w) cs += red2[w][r];
      const bool kp = r < R && r < ell && sg[r] > (double)tau * smax && smax > 0.0;
      keep[r] = kp ? (cs < 0.0 ? -1.f : 1.f) : 0.f;
      if (r < R) Bk[(int64_t)k * R + r] = kp ? (float)sg[r] : 0.f;
      rk += kp;
    }
    if (rank) rank[k] = rk;
  }
  __syncthreads();
  for (int e = tid; e < LP * R; e += MB_THREADS) t[e] *= keep[e % R];
  float* mk = Mblk + (int64_t)k * J * R;
  for (int j = tid; j < J; j += MB_THREADS) {
    float o[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) o[r] = 0.f;
    for (int c = 0; c < ell; ++c) {
      const float b = b1[(int64_t)c * Jp + j];
#pragma unroll
      for (int r = 0; r < RB; ++r) o[r] = fmaf(b, ts[c * RB + r], o[r]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (r < R) mk[(int64_t)j * R + r] = o[r] * keep[r];
  }
}

// -------------------------------------------- row-segment small products ----
// Out[row] (nout) = In[row] (nin, pitch ldin) * T_seg (nin x nout, stride tstride
// per segment), segments given by offsets (K + 1).
template <int NB>
__global__ void k_seg_product(const float* __restrict__ In, int ldin, int nin, const float* __restrict__ T,
                              int64_t tstride, int nout, float* __restrict__ Out, int ldout,
                              const int64_t* __restrict__ off) {
  extern __shared__ float tsm[];  // nin x NB
  const int k = blockIdx.y;
  const float* tk = T + (int64_t)k * tstride;
  for (int e = threadIdx.x; e < nin * NB; e += blockDim.x) {
    const int c = e / NB, r = e % NB;
    tsm[e] = r < nout ? tk[c * nout + r] : 0.f;
  }
  __syncthreads();
  const int64_t row = off[k] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= off[k + 1]) return;
  const float* in = In + row * ldin;
  float o[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) o[r] = 0.f;
  for (int c = 0; c < nin; ++c) {
    const float v = in[c];
#pragma unroll
    for (int r = 0; r < NB; ++r) o[r] = fmaf(v, tsm[c * NB + r], o[r]);
  }
  float* out = Out + row * ldout;
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nout) out[r] = o[r];
}

// ---------------------------------------------------------------- stage 2 ----
// Y2 partial for a chunk of slices: Y2p[chunk] (J x LP) = sum_k M_k Omega2_k.
template <int LP>
__global__ void __launch_bounds__(128) k_s2_sketch(const float* __restrict__ Mblk, int K, int J, int R,
                                                   const float* __restrict__ om2, int kchunk,
                                                   float* __restrict__ Y2p) {
  extern __shared__ __align__(16) float os[];  // kchunk x R x LP
  const int ch = blockIdx.y;
  const int k0 = ch * kchunk, k1 = min(K, k0 + kchunk);
  for (int e = threadIdx.x; e < (k1 - k0) * R * LP; e += blockDim.x) os[e] = om2[(int64_t)k0 * R * LP + e];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  float acc[LP];
#pragma unroll
  for (int c = 0; c < LP; ++c) acc[c] = 0.f;
  for (int k = k0; k < k1; ++k) {
    const float* mk = Mblk + ((int64_t)k * J + j) * R;
    for (int r = 0; r < R; ++r) {
      const float m = mk[r];
      const float4* orow = reinterpret_cast<const float4*>(os + ((k - k0) * R + r) * LP);
#pragma unroll
      for (int c4 = 0; c4 < LP / 4; ++c4) {
        const float4 o = orow[c4];
        acc[4 * c4] = fmaf(m, o.x, acc[4 * c4]);
        acc[4 * c4 + 1] = fmaf(m, o.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(m, o.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(m, o.w, acc[4 * c4 + 3]);
      }
    }
  }
  float4* dst = reinterpret_cast<float4*>(Y2p + ((int64_t)ch * J + j) * LP);
#pragma unroll
  for (int c4 = 0; c4 < LP / 4; ++c4) dst[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
}

__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int64_t n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * n + i];
    out[i] = s;
  }
}

// B2p[(k, r)] (LP) = sum_j M_k[j][r] Q2[j][:]  (row (k, r) of B2^T).
template <int LP>
__global__ void __launch_bounds__(128) k_s2_project(const float* __restrict__ Mblk, int K, int J, int R,
                                                    const float* __restrict__ Q2, float* __restrict__ B2p) {
  __shared__ __align__(16) float qs[64 * LP];
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (k, r) flattened
  const bool act = col < (int64_t)K * R;
  const int k = act ? (int)(col / R) : 0, r = act ? (int)(col % R) : 0;
  const float* mk = Mblk + (int64_t)k * J * R + r;
  float acc[LP];
#pragma unroll
  for (int c = 0; c < LP; ++c) acc[c] = 0.f;
  for (int j0 = 0; j0 < J; j0 += 64) {
    const int nj = min(64, J - j0);
    __syncthreads();
    for (int p = threadIdx.x; p < nj * LP / 4; p += blockDim.x)
      reinterpret_cast<float4*>(qs)[p] = reinterpret_cast<const float4*>(Q2 + (int64_t)j0 * LP)[p];
    __syncthreads();
    if (act) {
      for (int jj = 0; jj < nj; ++jj) {
        const float m = mk[(int64_t)(j0 + jj) * R];
        const float4* qrow = reinterpret_cast<const float4*>(qs + jj * LP);
#pragma unroll
        for (int c4 = 0; c4 < LP / 4; ++c4) {
          const float4 q = qrow[c4];
          acc[4 * c4] = fmaf(m, q.x, acc[4 * c4]);
          acc[4 * c4 + 1] = fmaf(m, q.y, acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(m, q.z, acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(m, q.w, acc[4 * c4 + 3]);
        }
      }
    }
  }
  if (act) {
    float4* dst = reinterpret_cast<float4*>(B2p + col * LP);
#pragma unroll
    for (int c4 = 0; c4 < LP / 4; ++c4) dst[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
  }
}

// E_r = ||Ft(:, r)|| over all K R rows (F E has columns of norm E_r since F
// has orthonormal columns); columns with E_r <= tau max E are zeroed in Ft and D.
__global__ void __launch_bounds__(1024) k_s2_enorm(float* __restrict__ Ft, int64_t rows, int R,
                                                   float* __restrict__ D, int J, float* __restrict__ E, float tau) {
  __shared__ double red[1024];
  __shared__ double e2[kMaxR];
  __shared__ float keep[kMaxR];
  __shared__ int ndrop;
  const int T = blockDim.x, t = threadIdx.x;
  const int tpe = T / R;  // threads per column, rows split among them (8 loads in flight each)
  const int r = t / tpe, sub = t % tpe;
  float s = 0.f;
  if (r < R) {
    int64_t i = sub;
    for (; i + 7 * tpe < rows; i += 8 * tpe) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = Ft[(i + u * tpe) * R + r];
#pragma unroll
      for (int u = 0; u < 8; ++u) s = fmaf(v[u], v[u], s);
    }
    for (; i < rows; i += tpe) s = fmaf(Ft[i * R + r], Ft[i * R + r], s);
  }
  red[t] = s;
  __syncthreads();
  if (r < R && sub == 0) {
    double a = 0.0;
    for (int q = 0; q < tpe; ++q) a += red[t + q];
    e2[r] = a;
  }
  __syncthreads();
  if (t == 0) {
    double mx = 0.0;
    for (int c = 0; c < R; ++c) mx = fmax(mx, sqrt(e2[c]));
    ndrop = 0;
    for (int c = 0; c < R; ++c) {
      const double e = sqrt(e2[c]);
      const bool kp = e > (double)tau * mx && mx > 0.0;
      keep[c] = kp ? 1.f : 0.f;
      E[c] = kp ? (float)e : 0.f;
      ndrop += !kp;
    }
  }
  __syncthreads();
  if (ndrop) {
    for (int64_t i = t; i < rows * R; i += T) Ft[i] *= keep[i % R];
    for (int i = t; i < J * R; i += T) D[i] *= keep[i % R];
  }
}

// out (n x n, FP64) = A^T A for A (rows x n, fp32); one block.
__global__ void __launch_bounds__(256) k_ata(const float* __restrict__ A, int64_t rows, int n,
                                            double* __restrict__ out) {
  __shared__ double red[256];
  for (int e = 0; e < n * n; ++e) {
    const int a = e / n, b = e % n;
    if (b < a) continue;
    float s = 0.f;
    for (int64_t i = threadIdx.x; i < rows; i += 256) s = fmaf(A[i * n + a], A[i * n + b], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[a * n + b] = red[0];
      out[b * n + a] = red[0];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- launchers --
// G[k] (+)= sum of the nsplit partial Grams Gpart[k * nsplit + i] (fixed order).
__global__ void k_sum_splits(const double* __restrict__ Gpart, int nsplit, int K, int n, double* __restrict__ G) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)K * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / n, e = i % n;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += Gpart[(k * nsplit + q) * n + e];
    G[i] = s;
  }
}

void launch_gram_dd(const float* Y, int LP, const int64_t* d_off, int K, int ell, double* G, double* Gpart,
                    int nsplit, cudaStream_t s) {
  if (nsplit <= 1 || !Gpart) {
    k_gram_dd<<<dim3(K, 1), GR_THREADS, GR_ROWS * LP * sizeof(float), s>>>(Y, LP, d_off, ell, G, 1);
    return;
  }
  k_gram_dd<<<dim3(K, nsplit), GR_THREADS, GR_ROWS * LP * sizeof(float), s>>>(Y, LP, d_off, ell, Gpart, nsplit);
  const int n = LP * LP;
  k_sum_splits<<<(K * n + 255) / 256, 256, 0, s>>>(Gpart, nsplit, K, n, G);
}

void launch_chol_drop(const double* G, int K, int ell, int LP, double tau, float* Minv, int* rank, int* status,
                      cudaStream_t s) {
  const int smem = 2 * ell * ell * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_drop, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 8);
    attr = true;
  }
  k_chol_drop<<<K, 32, smem, s>>>(G, ell, LP, tau, Minv, rank, status);
}

void launch_formq(float* Y, int LP, const int64_t* d_off, int K, int maxI, const float* M1, cudaStream_t s) {
  dim3 grid((maxI + 127) / 128, K);
  DP2_LP_SWITCH(LP, (k_formq<L><<<grid, 128, 0, s>>>(Y, d_off, M1)));
}

void launch_reduce_rows_f64(const double* part, int K, int n, double* out, cudaStream_t s) {
  k_reduce_rows_f64<<<(K + 127) / 128, 128, 0, s>>>(part, K, n, out);
}

void launch_gram_b1(const float* B1, int Jp, int J, int K, int LP, double* G, cudaStream_t s) {
  DP2_LP_SWITCH(LP, (k_gram_b1<L><<<K, GB_THREADS, 0, s>>>(B1, Jp, J, G)));
}

void launch_eig_top(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                    int* status, cudaStream_t s) {
  const int smem = (2 * ell * (ell + 1) + 2 * ell * ell) * (int)sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_eig_top, cudaFuncAttributeMaxDynamicSharedMemorySize, (2 * 64 * 65 + 2 * 64 * 64) * 4);
    attr = true;
  }
  k_eig_top<<<K, 32, smem, s>>>(G, M2, ell, LP, R, T, lam, status);
}

void launch_mblock(const float* B1, int Jp, int J, int K, int ell, int LP, int R, float* T, float* Bk, float* Mblk,
                   int* rank, float tau, cudaStream_t s) {
  DP2_LP_SWITCH(round_up(R, 8), (k_mblock<L><<<K, MB_THREADS, 0, s>>>(B1, Jp, J, ell, LP, R, T, Bk, Mblk, rank, tau)));
}

void launch_seg_product(const float* In, int ldin, int nin, const float* T, int64_t tstride, int nout, float* Out,
                        int ldout, const int64_t* d_off, int K, int64_t maxI, cudaStream_t s) {
  dim3 grid((unsigned)((maxI + 127) / 128), K);
  const int NBr = round_up(nout, 8);
  DP2_LP_SWITCH(NBr, (k_seg_product<L><<<grid, 128, nin * L * sizeof(float), s>>>(In, ldin, nin, T, tstride, nout,
                                                                                  Out, ldout, d_off)));
}

void launch_s2_sketch(const float* Mblk, int K, int J, int R, const float* om2, int LP, float* Y2p, int kchunk,
                      cudaStream_t s) {
  const int nch = (K + kchunk - 1) / kchunk;
  dim3 grid((J + 127) / 128, nch);
  const int smem = kchunk * R * LP * (int)sizeof(float);
  DP2_LP_SWITCH(LP, (k_s2_sketch<L><<<grid, 128, smem, s>>>(Mblk, K, J, R, om2, kchunk, Y2p)));
}

void launch_sum_parts(const float* part, int nparts, int64_t n, float* out, cudaStream_t s) {
  int g = (int)min64((n + 255) / 256, 4096);
  k_sum_parts<<<g < 1 ? 1 : g, 256, 0, s>>>(part, nparts, n, out);
}

void launch_s2_project(const float* Mblk, int K, int J, int R, const float* Q2, int LP, float* B2p, cudaStream_t s) {
  const int64_t cols = (int64_t)K * R;
  DP2_LP_SWITCH(LP, (k_s2_project<L><<<(unsigned)((cols + 127) / 128), 128, 0, s>>>(Mblk, K, J, R, Q2, B2p)));
}

void launch_s2_enorm(float* Ft, int64_t rows, int R, float* D, int J, float* E, float tau, cudaStream_t s) {
  k_s2_enorm<<<1, (1024 / R) * R, 0, s>>>(Ft, rows, R, D, J, E, tau);
}

void launch_ata(const float* A, int64_t rows, int n, double* out, cudaStream_t s) {
  k_ata<<<1, 256, 0, s>>>(A, rows, n, out);
}

}  // namespace dp2
