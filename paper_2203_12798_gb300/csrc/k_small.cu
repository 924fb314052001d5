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
// G_k (LP x LP, FP64) = Z_k^T Z_k over the rows of slice k, the rows split in
// nsplit contiguous ranges (one per blockIdx.y, partial Grams summed after),
// with Z = Y, or with FORMQ Z = Y Minv_k written back over Y (the first
// CholeskyQR step's Q1, whose Gram is the second step's).  Double-float
// accumulation of exact products (TwoProduct + TwoSum, about 48 significant
// bits), register tiled: a thread owns a 4 x 4 tile of the upper block
// triangle of the first 4 TE columns (TE = ceil(l / 4); columns past l are
// zero) for the rows of its row group, so that two 16-byte shared-memory loads
// feed 16 products, accumulated two at a time with packed f32x2 arithmetic;
// chunks of 128 rows are staged by cp.async one chunk ahead; the row groups'
// tiles are added in a fixed order at the end.
constexpr int GT_THREADS = 256;
constexpr int GT_ROWS = 128;

template <int LP, int TE>
struct GramT {
  static constexpr int NT = TE * (TE + 1) / 2;  // tiles
  static constexpr int NG = GT_THREADS / NT;     // row groups
  static constexpr int CH = GT_ROWS * LP;        // floats per staged chunk
  static constexpr int RED = NG * NT * 16 * 2;   // floats of the group reduction
  static constexpr int stage_floats(bool formq) { return 2 * CH + (formq ? CH + LP * LP : 0); }
  static constexpr int smem(bool formq) {
    return 4 * (stage_floats(formq) > RED ? stage_floats(formq) : RED);
  }
};

template <int LP, int TE, bool FORMQ>
__global__ void __launch_bounds__(GT_THREADS) k_gram_t(float* __restrict__ Y, const int64_t* __restrict__ off,
                                                      const float* __restrict__ Minv, int ell,
                                                      double* __restrict__ G, int nsplit) {
  using C = GramT<LP, TE>;
  constexpr int NT = C::NT, NG = C::NG, CH = C::CH;
  extern __shared__ __align__(16) float gsm[];
  float* ybuf = gsm;                          // 2 x CH: staged rows of Y
  float* qbuf = gsm + 2 * CH;                 // CH: rows of Q1 (FORMQ)
  float* msm = qbuf + CH;                     // LP x LP: Minv_k (FORMQ)
  float2* red = reinterpret_cast<float2*>(gsm);  // NG x NT x 16 (after the last chunk)
  const int k = blockIdx.x, split = blockIdx.y, tid = threadIdx.x;
  const int grp = tid / NT, tt = tid % NT;
  const bool act = grp < NG;
  int ta = 0, tb = 0;
  {
    int p = tt;
    while (p >= TE - ta) {
      p -= TE - ta;
      ++ta;
    }
    tb = ta + p;
  }
  DF2 acc[4][2];  // acc[a][h]: entries (4 ta + a, 4 tb + 2 h) and (.., 4 tb + 2 h + 1)
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0].hi = acc[a][0].lo = acc[a][1].hi = acc[a][1].lo = 0ull;
  if (FORMQ)
    for (int e = tid; e < LP * LP; e += GT_THREADS) msm[e] = Minv[(int64_t)k * LP * LP + e];
  const int64_t s0 = off[k], s1 = off[k + 1];
  const int64_t chunk = round_up64((s1 - s0 + nsplit - 1) / nsplit, GT_ROWS);
  const int64_t r0 = min64(s1, s0 + split * chunk), r1 = min64(s1, r0 + chunk);
  const int nch = (int)((r1 - r0 + GT_ROWS - 1) / GT_ROWS);
  // rows rs .. rs + GT_ROWS - 1 (zero past r1) -> dst
  auto stage = [&](int64_t rs, float* dst) {
    const int nv = (int)min64(GT_ROWS, r1 - rs) * LP;
    const float* src = Y + rs * LP;
    for (int e = 4 * tid; e < CH; e += 4 * GT_THREADS) {
      const bool ok = e < nv;
      cp_async16(dst + e, ok ? src + e : Y, ok ? 16 : 0);
    }
    cp_async_commit();
  };
  if (nch > 0) stage(r0, ybuf);
  for (int c = 0; c < nch; ++c) {
    const int64_t rs = r0 + (int64_t)c * GT_ROWS;
    const int nr = (int)min64(GT_ROWS, r1 - rs);
    const float* cur = ybuf + (c & 1) * CH;
    if (c + 1 < nch) {
      stage(rs + GT_ROWS, ybuf + ((c + 1) & 1) * CH);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* z = cur;
    if (FORMQ) {
      // Q1 rows = Y rows Minv_k: two threads per row, LP / 2 columns each
      constexpr int QC = LP / 2;
      const int row = tid >> 1, cq = (tid & 1) * QC;
      float2 q[QC / 2];  // packed FP32 FMAs over column pairs
#pragma unroll
      for (int u = 0; u < QC / 2; ++u) q[u] = make_float2(0.f, 0.f);
      const float* yr = cur + row * LP;
#pragma unroll 4
      for (int i = 0; i < LP; ++i) {
        const float2 yv = make_float2(yr[i], yr[i]);
        const float4* m4 = reinterpret_cast<const float4*>(msm + i * LP + cq);
#pragma unroll
        for (int u = 0; u < QC / 4; ++u) {
          const float4 m = m4[u];
          q[2 * u] = ffma2(yv, make_float2(m.x, m.y), q[2 * u]);
          q[2 * u + 1] = ffma2(yv, make_float2(m.z, m.w), q[2 * u + 1]);
        }
      }
      float4* qo = reinterpret_cast<float4*>(qbuf + row * LP + cq);
#pragma unroll
      for (int u = 0; u < QC / 4; ++u) qo[u] = make_float4(q[2 * u].x, q[2 * u].y, q[2 * u + 1].x, q[2 * u + 1].y);
      __syncthreads();
      float4* dst = reinterpret_cast<float4*>(Y + rs * LP);
      for (int e = tid; e < nr * LP / 4; e += GT_THREADS) dst[e] = reinterpret_cast<const float4*>(qbuf)[e];
      z = qbuf;
    }
    if (act) {
      for (int i = grp; i < nr; i += NG) {
        const float4 va = *reinterpret_cast<const float4*>(z + i * LP + 4 * ta);
        const float4 vb = *reinterpret_cast<const float4*>(z + i * LP + 4 * tb);
        const float xa[4] = {va.x, va.y, va.z, va.w};
        const uint64_t b01 = f2pack(vb.x, vb.y), b23 = f2pack(vb.z, vb.w);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const uint64_t a2 = f2pack(xa[a], xa[a]), na2 = f2pack(-xa[a], -xa[a]);
          df_mac2(acc[a][0], a2, na2, b01);
          df_mac2(acc[a][1], a2, na2, b23);
        }
      }
    }
    __syncthreads();  // the chunk's buffers are refilled next
  }
  if (act) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 hi = f2unpack(acc[a][h].hi), lo = f2unpack(acc[a][h].lo);
        red[(grp * NT + tt) * 16 + 4 * a + 2 * h] = make_float2(hi.x, lo.x);
        red[(grp * NT + tt) * 16 + 4 * a + 2 * h + 1] = make_float2(hi.y, lo.y);
      }
  }
  __syncthreads();
  double* g = G + ((int64_t)k * nsplit + split) * LP * LP;
  for (int e = tid; e < NT * 16; e += GT_THREADS) {
    DF sum;
    sum.hi = sum.lo = 0.f;
    for (int gq = 0; gq < NG; ++gq) {
      const float2 v = red[gq * NT * 16 + e];
      DF d;
      d.hi = v.x;
      d.lo = v.y;
      sum = df_add(sum, d);
    }
    int p = e / 16, ua = 0;
    while (p >= TE - ua) {
      p -= TE - ua;
      ++ua;
    }
    const int a = 4 * ua + (e % 16) / 4, b = 4 * (ua + p) + e % 4;
    if (a < LP && b < LP) {
      // diagonal tiles hold (a, b) and (b, a): equal sums of equal products
      const double v = a < ell && b < ell ? df_value(sum) : 0.0;
      g[a * LP + b] = v;
      g[b * LP + a] = v;
    }
  }
  for (int e = tid; e < LP * LP; e += GT_THREADS)
    if (e / LP >= 4 * TE || e % LP >= 4 * TE) g[e] = 0.0;
}

// ------------------------------------------------------- Cholesky (drop) ----
// G = R^T R (R upper triangular) in precision T: FP64 for the first
// CholeskyQR step (the Gram of the raw sketch squares its condition number),
// FP32 for the second (the Gram of Q1 is close to the identity).  A pivot
// d_j = G_jj - sum_i R_ij^2 <= tau * max_i G_ii marks column j as numerically
// dependent on the columns before it: its row of R is zero and it is left
// out of Q.  Output Minv (LP x LP float) = pseudo-inverse of R (zero rows and
// columns at dropped indices), so that Q = Y Minv has orthonormal columns on
// the kept index set and zero columns elsewhere.  One warp per slice.
template <typename T>
__global__ void __launch_bounds__(32) k_chol_drop(const double* __restrict__ G, int ell, int LP, double tau,
                                                  float* __restrict__ Minv, int* __restrict__ rank,
                                                  int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char chol_sh[];
  T* A = reinterpret_cast<T*>(chol_sh);  // ell x ell, becomes R
  T* Mi = A + ell * ell;                  // ell x ell
  __shared__ T rinv[kMaxEll];
  __shared__ unsigned short pairs[kMaxEll * (kMaxEll + 1) / 2];
  const int k = blockIdx.x, lane = threadIdx.x;
  const double* g = G + (int64_t)k * LP * LP;
  double md = 0.0;
  bool bad = false;
  for (int e = lane; e < ell * ell; e += 32) {
    const int i = e / ell, c = e - i * ell;
    const double v = g[i * LP + c];
    if (i == c) {
      if (!isfinite(v)) bad = true;
      md = fmax(md, v);
    }
    A[e] = (T)v;
    Mi[e] = T(0);
  }
  md = warp_max_d(md);
  bad = __any_sync(0xffffffffu, bad);
  warp_pair_table(pairs, ell);
  const int nd = warp_chol_upper<T>(A, ell, (T)(tau * md), bad, rinv, pairs);
  warp_tri_inv<T>(A, ell, rinv, Mi);
  float* out = Minv + (int64_t)k * LP * LP;
  for (int e = lane; e < LP * LP; e += 32) {
    const int i = e / LP, c = e - i * LP;
    const bool in = i < ell && c < ell && !bad && rinv[i] != T(0) && rinv[c] != T(0);
    out[e] = in ? (float)Mi[i * ell + c] : 0.f;
  }
  if (lane == 0) {
    if (rank) rank[k] = ell - nd;
    if (nd) set_status(status, ST_RANK_DROP);
    if (bad) set_status(status, ST_NONFINITE);
  }
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
// G_k (LP x LP, FP64) = B1_k B1_k^T over columns j < J; B1_k is LP x Jp (rows
// >= l zero).  Threads own 4x4 tiles of the upper triangle; thread groups
// split the columns.  The next chunk of 128 (64 for l > 32) columns is loaded
// into registers while the current one is consumed from shared memory.
constexpr int GB_THREADS = 256;

template <int LP, int TE>  // TE = ceil(l / 4) tiles carry data (rows >= l of B1 are zero)
__global__ void __launch_bounds__(GB_THREADS, 4) k_gram_b1(const float* __restrict__ B1, int Jp, int J, int ell,
                                                        double* __restrict__ G) {
  constexpr int CR = 4 * TE;                   // rows of B1 staged
  // columns per chunk: as many as keep the staging buffer within 48 KB of
  // static shared memory (more loads in flight per thread)
  constexpr int GB_CJ = CR <= 24 ? 256 : (CR <= 48 ? 128 : 64);
  constexpr int NT = TE * (TE + 1) / 2;
  constexpr int NG = GB_THREADS / NT > 0 ? GB_THREADS / NT : 1;
  constexpr int PER = CR * GB_CJ / GB_THREADS;  // chunk elements per thread
  static_assert(CR * GB_CJ % GB_THREADS == 0, "chunk split");
  constexpr int BS_FLOATS = GB_CJ * (CR + 4), RED_FLOATS = (NG > 1 ? NG : 1) * CR * (CR + 1);
  // the block reduction reuses the staging buffer after the last chunk
  __shared__ __align__(16) float smem_[BS_FLOATS > RED_FLOATS ? BS_FLOATS : RED_FLOATS];
  float (*bs)[CR + 4] = reinterpret_cast<float (*)[CR + 4]>(smem_);
  float (*red)[CR][CR + 1] = reinterpret_cast<float (*)[CR][CR + 1]>(smem_);
  const int k = blockIdx.x, tid = threadIdx.x;
  const int grp = tid / NT, tt = tid % NT;
  int ta = 0, tb = 0;
  {
    int p = tt;
    while (p >= TE - ta) { p -= TE - ta; ++ta; }
    tb = ta + p;
  }
  const bool act = grp < NG;
  // acc[a][h] holds entries (4 ta + a, 4 tb + 2 h) and (.., 4 tb + 2 h + 1):
  // packed FP32 FMAs update both
  float2 acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
  const float* src = B1 + (int64_t)k * LP * Jp;
  float pre[PER];
  auto fetch = [&](int j0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * GB_THREADS;
      const int c = e / GB_CJ, jj = e % GB_CJ;
      pre[u] = (c < ell && j0 + jj < J) ? __ldg(src + (int64_t)c * Jp + j0 + jj) : 0.f;
    }
  };
  fetch(0);
  for (int j0 = 0; j0 < J; j0 += GB_CJ) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * GB_THREADS;
      bs[e % GB_CJ][e / GB_CJ] = pre[u];
    }
    __syncthreads();
    if (j0 + GB_CJ < J) fetch(j0 + GB_CJ);
    if (act) {
      for (int jj = grp; jj < GB_CJ; jj += NG) {
        const float4 va = *reinterpret_cast<const float4*>(&bs[jj][4 * ta]);
        const float4 vb = *reinterpret_cast<const float4*>(&bs[jj][4 * tb]);
        const float xa[4] = {va.x, va.y, va.z, va.w};
        const float2 b01 = make_float2(vb.x, vb.y), b23 = make_float2(vb.z, vb.w);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 aa = make_float2(xa[a], xa[a]);
          acc[a][0] = ffma2(aa, b01, acc[a][0]);
          acc[a][1] = ffma2(aa, b23, acc[a][1]);
        }
      }
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        red[NG > 1 ? grp : 0][4 * ta + a][4 * tb + b] = (b & 1) ? acc[a][b >> 1].y : acc[a][b >> 1].x;
  }
  __syncthreads();
  double* g = G + (int64_t)k * LP * LP;
  for (int e = tid; e < LP * LP; e += GB_THREADS) {
    const int a = e / LP, b = e % LP;
    float s = 0.f;
    if (a < CR && b < CR) {
      // off-diagonal tiles hold only the (ua, ub) order; diagonal tiles both
      const bool diag = (a / 4) == (b / 4);
      const int ra = diag ? a : min(a, b), rb = diag ? b : max(a, b);
#pragma unroll
      for (int q = 0; q < NG; ++q) s += red[q][ra][rb];
    }
    g[e] = (double)s;
  }
}

// ------------------------------------------------------ Jacobi eigensolver ----
// Two-sided Jacobi eigensolver for a symmetric n x n matrix A (shared memory,
// pitch n + 1) by one warp: each round of the cyclic round-robin ordering
// rotates up to n/2 disjoint (p, q) planes at once, with the rows of all
// planes, then the columns, spread over the lanes.  A is overwritten by its
// eigenvalues on the diagonal and V (pitch n + 1) by the eigenvectors.  A
// plane is left alone when |a_pq| <= tol sqrt|a_pp| sqrt|a_qq| or
// |a_pq| <= tol ||A||_F / n; a rotated a_pq is set to zero.  Stops after a
// sweep without rotations (true) or after max_sweeps (false).
struct JacobiRound {
  int p[32], q[32];
  float c[32], s[32];
};

// Only planes touching one of the `want` largest diagonal entries (at the
// start of a sweep) count towards convergence: the others mix directions
// outside the wanted leading eigenpairs, which for a rank-deficient A are
// rounding noise of zero eigenvalues that never pass the test (n <= 64).
__device__ bool warp_jacobi_eig(float* A, float* V, int n, float tol, int max_sweeps, JacobiRound& rd, int want) {
  const int lane = threadIdx.x & 31;
  const int ld = n + 1;
  const int m = n + (n & 1);  // players (one dummy when n is odd)
  const int half = m / 2;
  for (int e = lane; e < n * n; e += 32) V[(e / n) * ld + e % n] = (e / n == e % n) ? 1.f : 0.f;
  float fro = 0.f;
  for (int e = lane; e < n * n; e += 32) fro += A[(e / n) * ld + e % n] * A[(e / n) * ld + e % n];
  fro = warp_sum(fro);
  const float floor_abs = tol * sqrtf(fro) / (float)n;
  __syncwarp();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool any = false;
    unsigned long long topm = ~0ull;  // indices of the `want` largest diagonal entries
    if (want < n) {
      bool in0 = false, in1 = false;
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        bool in = false;
        if (c < n) {
          const float dc = A[c * ld + c];
          int above = 0;
          for (int j = 0; j < n; ++j) {
            const float dj = A[j * ld + j];
            above += (dj > dc || (dj == dc && j < c)) ? 1 : 0;
          }
          in = above < want;
        }
        if (h == 0) in0 = in;
        else in1 = in;
      }
      topm = ((unsigned long long)__ballot_sync(0xffffffffu, in1) << 32) | __ballot_sync(0xffffffffu, in0);
    }
    for (int r = 0; r < m - 1; ++r) {
      bool rot = false, counts = false;
      if (lane < half) {
        int p, q;
        if (lane == 0) {
          p = 0;
          q = 1 + (r % (m - 1));
        } else {
          p = 1 + ((r + lane) % (m - 1));
          q = 1 + ((r - lane + (m - 1)) % (m - 1));
        }
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < n) {
          const float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          const float mag = fabsf(apq);
          if (mag > floor_abs && mag > tol * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq))) {
            const float th = (aqq - app) / (2.f * apq);
            const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
            c = rsqrtf(fmaf(t, t, 1.f));
            s = t * c;
            rot = true;
            counts = ((topm >> p) | (topm >> q)) & 1ull;
          }
        }
        rd.p[lane] = p;
        rd.q[lane] = q;
        rd.c[lane] = c;
        rd.s[lane] = rot ? s : 0.f;
      }
      if (!__any_sync(0xffffffffu, rot)) continue;
      any |= __any_sync(0xffffffffu, counts);
      __syncwarp();
      // rows: A <- J^T A, every (plane, column) item
      for (int t = lane; t < half * n; t += 32) {
        const int pi = t / n, col = t - pi * n;
        const float ss = rd.s[pi];
        if (ss == 0.f) continue;
        const int pp = rd.p[pi], qq = rd.q[pi];
        const float cc = rd.c[pi];
        const float ap = A[pp * ld + col], aq = A[qq * ld + col];
        A[pp * ld + col] = cc * ap - ss * aq;
        A[qq * ld + col] = ss * ap + cc * aq;
      }
      __syncwarp();
      // columns: A <- A J, V <- V J, every (plane, row) item
      for (int t = lane; t < half * n; t += 32) {
        const int pi = t / n, row = t - pi * n;
        const float ss = rd.s[pi];
        if (ss == 0.f) continue;
        const int pp = rd.p[pi], qq = rd.q[pi];
        const float cc = rd.c[pi];
        const float ap = A[row * ld + pp], aq = A[row * ld + qq];
        A[row * ld + pp] = cc * ap - ss * aq;
        A[row * ld + qq] = ss * ap + cc * aq;
        const float vp = V[row * ld + pp], vq = V[row * ld + qq];
        V[row * ld + pp] = cc * vp - ss * vq;
        V[row * ld + qq] = ss * vp + cc * vq;
      }
      __syncwarp();
      if (lane < half && rot) {
        A[rd.p[lane] * ld + rd.q[lane]] = 0.f;
        A[rd.q[lane] * ld + rd.p[lane]] = 0.f;
      }
      __syncwarp();
    }
    if (!any) return true;
  }
  return false;
}

// --------------------------------------------------------- top eigenpairs ----
// For slice k: Gt = M2^T G M2 (ell x ell, FP32), eigen-decomposed; T_k (LP x R)
// = M2 U~_R with U~_R the eigenvectors of the R largest eigenvalues.  (B =
// M2^T B1 is the projected sketch Q^T X, B B^T = Gt, and A_k = Q1 T_k.)  Only
// the R leading eigenvectors are used, so FP32 products suffice: their error
// is a rounding of ||Gt|| while those eigenvalues are a sizeable part of it.
__global__ void __launch_bounds__(32) k_eig_top(const double* __restrict__ G, const float* __restrict__ M2,
                                                int ell, int LP, int R, float* __restrict__ T,
                                                float* __restrict__ lam, int* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  const int n = ell, ld = n + 1;
  float* A = sm;               // n x ld
  float* V = A + n * ld;       // n x ld
  float* Ms = V + n * ld;      // n x n  (M2 restricted)
  float* Wt = Ms + n * n;      // n x n  (G, then G M2)
  __shared__ int order[kMaxEll];
  __shared__ JacobiRound rd;
  const int k = blockIdx.x, lane = threadIdx.x;
  const double* g = G + (int64_t)k * LP * LP;
  const float* m2 = M2 + (int64_t)k * LP * LP;
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, c = e - i * n;
    Ms[e] = m2[i * LP + c];
    A[i * ld + c] = (float)g[i * LP + c];
  }
  __syncwarp();
  // Wt = G M2
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, c = e - i * n;
    float s = 0.f;
    for (int q = 0; q < n; ++q) s = fmaf(A[i * ld + q], Ms[q * n + c], s);
    Wt[e] = s;
  }
  __syncwarp();
  // A = M2^T Wt, symmetrised
  for (int e = lane; e < n * n; e += 32) {
    const int a = e / n, c = e - a * n;
    if (a > c) continue;
    float s1 = 0.f, s2 = 0.f;
    for (int i = 0; i < n; ++i) {
      s1 = fmaf(Ms[i * n + a], Wt[i * n + c], s1);
      s2 = fmaf(Ms[i * n + c], Wt[i * n + a], s2);
    }
    const float v = 0.5f * (s1 + s2);
    A[a * ld + c] = v;
    A[c * ld + a] = v;
  }
  __syncwarp();
  const bool ok = warp_jacobi_eig(A, V, n, 1e-7f, 40, rd, R < n ? R : n);
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
// M is stored for the stage-2 tensor-core passes as M^T (KR x Jq, Jq = J
// rounded up to 64) in three BF16 parts (part p at Ms + p pstride) whose sum
// is M exactly: row k R + r of each part holds column r of M_k, zero past J.
// Writes M_k(j, r) = val(j, r) for rows k R .. k R + R - 1, two columns per
// thread and store.
template <typename F>
__device__ inline void store_mt_parts(__nv_bfloat16* __restrict__ Ms, int64_t pstride, int k, int R, int J, int Jq,
                                      int tid, int nthreads, F val) {
  for (int r = 0; r < R; ++r) {
    __nv_bfloat16* d = Ms + ((int64_t)k * R + r) * Jq;
    for (int j = 2 * tid; j < Jq; j += 2 * nthreads) {
      const float v0 = j < J ? val(j, r) : 0.f, v1 = j + 1 < J ? val(j + 1, r) : 0.f;
      __nv_bfloat16 h0, m0, l0, h1, m1, l1;
      split3_bf16(v0, &h0, &m0, &l0);
      split3_bf16(v1, &h1, &m1, &l1);
      *reinterpret_cast<__nv_bfloat162*>(d + j) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(d + pstride + j) = __halves2bfloat162(m0, m1);
      *reinterpret_cast<__nv_bfloat162*>(d + 2 * pstride + j) = __halves2bfloat162(l0, l1);
    }
  }
}

// M_k (J x R) = B1_k^T T_k; sigma_r = ||M_k(:, r)|| (the stage-1 singular
// values B_k); columns with sigma_r <= tau * max sigma are zeroed in M_k and
// T_k (numerical rank rule).  Two passes over B1_k (norms and signs, then
// M_k); a shared-memory reservation caps the resident blocks at three per SM
// so that the slices being processed (~80 MB in all) stay in L2 for the
// second pass.  Every thread keeps 8 rows of B1_k in flight.
constexpr int MB_THREADS = 512;
constexpr int MB_SMEM_CAP = 64 * 1024;  // dynamic shared memory requested per block (unused)

template <int RB>
__device__ inline void mblock_col(const float* __restrict__ b1, int Jp, int j, int ell, const float* ts, float* o) {
#pragma unroll
  for (int r = 0; r < RB; ++r) o[r] = 0.f;
  for (int c0 = 0; c0 < ell; c0 += 8) {
    float b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) b[u] = (c0 + u < ell) ? __ldg(b1 + (int64_t)(c0 + u) * Jp + j) : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int r = 0; r < RB; ++r) o[r] = fmaf(b[u], ts[(c0 + u) * RB + r], o[r]);
  }
}

template <int RB>
__global__ void __launch_bounds__(MB_THREADS, RB <= 16 ? 2 : 1) k_mblock(const float* __restrict__ B1, int Jp, int J, int ell,
                                                       int LP, int R, float* __restrict__ T,
                                                       float* __restrict__ Bk, __nv_bfloat16* __restrict__ Ms,
                                                       int64_t pstride, int Jq, int* __restrict__ rank, float tau) {
  __shared__ __align__(16) float ts[kMaxEll * RB];
  __shared__ double red[MB_THREADS / 32][RB];
  __shared__ double red2[MB_THREADS / 32][RB];
  __shared__ float keep[RB];  // 0 (dropped) or the sign +-1 of a kept component
  const int k = blockIdx.x, tid = threadIdx.x;
  float* t = T + (int64_t)k * LP * R;
  const int ellp = round_up(ell, 8);
  for (int e = tid; e < ellp * RB; e += MB_THREADS) {
    const int c = e / RB, r = e % RB;
    ts[e] = (r < R && c < ell) ? t[c * R + r] : 0.f;
  }
  __syncthreads();
  const float* b1 = B1 + (int64_t)k * LP * Jp;
  float nrm[RB], csum[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) nrm[r] = csum[r] = 0.f;
  for (int j = tid; j < J; j += MB_THREADS) {
    float o[RB];
    mblock_col<RB>(b1, Jp, j, ell, ts, o);
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
  if (tid < 32) {
    // sigma_r and the column sum of component r for r = lane, lane + 32
    double sg[2] = {0.0, 0.0}, cs[2] = {0.0, 0.0};
    double smax = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = tid + 32 * h;
      if (r < RB) {
        for (int w = 0; w < MB_THREADS / 32; ++w) {
          sg[h] += red[w][r];
          cs[h] += red2[w][r];
        }
        sg[h] = sqrt(sg[h]);
        if (r < R) smax = fmax(smax, sg[h]);
      }
    }
    smax = warp_max_d(smax);
    int rk = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = tid + 32 * h;
      // sign rule: the right singular vector (column of C_k) has a non-negative sum
      const bool kp = r < R && r < ell && sg[h] > (double)tau * smax && smax > 0.0;
      if (r < RB) keep[r] = kp ? (cs[h] < 0.0 ? -1.f : 1.f) : 0.f;
      if (r < R) Bk[(int64_t)k * R + r] = kp ? (float)sg[h] : 0.f;
      rk += kp;
    }
    rk = __reduce_add_sync(0xffffffffu, rk);
    if (tid == 0 && rank) rank[k] = rk;
  }
  __syncthreads();
  for (int e = tid; e < LP * R; e += MB_THREADS) t[e] *= keep[e % R];
  // second pass over B1_k (rows L2 resident from the first): one column per
  // thread, all components, stored as the three parts of M^T
  for (int j = tid; j < Jq; j += MB_THREADS) {
    float o[RB];
    if (j < J) {
      mblock_col<RB>(b1, Jp, j, ell, ts, o);
    } else {
#pragma unroll
      for (int r = 0; r < RB; ++r) o[r] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (r < R) {
        __nv_bfloat16* d = Ms + ((int64_t)k * R + r) * Jq + j;
        split3_bf16(o[r] * keep[r], d, d + pstride, d + 2 * pstride);
      }
  }
}

// Single-pass form for M_k that fits in shared memory: every column of B1_k is
// read once (all l rows at once), M_k is kept in shared memory while its
// column norms and sums are reduced, then scaled by the keep / sign factors
// and written out as the three parts of M^T.  EB = l rounded up to 8.
constexpr int MB1_THREADS = 256;

template <int RB, int EB>
__global__ void __launch_bounds__(MB1_THREADS, 2) k_mblock1(const float* __restrict__ B1, int Jp, int J, int ell,
                                                            int LP, int R, float* __restrict__ T,
                                                            float* __restrict__ Bk, __nv_bfloat16* __restrict__ Ms,
                                                            int64_t pstride, int Jq, int* __restrict__ rank,
                                                            float tau) {
  constexpr int RP = (RB + 3) / 4 * 4;  // T_k rows padded for 16-byte loads
  extern __shared__ __align__(16) float msm[];  // J x R
  __shared__ __align__(16) float ts[EB * RP];
  __shared__ float red[MB1_THREADS / 32][RB];
  __shared__ float red2[MB1_THREADS / 32][RB];
  __shared__ float keep[RB];
  const int k = blockIdx.x, tid = threadIdx.x;
  float* t = T + (int64_t)k * LP * R;
  for (int e = tid; e < EB * RP; e += MB1_THREADS) {
    const int c = e / RP, r = e % RP;
    ts[e] = (r < R && c < ell) ? t[c * R + r] : 0.f;
  }
  __syncthreads();
  const float* b1 = B1 + (int64_t)k * LP * Jp;
  float nrm[RB], csum[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) nrm[r] = csum[r] = 0.f;
  // two columns per thread (j and j + MB1_THREADS): every T_k value read from
  // shared memory feeds two FMAs
  for (int j = tid; j < J; j += 2 * MB1_THREADS) {
    const int j2 = j + MB1_THREADS;
    const bool has2 = j2 < J;
    float b[EB], bb[EB];
#pragma unroll
    for (int c = 0; c < EB; ++c) {
      b[c] = (c < ell) ? __ldg(b1 + (int64_t)c * Jp + j) : 0.f;
      bb[c] = (c < ell && has2) ? __ldg(b1 + (int64_t)c * Jp + j2) : 0.f;
    }
    float o[RP], oo[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) o[r] = oo[r] = 0.f;
#pragma unroll
    for (int c = 0; c < EB; ++c) {
#pragma unroll
      for (int q = 0; q < RP / 4; ++q) {
        const float4 w = *reinterpret_cast<const float4*>(ts + c * RP + 4 * q);
        o[4 * q] = fmaf(b[c], w.x, o[4 * q]);
        o[4 * q + 1] = fmaf(b[c], w.y, o[4 * q + 1]);
        o[4 * q + 2] = fmaf(b[c], w.z, o[4 * q + 2]);
        o[4 * q + 3] = fmaf(b[c], w.w, o[4 * q + 3]);
        oo[4 * q] = fmaf(bb[c], w.x, oo[4 * q]);
        oo[4 * q + 1] = fmaf(bb[c], w.y, oo[4 * q + 1]);
        oo[4 * q + 2] = fmaf(bb[c], w.z, oo[4 * q + 2]);
        oo[4 * q + 3] = fmaf(bb[c], w.w, oo[4 * q + 3]);
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < R) {
        msm[j * R + r] = o[r];
        if (has2) msm[j2 * R + r] = oo[r];
      }
      nrm[r] = fmaf(o[r], o[r], fmaf(oo[r], oo[r], nrm[r]));
      csum[r] += o[r] + oo[r];
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
  if (tid < 32) {
    // FP32 suffices: sigma_r to FP32 accuracy against the 1e-5 rank threshold
    float sg[2] = {0.f, 0.f}, cs[2] = {0.f, 0.f};
    float smax = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = tid + 32 * h;
      if (r < RB) {
        for (int w = 0; w < MB1_THREADS / 32; ++w) {
          sg[h] += red[w][r];
          cs[h] += red2[w][r];
        }
        sg[h] = sqrtf(sg[h]);
        if (r < R) smax = fmaxf(smax, sg[h]);
      }
    }
    smax = warp_max(smax);
    int rk = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = tid + 32 * h;
      // sign rule: the right singular vector (column of C_k) has a non-negative sum
      const bool kp = r < R && r < ell && sg[h] > tau * smax && smax > 0.f;
      if (r < RB) keep[r] = kp ? (cs[h] < 0.f ? -1.f : 1.f) : 0.f;
      if (r < R) Bk[(int64_t)k * R + r] = kp ? sg[h] : 0.f;
      rk += kp;
    }
    rk = __reduce_add_sync(0xffffffffu, rk);
    if (tid == 0 && rank) rank[k] = rk;
  }
  __syncthreads();
  for (int e = tid; e < LP * R; e += MB1_THREADS) t[e] *= keep[e % R];
  store_mt_parts(Ms, pstride, k, R, J, Jq, tid, MB1_THREADS,
                 [&](int j, int r) { return msm[j * R + r] * keep[r]; });
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
  if ((ldin & 3) == 0 && (nin & 3) == 0 && (reinterpret_cast<uintptr_t>(In) & 15) == 0) {
    // 16-byte loads, four of them issued before their products
    const float4* in4 = reinterpret_cast<const float4*>(in);
    int c4 = 0;
    for (; c4 + 4 <= nin / 4; c4 += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = in4[c4 + u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int r = 0; r < NB; ++r) o[r] = fmaf(w[q], tsm[(4 * (c4 + u) + q) * NB + r], o[r]);
      }
    }
    for (; c4 < nin / 4; ++c4) {
      const float4 v = in4[c4];
      const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < NB; ++r) o[r] = fmaf(w[q], tsm[(4 * c4 + q) * NB + r], o[r]);
    }
  } else {
#pragma unroll 4
    for (int c = 0; c < nin; ++c) {
      const float v = in[c];
#pragma unroll
      for (int r = 0; r < NB; ++r) o[r] = fmaf(v, tsm[c * NB + r], o[r]);
    }
  }
  float* out = Out + row * ldout;
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nout) out[r] = o[r];
}

// ---------------------------------------------------------------- stage 2 ----
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int64_t n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * n + i];
    out[i] = s;
  }
}

// E_r = ||Ft(:, r)|| over all K R rows (F E has columns of norm E_r since F
// has orthonormal columns); columns with E_r <= tau max E are zeroed in Ft and
// D.  Three launches: block partials of the squared column norms, their
// fixed-order sum with the keep rule (one block), and the zeroing of dropped
// columns (a no-op unless a column was dropped).
constexpr int EN_THREADS = 256;

__global__ void __launch_bounds__(EN_THREADS) k_colnorm_part(const float* __restrict__ Ft, int64_t rows, int R,
                                                             int64_t chunk, double* __restrict__ part) {
  __shared__ float red[EN_THREADS];
  const int t = threadIdx.x;
  const int per = EN_THREADS / R;  // rows per step
  const int rr = t / R, r = t - rr * R;
  const int64_t r0 = blockIdx.x * chunk, r1 = min64(rows, r0 + chunk);
  float s = 0.f;
  if (rr < per)
    for (int64_t i = r0 + rr; i < r1; i += per) {
      const float v = Ft[i * R + r];
      s = fmaf(v, v, s);
    }
  red[t] = (rr < per) ? s : 0.f;
  __syncthreads();
  if (t < R) {
    double a = 0.0;
    for (int q = 0; q < per; ++q) a += (double)red[q * R + t];
    part[(int64_t)blockIdx.x * R + t] = a;
  }
}

__global__ void __launch_bounds__(EN_THREADS) k_enorm_fin(const double* __restrict__ part, int nb, int R,
                                                          float* __restrict__ E, float* __restrict__ keep,
                                                          int* __restrict__ ndrop, float tau) {
  __shared__ double red[EN_THREADS];
  __shared__ double e2[kMaxR];
  const int t = threadIdx.x;
  const int tpe = EN_THREADS / R;
  const int r = t / tpe, sub = t - r * tpe;
  double a = 0.0;
  if (r < R)
    for (int b = sub; b < nb; b += tpe) a += part[(int64_t)b * R + r];
  red[t] = a;
  __syncthreads();
  if (r < R && sub == 0) {
    double v = 0.0;
    for (int q = 0; q < tpe; ++q) v += red[t + q];
    e2[r] = v;
  }
  __syncthreads();
  if (t == 0) {
    double mx = 0.0;
    for (int c = 0; c < R; ++c) mx = fmax(mx, sqrt(e2[c]));
    int nd = 0;
    for (int c = 0; c < R; ++c) {
      const double e = sqrt(e2[c]);
      const bool kp = e > (double)tau * mx && mx > 0.0;
      keep[c] = kp ? 1.f : 0.f;
      E[c] = kp ? (float)e : 0.f;
      nd += !kp;
    }
    *ndrop = nd;
  }
}

__global__ void k_enorm_apply(float* __restrict__ Ft, int64_t rows, int R, float* __restrict__ D, int J,
                              const float* __restrict__ keep, const int* __restrict__ ndrop) {
  if (*ndrop == 0) return;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * R; i += nt) Ft[i] *= keep[i % R];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)J * R; i += nt) D[i] *= keep[i % R];
}

// ---------------------------------------------------------------- launchers --
// G[k] = sum of the nsplit partial Grams Gpart[k * nsplit + i]: one warp per
// entry, lanes over the splits, then a fixed-order butterfly.
__global__ void k_sum_splits(const double* __restrict__ Gpart, int nsplit, int K, int n, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= (int64_t)K * n) return;
  const int64_t k = w / n, e = w % n;
  double s = 0.0;
  for (int q = lane; q < nsplit; q += 32) s += Gpart[(k * nsplit + q) * n + e];
  s = warp_sum(s);
  if (lane == 0) G[w] = s;
}

template <int LP, int TE, bool FORMQ>
static void gram_t_launch(float* Y, const int64_t* d_off, int K, int ell, const float* Minv, double* G, int nsplit,
                          cudaStream_t s) {
  constexpr int smem = GramT<LP, TE>::smem(FORMQ);
  static bool attr = false;
  if (!attr) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_gram_t<LP, TE, FORMQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  DP2_COUNTED(k_gram_t<LP, TE, FORMQ><<<dim3(K, nsplit), GT_THREADS, smem, s>>>(Y, d_off, Minv, ell, G, nsplit));
}

// TE = ceil(ell / 4) when that is LP / 4 - 1 (LP = ell rounded up to 8),
// else LP / 4 (a Gram of fewer columns than the pitch computes the rest and
// writes zeros there)
template <int LP, bool FORMQ>
static void gram_t_dispatch(float* Y, const int64_t* d_off, int K, int ell, const float* Minv, double* G,
                            int nsplit, cudaStream_t s) {
  constexpr int T1 = LP / 4, T0 = LP / 4 > 1 ? LP / 4 - 1 : 1;
  if ((ell + 3) / 4 == T0) gram_t_launch<LP, T0, FORMQ>(Y, d_off, K, ell, Minv, G, nsplit, s);
  else gram_t_launch<LP, T1, FORMQ>(Y, d_off, K, ell, Minv, G, nsplit, s);
}

static void gram_run(float* Y, int LP, const int64_t* d_off, int K, int ell, const float* Minv, double* G,
                     int nsplit, bool formq, cudaStream_t s) {
  if (formq) {
    DP2_LP_SWITCH(LP, (gram_t_dispatch<L, true>(Y, d_off, K, ell, Minv, G, nsplit, s)));
  } else {
    DP2_LP_SWITCH(LP, (gram_t_dispatch<L, false>(Y, d_off, K, ell, Minv, G, nsplit, s)));
  }
}

void launch_gram_dd(const float* Y, int LP, const int64_t* d_off, int K, int ell, double* G, double* Gpart,
                    int nsplit, cudaStream_t s) {
  float* Yw = const_cast<float*>(Y);  // read only without FORMQ
  if (nsplit <= 1 || !Gpart) {
    gram_run(Yw, LP, d_off, K, ell, nullptr, G, 1, false, s);
    return;
  }
  gram_run(Yw, LP, d_off, K, ell, nullptr, Gpart, nsplit, false, s);
  const int64_t n = (int64_t)LP * LP, warps = (int64_t)K * n;
  DP2_COUNTED(k_sum_splits<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(Gpart, nsplit, K, (int)n, G));
}

void launch_formq_gram(float* Y, int LP, const int64_t* d_off, int K, int ell, const float* Minv, double* G,
                       double* Gpart, int nsplit, cudaStream_t s) {
  if (nsplit <= 1 || !Gpart) {
    gram_run(Y, LP, d_off, K, ell, Minv, G, 1, true, s);
    return;
  }
  gram_run(Y, LP, d_off, K, ell, Minv, Gpart, nsplit, true, s);
  const int64_t n = (int64_t)LP * LP, warps = (int64_t)K * n;
  DP2_COUNTED(k_sum_splits<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(Gpart, nsplit, K, (int)n, G));
}

void launch_chol_drop(const double* G, int K, int ell, int LP, double tau, float* Minv, int* rank, int* status,
                      bool fp64, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_chol_drop<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 8);
    attr = true;
  }
  if (fp64)
    DP2_COUNTED(k_chol_drop<double><<<K, 32, 2 * ell * ell * sizeof(double), s>>>(G, ell, LP, tau, Minv, rank, status));
  else
    DP2_COUNTED(k_chol_drop<float><<<K, 32, 2 * ell * ell * sizeof(float), s>>>(G, ell, LP, tau, Minv, rank, status));
}

void launch_reduce_rows_f64(const double* part, int K, int n, double* out, cudaStream_t s) {
  DP2_COUNTED(k_reduce_rows_f64<<<(K + 127) / 128, 128, 0, s>>>(part, K, n, out));
}

void launch_gram_b1(const float* B1, int Jp, int J, int K, int ell, int LP, double* G, cudaStream_t s) {
  if (LP == 24 && ell <= 20) {  // the common l = R + p = 20
    DP2_COUNTED(k_gram_b1<24, 5><<<K, GB_THREADS, 0, s>>>(B1, Jp, J, ell, G));
    return;
  }
  DP2_LP_SWITCH(LP, (DP2_COUNTED(k_gram_b1<L, L / 4><<<K, GB_THREADS, 0, s>>>(B1, Jp, J, ell, G))));
}

void launch_eig_top(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                    int* status, cudaStream_t s) {
  const int smem = (2 * ell * (ell + 1) + 2 * ell * ell) * (int)sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_eig_top, cudaFuncAttributeMaxDynamicSharedMemorySize, (2 * 64 * 65 + 2 * 64 * 64) * 4);
    attr = true;
  }
  if (launch_eig_reg(G, M2, K, ell, LP, R, T, lam, status, s)) return;
  if (launch_eig_wide(G, M2, K, ell, LP, R, T, lam, status, s)) return;
  DP2_COUNTED(k_eig_top<<<K, 32, smem, s>>>(G, M2, ell, LP, R, T, lam, status));
}

void launch_mblock(const float* B1, int Jp, int J, int K, int ell, int LP, int R, float* T, float* Bk, void* Ms_,
                   int64_t pstride, int Jq, int* rank, float tau, cudaStream_t s) {
  __nv_bfloat16* Ms = static_cast<__nv_bfloat16*>(Ms_);
#define DP2_MB(RB)                                                                                   \
  do {                                                                                               \
    cudaFuncSetAttribute(k_mblock<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, MB_SMEM_CAP);    \
    DP2_COUNTED(k_mblock<RB><<<K, MB_THREADS, MB_SMEM_CAP, s>>>(B1, Jp, J, ell, LP, R, T, Bk, Ms, pstride, Jq, \
                                                                 rank, tau));                        \
  } while (0)
  // single pass when M_k fits twice per SM in shared memory
  const size_t msm = (size_t)J * R * sizeof(float);
  const int eb = round_up(ell, 8);
#define DP2_MB1(RB, EB)                                                                                  \
  do {                                                                                                   \
    cudaFuncSetAttribute(k_mblock1<RB, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm);      \
    DP2_COUNTED(k_mblock1<RB, EB><<<K, MB1_THREADS, msm, s>>>(B1, Jp, J, ell, LP, R, T, Bk, Ms, pstride, Jq, rank, \
                                                              tau));                                             \
  } while (0)
  if (msm <= 100 * 1024) {
    if (R == 10 && eb == 24) { DP2_MB1(10, 24); return; }
    if (R == 20 && eb == 32) { DP2_MB1(20, 32); return; }
    if (R == 30 && eb == 40) { DP2_MB1(30, 40); return; }
  }
#undef DP2_MB1
  switch (R) {
    case 10: DP2_MB(10); return;
    case 20: DP2_MB(20); return;
    case 30: DP2_MB(30); return;
    default: break;
  }
  DP2_LP_SWITCH(round_up(R, 8), DP2_MB(L));
#undef DP2_MB
}

void launch_seg_product(const float* In, int ldin, int nin, const float* T, int64_t tstride, int nout, float* Out,
                        int ldout, const int64_t* d_off, int K, int64_t maxI, cudaStream_t s) {
  dim3 grid((unsigned)((maxI + 127) / 128), K);
  const int NBr = round_up(nout, 8);
  DP2_LP_SWITCH(NBr, (DP2_COUNTED(k_seg_product<L><<<grid, 128, nin * L * sizeof(float), s>>>(In, ldin, nin, T, tstride, nout,
                                                                                  Out, ldout, d_off))));
}

void launch_sum_parts(const float* part, int nparts, int64_t n, float* out, cudaStream_t s) {
  int g = (int)min64((n + 255) / 256, 4096);
  DP2_COUNTED(k_sum_parts<<<g < 1 ? 1 : g, 256, 0, s>>>(part, nparts, n, out));
}

void launch_s2_enorm(float* Ft, int64_t rows, int R, float* D, int J, float* E, float tau, double* part,
                     float* keep, int* ndrop, cudaStream_t s) {
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kEnormBlocks, (rows + 255) / 256));
  const int64_t chunk = (rows + nb - 1) / nb;
  DP2_COUNTED(k_colnorm_part<<<nb, EN_THREADS, 0, s>>>(Ft, rows, R, chunk, part));
  DP2_COUNTED(k_enorm_fin<<<1, EN_THREADS, 0, s>>>(part, nb, R, E, keep, ndrop, tau));
  DP2_COUNTED(k_enorm_apply<<<128, 256, 0, s>>>(Ft, rows, R, D, J, keep, ndrop));
}


}  // namespace dp2
