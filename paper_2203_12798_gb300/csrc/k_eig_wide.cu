// Top-R eigenpairs of Gt_k = M2_k^T G_k M2_k (Alg. 1's small SVD, B B^T = Gt)
// for sketch widths 32 < l <= 64, register resident.  (k_eig_reg covers
// l <= 32 with one column per lane.)
//
// Same factorisation as k_eig_reg: FP32 Cholesky Gt = L^T L, then the
// one-sided (Hestenes) Jacobi method on F = L^T; the eigenvectors are the
// normalised final columns and the eigenvalues their squared norms.
//
// Ordering for more columns than lanes: lane i < N/2 holds a pair of columns
// (top_i, bot_i) and rotates them against each other in its own registers.
// Between rounds every column but top_0 moves one step along the ring
//   top_1 -> top_2 -> ... -> top_{H-1} -> bot_{H-1} -> ... -> bot_0 -> top_1
// (H = N/2; the round-robin tournament with one fixed player): positions on
// the ring differ by a fixed amount mod N - 1 in every pair, and the ring has
// an odd length, so after N - 1 rounds every two columns have met exactly
// once and every column is back where it started.  A move is two shuffles
// per row (the top row shifts up a lane, the bottom row down a lane).
//
// Convergence: judged on the pairs that touch one of the `want` = min(R, l)
// largest columns (ranked by norm at the sweep start; only those
// eigenvectors are used), by the rule of k_eig_reg.
#include "common.cuh"
#include "internal.h"

namespace dp2 {

constexpr int EIGW_WARPS = 2;

template <int N>
static size_t eigw_smem() {
  // per warp: A (N x N) and M2 (N x N), rinv (N); then the pair table
  return (size_t)EIGW_WARPS * (2 * N * N + N) * sizeof(float) + (size_t)(N * (N + 1) / 2) * sizeof(unsigned short);
}

// One step along the ring for a column pair held as (top[], bot[]) per lane.
template <int N, typename V>
__device__ __forceinline__ void ring_move(V& top, V& bot, int lane) {
  constexpr int H = N / 2;
  constexpr unsigned FULL = 0xffffffffu;
  const V up = __shfl_up_sync(FULL, lane == 0 ? bot : top, 1);
  const V dn = __shfl_down_sync(FULL, bot, 1);
  const V ot = top;
  if (lane != 0) top = up;
  bot = (lane == H - 1) ? ot : dn;
}

template <int N>
__global__ void __launch_bounds__(32 * EIGW_WARPS) k_eig_wide(int K, const double* __restrict__ G,
                                                              const float* __restrict__ M2, int ell, int LP, int R,
                                                              float* __restrict__ T, float* __restrict__ lam,
                                                              int* __restrict__ status) {
  static_assert(N % 2 == 0 && N > 32 && N <= 64, "32 < N <= 64, even");
  constexpr int H = N / 2;
  constexpr int NN = N * N;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) float sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* A = sm + (size_t)warp * (2 * NN + N);
  float* Ms = A + NN;
  float* rinv = Ms + NN;
  unsigned short* pairs = reinterpret_cast<unsigned short*>(sm + (size_t)EIGW_WARPS * (2 * NN + N));
  if (warp == 0) warp_pair_table(pairs, N);
  __syncthreads();
  const int k = blockIdx.x * EIGW_WARPS + warp;
  if (k >= K) return;
  const double* g = G + (int64_t)k * LP * LP;
  const float* m2 = M2 + (int64_t)k * LP * LP;
  for (int e = lane; e < NN; e += 32) {
    const int i = e / N, c = e - i * N;
    const bool in = i < ell && c < ell;
    A[e] = in ? (float)g[i * LP + c] : 0.f;
    Ms[e] = in ? m2[i * LP + c] : 0.f;
  }
  __syncwarp();
  // columns c0 = lane and c1 = lane + 32 of G M2, then of Gt = M2^T (G M2)
  const int c0 = lane, c1 = lane + 32;
  const bool has1 = c1 < N;
  float w0[N], w1[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
    for (int q = 0; q < N; ++q) {
      const float a = A[i * N + q];
      s0 = fmaf(a, Ms[q * N + c0], s0);
      if (has1) s1 = fmaf(a, Ms[q * N + c1], s1);
    }
    w0[i] = s0;
    w1[i] = s1;
  }
  __syncwarp();
  float dg = 0.f;
#pragma unroll 2
  for (int a = 0; a < N; ++a) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float m = Ms[i * N + a];
      s0 = fmaf(m, w0[i], s0);
      s1 = fmaf(m, w1[i], s1);
    }
    A[a * N + c0] = s0;
    if (has1) A[a * N + c1] = s1;
    if (a == c0) dg = fmaxf(dg, s0);
    if (has1 && a == c1) dg = fmaxf(dg, s1);
  }
  const float md = warp_max(dg);
  __syncwarp();
  const bool bad = !(md < 3.0e38f);  // non-finite or overflowing Gram
  warp_chol_upper<float>(A, N, 1e-12f * md, bad, rinv, pairs);

  // F = L^T: column j is row j of the upper-triangular L.  Lane i < H holds
  // columns i (top) and H + i (bot).
  const bool act = lane < H;
  float top[N], bot[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    top[i] = (act && i >= lane) ? A[lane * N + i] : 0.f;
    bot[i] = (act && i >= H + lane) ? A[(H + lane) * N + i] : 0.f;
  }
  const int want = R < ell ? R : ell;
  const float tol = 1.2e-7f * (float)N;
  const float rstop = sqrtf(tol * rsqrtf((float)N));  // as in k_eig_reg
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    float na = 0.f, nb = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      na = fmaf(top[i], top[i], na);
      nb = fmaf(bot[i], bot[i], nb);
    }
    // rank of the two columns among all N (descending norm, ties by index)
    int at = 0, ab = 0;
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
      const float xa = __shfl_sync(FULL, na, j), xb = __shfl_sync(FULL, nb, j);
      at += (xa > na || (xa == na && j < lane)) ? 1 : 0;
      at += (xb > na) ? 1 : 0;  // column H + j > lane: ties rank behind
      ab += (xa >= nb) ? 1 : 0;  // column j < H + lane: ties rank ahead
      ab += (xb > nb || (xb == nb && j < lane)) ? 1 : 0;
    }
    int ft = (act && at < want) ? 1 : 0, fb = (act && ab < want) ? 1 : 0;
    float rmax = 0.f;  // largest ratio over pairs touching a wanted column
    for (int rr = 0; rr < N - 1; ++rr) {
      float g0 = 0.f, g1 = 0.f;
#pragma unroll
      for (int i = 0; i < N; i += 2) {
        g0 = fmaf(top[i], bot[i], g0);
        g1 = fmaf(top[i + 1], bot[i + 1], g1);
      }
      const float gm = g0 + g1;
      const float rel = (act && na > 0.f && nb > 0.f) ? fabsf(gm) / (sqrtf(na) * sqrtf(nb)) : 0.f;
      if (ft | fb) rmax = fmaxf(rmax, rel);
      if (rel > tol) {
        const float zeta = (nb - na) / (2.f * gm);
        const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
        const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float x = top[i], y = bot[i];
          top[i] = fmaf(cs, x, -sn * y);
          bot[i] = fmaf(sn, x, cs * y);
        }
        na = fmaf(-tt, gm, na);
        nb = fmaf(tt, gm, nb);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) ring_move<N>(top[i], bot[i], lane);
      ring_move<N>(na, nb, lane);
      ring_move<N>(ft, fb, lane);
    }
    if (warp_max(rmax) <= rstop) break;
  }
  if (sweep == 40 && lane == 0) set_status(status, ST_SWEEP_CAP);

  // eigenvalues of the two columns and their ranks (descending, ties by index)
  float et = 0.f, eb = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    et = fmaf(top[i], top[i], et);
    eb = fmaf(bot[i], bot[i], eb);
  }
  int rt = 0, rb = 0;
#pragma unroll 4
  for (int j = 0; j < H; ++j) {
    const float xa = __shfl_sync(FULL, et, j), xb = __shfl_sync(FULL, eb, j);
    rt += (xa > et || (xa == et && j < lane)) ? 1 : 0;
    rt += (xb > et) ? 1 : 0;
    rb += (xa >= eb) ? 1 : 0;
    rb += (xb > eb || (xb == eb && j < lane)) ? 1 : 0;
  }
  // T_k (LP x R) column `rank` = M2 z, z the normalised column
  float* tk = T + (int64_t)k * LP * R;
  if (act && rt < R) {
    const float inv = et > 0.f ? rsqrtf(et) : 0.f;
    for (int i = 0; i < LP; ++i) {
      float s = 0.f;
      if (i < N) {
#pragma unroll
        for (int m = 0; m < N; ++m) s = fmaf(Ms[i * N + m], top[m], s);
      }
      tk[i * R + rt] = s * inv;
    }
    if (lam) lam[(int64_t)k * R + rt] = et;
  }
  if (act && rb < R) {
    const float inv = eb > 0.f ? rsqrtf(eb) : 0.f;
    for (int i = 0; i < LP; ++i) {
      float s = 0.f;
      if (i < N) {
#pragma unroll
        for (int m = 0; m < N; ++m) s = fmaf(Ms[i * N + m], bot[m], s);
      }
      tk[i * R + rb] = s * inv;
    }
    if (lam) lam[(int64_t)k * R + rb] = eb;
  }
}

template <int N>
static void eigw(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam, int* status,
                 cudaStream_t s) {
  static bool attr = false;
  const size_t smem = eigw_smem<N>();
  if (!attr) {
    cudaFuncSetAttribute(k_eig_wide<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const unsigned grid = (unsigned)((K + EIGW_WARPS - 1) / EIGW_WARPS);
  DP2_COUNTED(k_eig_wide<N><<<grid, 32 * EIGW_WARPS, smem, s>>>(K, G, M2, ell, LP, R, T, lam, status));
}

// Register columns N: l itself for the sketch widths 50 and 60, else LP.
// Returns false outside 32 < LP <= 64.
bool launch_eig_wide(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                     int* status, cudaStream_t s) {
  if (ell == 50) { eigw<50>(G, M2, K, ell, LP, R, T, lam, status, s); return true; }
  if (ell == 60) { eigw<60>(G, M2, K, ell, LP, R, T, lam, status, s); return true; }
  switch (LP) {
    case 40: eigw<40>(G, M2, K, ell, LP, R, T, lam, status, s); return true;
    case 48: eigw<48>(G, M2, K, ell, LP, R, T, lam, status, s); return true;
    case 56: eigw<56>(G, M2, K, ell, LP, R, T, lam, status, s); return true;
    case 64: eigw<64>(G, M2, K, ell, LP, R, T, lam, status, s); return true;
    default: return false;
  }
}

}  // namespace dp2
