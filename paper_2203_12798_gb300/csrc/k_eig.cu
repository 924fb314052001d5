// Top-R eigenpairs of the l x l matrices Gt_k = M2_k^T G_k M2_k of the
// stage-1 small SVD (Alg. 1: B = Q^T X_k, B B^T = Gt_k) and of stage 2,
// register resident.
//
// Gt = L^T L (FP32 Cholesky, warp-parallel, L upper triangular).  The
// one-sided (Hestenes) Jacobi method orthogonalises the columns of F = L^T by
// plane rotations from the right: F W = Z Sigma, and Gt = F F^T = Z Sigma^2
// Z^T, so the eigenvectors are the normalised final columns and the
// eigenvalues their squared norms; the rotations themselves are not needed.
// Working on the factor keeps the condition number at that of B.
//
// Layout: one problem per warp, lane c holds column c of F (row c of L) in
// registers (N <= 32 columns; columns >= l are zero and never rotated).
// Pairs follow the cyclic round-robin ordering; the two lanes of a pair
// exchange columns with shuffles and compute the same rotation from the same
// operands.  Column norms are carried along with the rotations (Hestenes'
// update a' = a - t g, b' = b + t g) and recomputed at every sweep start.
//
// Convergence: pairs with |g| / sqrt(a b) <= tol are not rotated.  Rotating a
// pair perturbs the inner products of its columns with the others by the
// rotation angle times those inner products, so a sweep whose largest ratio
// is r leaves ratios of about sqrt(N) r^2; once r <= rstop = sqrt(tol /
// sqrt(N)) that is at the tolerance and the iteration ends without the sweep
// that would only confirm it.
#include "common.cuh"
#include "internal.h"

namespace dp2 {

constexpr int EIG_WARPS = 4;

template <int N>
__global__ void __launch_bounds__(32 * EIG_WARPS) k_eig_reg(int K, const double* __restrict__ G,
                                                            const float* __restrict__ M2, int ell, int LP, int R,
                                                            float* __restrict__ T, float* __restrict__ lam,
                                                            int* __restrict__ status) {
  constexpr int NN = N * N;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ __align__(16) float sh_a[EIG_WARPS][NN];  // G, then Gt (upper triangle), then L
  __shared__ __align__(16) float sh_m[EIG_WARPS][NN];  // M2
  __shared__ float sh_rinv[EIG_WARPS][N];
  __shared__ unsigned short pairs[N * (N + 1) / 2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * EIG_WARPS + warp;
  if (warp == 0) warp_pair_table(pairs, N);
  __syncthreads();
  if (k >= K) return;
  float* A = sh_a[warp];
  float* Ms = sh_m[warp];
  const double* g = G + (int64_t)k * LP * LP;
  const float* m2 = M2 + (int64_t)k * LP * LP;
  for (int e = lane; e < NN; e += 32) {
    const int i = e / N, c = e - i * N;
    const bool in = i < ell && c < ell;
    A[e] = in ? (float)g[i * LP + c] : 0.f;
    Ms[e] = in ? m2[i * LP + c] : 0.f;
  }
  __syncwarp();
  const bool act = lane < N;
  // column `lane` of G M2, then of Gt = M2^T (G M2) (only its upper part is used)
  float w[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float s = 0.f;
    if (act) {
#pragma unroll 8
      for (int q = 0; q < N; ++q) s = fmaf(A[i * N + q], Ms[q * N + lane], s);
    }
    w[i] = s;
  }
  __syncwarp();
  float dg = 0.f;
  if (act) {
#pragma unroll 4
    for (int a = 0; a < N; ++a) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) s = fmaf(Ms[i * N + a], w[i], s);
      A[a * N + lane] = s;
      if (a == lane) dg = s;
    }
  }
  const float md = warp_max(dg);
  __syncwarp();
  const bool bad = !(md < 3.0e38f);  // non-finite or overflowing Gram
  warp_chol_upper<float>(A, N, 1e-12f * md, bad, sh_rinv[warp], pairs);

  // column `lane` of F = L^T (row `lane` of L) into registers
  float t[N];
#pragma unroll
  for (int i = 0; i < N; ++i) t[i] = (act && i >= lane) ? A[lane * N + i] : 0.f;
  const float tol = 1.2e-7f * (float)N;
  // a sweep whose largest ratio |g| / sqrt(a b) is r leaves ratios of about
  // sqrt(N) r^2 behind: below rstop that is below tol, and the sweep that
  // would only confirm it is skipped
  const float rstop = sqrtf(tol * rsqrtf((float)N));
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    float na = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) na = fmaf(t[i], t[i], na);
    float rmax = 0.f;
    for (int rr = 0; rr < N - 1; ++rr) {
      int p;
      if (lane == 0) {
        p = 1 + rr;
      } else {
        const int x = lane - 1;
        p = (x == rr) ? 0 : 1 + ((2 * rr - x + 2 * (N - 1)) % (N - 1));
      }
      const int src = act ? p : lane;
      const bool lo = lane < p;
      float tp[N];
#pragma unroll
      for (int i = 0; i < N; ++i) tp[i] = __shfl_sync(FULL, t[i], src);
      const float nb = __shfl_sync(FULL, na, src);
      // the same products in the same order in both lanes of a pair
      float gm = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) gm = fmaf(t[i], tp[i], gm);
      const float a = lo ? na : nb, b = lo ? nb : na;
      const float rel = (act && a > 0.f && b > 0.f) ? fabsf(gm) / (sqrtf(a) * sqrtf(b)) : 0.f;
      rmax = fmaxf(rmax, rel);
      if (rel > tol) {
        const float zeta = (b - a) / (2.f * gm);
        const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
        const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
        const float sg = lo ? -sn : sn;
#pragma unroll
        for (int i = 0; i + 1 < N; i += 2) rot2(t[i], t[i + 1], tp[i], tp[i + 1], cs, sg);
        if (N & 1) t[N - 1] = fmaf(cs, t[N - 1], sg * tp[N - 1]);
        na = lo ? fmaf(-tt, gm, na) : fmaf(tt, gm, na);
      }
    }
    if (warp_max(rmax) <= rstop) break;
  }
  if (sweep == 40 && lane == 0) set_status(status, ST_SWEEP_CAP);

  // eigenvalue of column `lane` and its rank (descending, ties by index)
  float ev = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) ev = fmaf(t[i], t[i], ev);
  if (!act) ev = -1.f;
  int rank = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float ej = __shfl_sync(FULL, ev, j);
    rank += (ej > ev || (ej == ev && j < lane)) ? 1 : 0;
  }
  // T_k (LP x R) column `rank` = M2 z, z the normalised column
  if (act && rank < R) {
    const float inv = ev > 0.f ? rsqrtf(ev) : 0.f;
    float* tk = T + (int64_t)k * LP * R;
    for (int i = 0; i < LP; ++i) {
      float s = 0.f;
      if (i < N) {
#pragma unroll
        for (int m = 0; m < N; ++m) s = fmaf(Ms[i * N + m], t[m], s);
      }
      tk[i * R + rank] = s * inv;
    }
    if (lam) lam[(int64_t)k * R + rank] = ev;
  }
}

// Register columns N: l itself for the common sketch widths 20 and 30, else
// LP.  Returns false when LP > 32 (no register instantiation).
bool launch_eig_reg(const double* G, const float* M2, int K, int ell, int LP, int R, float* T, float* lam,
                    int* status, cudaStream_t s) {
  const unsigned grid = (unsigned)((K + EIG_WARPS - 1) / EIG_WARPS);
#define DP2_EIG(NC) DP2_COUNTED(k_eig_reg<NC><<<grid, 32 * EIG_WARPS, 0, s>>>(K, G, M2, ell, LP, R, T, lam, status))
  if (ell == 20) { DP2_EIG(20); return true; }
  if (ell == 30) { DP2_EIG(30); return true; }
  switch (LP) {
    case 8: DP2_EIG(8); return true;
    case 16: DP2_EIG(16); return true;
    case 24: DP2_EIG(24); return true;
    case 32: DP2_EIG(32); return true;
    default: return false;
  }
#undef DP2_EIG
}

}  // namespace dp2
