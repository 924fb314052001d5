// Q-step of the ALS iterations (Alg. 3 first inner loop; Eq. q_k), register
// resident: for every slice k
//   T_k = F~_k Psi S_k H^T  (R x R),  T_k = Z_k Sigma_k P_k^T  (one-sided Jacobi),
//   Upol_k = Z_k P_k^T,  Pi_k = Upol_k^T F~_k,
// plus the Lemma 1 partial sum  G1 += (Pi_k Psi) diag(W(k,:)).
//
// The per-warp work is qstep_warp (qstep_reg.cuh); this kernel runs it over
// a grid of blocks, reduces the groups' Lemma 1 slots per block and, with
// pre_on, factors the next H update's matrix in an extra block (pre_solve).
#include "common.cuh"
#include "internal.h"
#include "qstep_reg.cuh"
#include "small_solve.cuh"

namespace dp2 {

template <int R>
__global__ void __launch_bounds__(R <= 12 ? 192 : 256, R <= 12 ? 3 : 1) k_qstep_reg(int K, int Ra, const float* __restrict__ Ft,
                                                   const double* __restrict__ Psi, const float* __restrict__ W,
                                                   const float* __restrict__ H, float* __restrict__ Upol,
                                                   float* __restrict__ Pi, float* __restrict__ part, int pstride,
                                                   int* __restrict__ status, int want_g1,
                                                   float* __restrict__ Prot, const int* __restrict__ rank,
                                                   PreSolve pre, int pre_on) {
  constexpr int G = 32 / R;  // problems per warp
  constexpr int RR = R * R;
  __shared__ float ps[RR], hs[RR];
  extern __shared__ __align__(16) float sm[];  // [nw][G][3 RR] group scratch, then [nw][G][RR] G1 slots
  if (pre_on && blockIdx.x == gridDim.x - 1) {  // the H update's factor (pre_solve)
    pre_solve(pre, reinterpret_cast<double*>(sm));
    return;
  }
  const int nb = gridDim.x - pre_on;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
  float* slots = sm + (size_t)nw * G * 3 * RR;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e % R;
    const bool in = a < Ra && b < Ra;
    ps[e] = in ? (float)Psi[a * Ra + b] : 0.f;
    hs[e] = in ? H[a * Ra + b] : 0.f;
  }
  __syncthreads();
  const int RaRa = Ra * Ra;
  qstep_warp<R>(K, Ra, Ft, ps, hs, W, Upol, Pi, status, want_g1, Prot, rank, sm + (size_t)warp * G * 3 * RR,
                slots + (size_t)warp * G * RR, (int64_t)blockIdx.x * nw + warp, (int64_t)nb * nw);
  if (!want_g1) return;
  __syncthreads();
  for (int e = threadIdx.x; e < RaRa; e += blockDim.x) {
    const int i = e / Ra, cc = e % Ra;
    float s = 0.f;
    for (int q = 0; q < nw * G; ++q) s += slots[(size_t)q * RR + i * R + cc];
    part[(int64_t)blockIdx.x * pstride + e] = s;
  }
}

// Warps per block: six for R <= 12 (three resident blocks per SM at <= 112
// registers, so that K = 8000 fits one wave), else eight (shared-memory bound).
template <int R>
constexpr int qreg_warps() { return R <= 12 ? 6 : 8; }

template <int R>
static int qreg_nw() {
  constexpr int G = 32 / R;
  const size_t per_warp = (size_t)G * 4 * R * R * sizeof(float);
  return (int)std::min<size_t>(qreg_warps<R>(), std::max<size_t>(1, (96 * 1024) / per_warp));
}

template <int R>
static void qreg(const AlsBufs& b, float* part, int pstride, int want_g1, cudaStream_t s, const PreSolve* pre) {
  constexpr int G = 32 / R;
  const size_t per_warp = (size_t)G * 4 * R * R * sizeof(float);
  const int nw = qreg_nw<R>();
  size_t smem = nw * per_warp;
  PreSolve p0;
  const int on = pre ? 1 : 0;
  if (pre) {
    p0 = *pre;
    smem = std::max(smem, pre_solve_words(b.R, nw * 32) * sizeof(double));
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_qstep_reg<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr = true;
  }
  DP2_COUNTED(k_qstep_reg<R><<<b.nq + on, nw * 32, smem, s>>>(b.K, b.R, b.Ft, b.Psi, b.W, b.H, b.Upol, b.Pi, part, pstride,
                                                  b.status, want_g1, b.Prot, b.rank, p0, on));
}

template <int R>
static int qblocks(int K) {
  const int per = qreg_nw<R>() * (32 / R);
  return std::max(1, (K + per - 1) / per);
}

int qstep_blocks(int K, int R, int nblk) {
  switch (R) {
    case 10: return qblocks<10>(K);
    case 20: return qblocks<20>(K);
    case 30: return qblocks<30>(K);
    default: break;
  }
  if (R <= 8) return qblocks<8>(K);
  if (R <= 16) return qblocks<16>(K);
  if (R <= 24) return qblocks<24>(K);
  if (R <= 32) return qblocks<32>(K);
  if (R <= 64) return qstep_wide_blocks(K, R, nblk);
  return nblk;  // R > 64: the shared-memory Q-step on the Lemma 2 / 3 grid
}

// Launches the register-resident Q-step when the rank has an instantiation
// (exact for R in {10, 20, 30}, zero-padded to 8, 16, 24 or 32 otherwise;
// the warp-pair kernel for 32 < R <= 64); returns false for R > 64.
bool launch_qstep_reg(const AlsBufs& b, float* part, int pstride, int want_g1, cudaStream_t s, const PreSolve* pre) {
  switch (b.R) {
    case 10: qreg<10>(b, part, pstride, want_g1, s, pre); return true;
    case 20: qreg<20>(b, part, pstride, want_g1, s, pre); return true;
    case 30: qreg<30>(b, part, pstride, want_g1, s, pre); return true;
    default: break;
  }
  if (b.R <= 8) qreg<8>(b, part, pstride, want_g1, s, pre);
  else if (b.R <= 16) qreg<16>(b, part, pstride, want_g1, s, pre);
  else if (b.R <= 24) qreg<24>(b, part, pstride, want_g1, s, pre);
  else if (b.R <= 32) qreg<32>(b, part, pstride, want_g1, s, pre);
  else return launch_qstep_wide(b, part, pstride, want_g1, s, pre);
  return true;
}

}  // namespace dp2
