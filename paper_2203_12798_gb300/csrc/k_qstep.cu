// Q-step of the ALS iterations (Alg. 3 first inner loop; Eq. q_k), register
// resident: for every slice k
//   T_k = F~_k Psi S_k H^T  (R x R),  T_k = Z_k Sigma_k P_k^T  (one-sided Jacobi),
//   Upol_k = Z_k P_k^T,  Pi_k = Upol_k^T F~_k,
// plus the Lemma 1 partial sum  G1 += (Pi_k Psi) diag(W(k,:)).
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
#include "common.cuh"
#include "internal.h"
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
  constexpr int M = R + (R & 1);  // round-robin players (one dummy when R is odd)
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ float ps[RR], hs[RR];
  extern __shared__ __align__(16) float sm[];  // [nw][G][3 RR] group scratch, then [nw][G][RR] G1 slots
  if (pre_on && blockIdx.x == gridDim.x - 1) {  // the H update's factor (pre_solve)
    pre_solve(pre, reinterpret_cast<double*>(sm));
    return;
  }
  const int nb = gridDim.x - pre_on;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / R, c = lane - g * R;
  const bool lane_act = g < G;
  float* gs = sm + (size_t)(warp * G + (lane_act ? g : 0)) * 3 * RR;
  float* Fs = gs;
  float* Ts = gs + RR;
  float* Ps = gs + 2 * RR;
  float* slots = sm + (size_t)nw * G * 3 * RR;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e % R;
    const bool in = a < Ra && b < Ra;
    ps[e] = in ? (float)Psi[a * Ra + b] : 0.f;
    hs[e] = in ? H[a * Ra + b] : 0.f;
  }
  __syncthreads();
  const float tol = fmaxf(1e-6f, (float)Ra * 1.2e-7f);
  // a sweep whose largest kept-pair ratio |g| / sqrt(a b) is r leaves ratios
  // of about sqrt(R) r^2 behind: below rstop that is below tol, and the
  // sweep that would only confirm it is skipped
  const float rstop = sqrtf(tol * rsqrtf((float)Ra));
  const int RaRa = Ra * Ra;
  // Lemma 1 partial of this group, column c owned by lane c (accumulated in
  // shared memory: no registers held across the sweeps)
  float* gslot = slots + (size_t)(warp * G + (lane_act ? g : 0)) * RR;
  if (lane_act) {
#pragma unroll
    for (int i = 0; i < R; ++i) gslot[i * R + c] = 0.f;
  }

  for (int64_t kb = ((int64_t)blockIdx.x * nw + warp) * G; kb < K; kb += (int64_t)nb * nw * G) {
    const int64_t k = kb + g;
    const bool act = lane_act && k < K;
    // F~_k, column c
    if (lane_act) {
#pragma unroll
      for (int i = 0; i < R; ++i) Fs[i * R + c] = (act && i < Ra && c < Ra) ? Ft[k * RaRa + i * Ra + c] : 0.f;
    }
    float wk[R];
    float wc = 0.f;  // W(k, c), picked without indexing wk by the lane's column
#pragma unroll
    for (int r = 0; r < R; ++r) {
      wk[r] = (act && r < Ra) ? W[k * Ra + r] : 0.f;
      if (r == c) wc = wk[r];
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
      for (int r = 0; r < R; ++r) s = fmaf(Ts[i * R + r], wk[r] * hs[c * R + r], s);
      t[i] = s;
    }
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
            for (int i = 0; i < R; ++i) {
              t[i] = fmaf(cs, t[i], sg * tp[i]);
              v[i] = fmaf(cs, v[i], sg * vp[i]);
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
          for (int i = 0; i < R; ++i) {
            const float tpi = __shfl_sync(FULL, t[i], src);
            const float vpi = __shfl_sync(FULL, v[i], src);
            if (rot) {
              t[i] = fmaf(cs, t[i], sg * tpi);
              v[i] = fmaf(cs, v[i], sg * vpi);
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
