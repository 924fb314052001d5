// Q-step of the ALS iterations (Alg. 3 first inner loop; Eq. q_k) for ranks
// 32 < R <= 64, register resident.  For every slice k
//   T_k = F~_k Psi S_k H^T  (R x R),  T_k = Z_k Sigma_k P_k^T  (one-sided Jacobi),
//   Upol_k = Z_k P_k^T over the r_k largest singular values,  Pi_k = Upol_k^T F~_k,
// plus the Lemma 1 partial sum  G1 += (Pi_k Psi) diag(W(k,:)).
// (k_qstep_reg covers R <= 32 with one column per lane.)
//
// One pair of warps per slice.  The T warp holds the columns of T_k V and the
// V warp those of V (the accumulated right rotations), in registers, in the
// ordering of k_eig_wide: lane i < R/2 holds the column pair (top_i, bot_i)
// and rotates it in its own registers; between rounds every column but top_0
// moves one step along the ring top_1 .. top_{H-1}, bot_{H-1} .. bot_0, so a
// sweep of R - 1 rounds meets every pair of columns once and ends with every
// column back in place.  The T warp computes each rotation and stores its
// (cos, sin) in shared memory, one sweep per buffer; the V warp applies a
// sweep's rotations while the T warp computes the next (two buffers, one pair
// barrier per sweep).  Splitting T and V over two warps keeps 2R values per
// thread in registers at R = 64.
//
// Warm start as in k_qstep_reg: V0 = Prot_k (the previous Q-step's right
// rotations) after one Newton-Schulz step V0 <- V0 (3 I - V0^T V0) / 2; the
// sweeps start from T_k V0.  Convergence (the rstop rule of k_eig_reg) is
// judged on the r_k largest columns (r_k = the slice's stage-1 rank), and the
// polar factor keeps those columns.
// Ranks without an instantiation run zero-padded (zero columns of T never
// rotate).
#include "common.cuh"
#include "internal.h"
#include "small_solve.cuh"

namespace dp2 {

constexpr int QW_SWEEPS = 30;

// pairs of warps per block: as many as fit about 220 KB of shared memory
template <int R>
constexpr int qw_ld() { return R + 1; }
template <int R>
constexpr size_t qw_pair_floats() { return (size_t)4 * R * qw_ld<R>() + R * R + R + 2; }
template <int R>
constexpr int qw_pairs() {
  const size_t shared = (size_t)2 * R * qw_ld<R>();
  const size_t avail = 220 * 1024 / 4 - shared;
  const size_t np = avail / qw_pair_floats<R>();
  return np > 6 ? 6 : (int)np;
}
template <int R>
constexpr size_t qw_smem() { return ((size_t)2 * R * qw_ld<R>() + qw_pairs<R>() * qw_pair_floats<R>()) * 4; }

__device__ __forceinline__ void pair_bar(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// One step along the ring (see k_eig_wide).
template <int H, typename V>
__device__ __forceinline__ void ring_step(V& top, V& bot, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  const V up = __shfl_up_sync(FULL, lane == 0 ? bot : top, 1);
  const V dn = __shfl_down_sync(FULL, bot, 1);
  const V ot = top;
  if (lane != 0) top = up;
  bot = (lane == H - 1) ? ot : dn;
}

template <int R>
__global__ void __launch_bounds__(64 * qw_pairs<R>()) k_qstep_wide(
    int K, int Ra, const float* __restrict__ Ft, const double* __restrict__ Psi, const float* __restrict__ W,
    const float* __restrict__ H, float* __restrict__ Upol, float* __restrict__ Pi, float* __restrict__ part,
    int pstride, int* __restrict__ status, int want_g1, float* __restrict__ Prot, const int* __restrict__ rank,
    PreSolve pre, int pre_on) {
  static_assert(R % 2 == 0 && R > 32 && R <= 64, "32 < R <= 64, even");
  constexpr int HP = R / 2;  // column pairs
  constexpr int LD = qw_ld<R>();
  constexpr int RR = R * R;
  constexpr int NP = qw_pairs<R>();
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) float sm[];
  if (pre_on && blockIdx.x == gridDim.x - 1) {  // the H update's factor (pre_solve)
    pre_solve(pre, reinterpret_cast<double*>(sm));
    return;
  }
  const int nb = gridDim.x - pre_on;
  float* ps = sm;            // Psi (R x LD)
  float* hs = ps + R * LD;   // H
  const int pair = threadIdx.x >> 6, pt = threadIdx.x & 63, lane = threadIdx.x & 31;
  const bool vwarp = pt >= 32;
  const int bar_id = 1 + pair;
  float* mine = sm + 2 * R * LD + (size_t)pair * qw_pair_floats<R>();
  float* Fs = mine;          // F~_k
  float* S1 = Fs + R * LD;   // scratch; S1 and S2 together hold the rotation buffers
  float* S2 = S1 + R * LD;
  float* S3 = S2 + R * LD;
  float* slot = S3 + R * LD; // Lemma 1 partial (R x R), entry e owned by thread e mod 64
  float* wks = slot + RR;    // W(k, :)
  int* ctrl = reinterpret_cast<int*>(wks + R);
  float2* rot = reinterpret_cast<float2*>(S1);  // [2][R - 1][HP]

  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e / R, b = e % R;
    const bool in = a < Ra && b < Ra;
    ps[a * LD + b] = in ? (float)Psi[a * Ra + b] : 0.f;
    hs[a * LD + b] = in ? H[a * Ra + b] : 0.f;
  }
  for (int e = pt; e < RR; e += 64) slot[e] = 0.f;
  __syncthreads();
  const float tol = fmaxf(1e-6f, (float)Ra * 1.2e-7f);
  const float rstop = sqrtf(tol * rsqrtf((float)Ra));  // as in k_qstep_reg
  const int RaRa = Ra * Ra;
  const bool act = lane < HP;
  const int j0 = lane, j1 = HP + lane;  // the columns this lane starts with

  for (int64_t k = (int64_t)blockIdx.x * NP + pair; k < K; k += (int64_t)nb * NP) {
    // ---- F~_k, V0, W(k, :)
    for (int e = pt; e < RR; e += 64) {
      const int i = e / R, c = e % R;
      const bool in = i < Ra && c < Ra;
      Fs[i * LD + c] = in ? Ft[k * RaRa + i * Ra + c] : 0.f;
      S2[i * LD + c] = (Prot && in) ? Prot[k * RaRa + i * Ra + c] : (i == c ? 1.f : 0.f);
    }
    for (int r = pt; r < R; r += 64) wks[r] = r < Ra ? W[k * Ra + r] : 0.f;
    pair_bar(bar_id);
    // ---- A1 = F~_k Psi (S1); Gv = V0^T V0 (S3)
    for (int e = pt; e < RR; e += 64) {
      const int i = e / R, c = e % R;
      float s = 0.f;
#pragma unroll 8
      for (int m = 0; m < R; ++m) s = fmaf(Fs[i * LD + m], ps[m * LD + c], s);
      S1[i * LD + c] = s;
      if (Prot) {
        float g = 0.f;
#pragma unroll 8
        for (int m = 0; m < R; ++m) g = fmaf(S2[m * LD + i], S2[m * LD + c], g);
        S3[i * LD + c] = g;
      }
    }
    pair_bar(bar_id);

    if (!vwarp) {
      // ================================ T warp ================================
      float top[R], bot[R];
      // T0 = A1 S_k H^T, columns j0 and j1:  T0(i, j) = sum_r A1(i, r) W(k, r) H(j, r)
#pragma unroll
      for (int i = 0; i < R; ++i) {
        float s0 = 0.f, s1 = 0.f;
        if (act) {
#pragma unroll 4
          for (int r = 0; r < R; ++r) {
            const float a = S1[i * LD + r] * wks[r];
            s0 = fmaf(a, hs[j0 * LD + r], s0);
            s1 = fmaf(a, hs[j1 * LD + r], s1);
          }
        }
        top[i] = s0;
        bot[i] = s1;
      }
      pair_bar(bar_id);
      if (act) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          S1[i * LD + j0] = top[i];
          S1[i * LD + j1] = bot[i];
        }
      }
      pair_bar(bar_id);  // the V warp has put V0 (after Newton-Schulz) in S3
      if (Prot && act) {
        // T0 V0, columns j0 and j1
#pragma unroll
        for (int i = 0; i < R; ++i) {
          float s0 = 0.f, s1 = 0.f;
#pragma unroll 4
          for (int m = 0; m < R; ++m) {
            const float a = S1[i * LD + m];
            s0 = fmaf(a, S3[m * LD + j0], s0);
            s1 = fmaf(a, S3[m * LD + j1], s1);
          }
          top[i] = s0;
          bot[i] = s1;
        }
      }
      __syncwarp();  // S1 is read by the whole warp before the rotation buffers overwrite it

      // ---- one-sided Jacobi sweeps
      const int rk = (rank ? min(rank[k], Ra) : Ra);
      for (int sweep = 0;; ++sweep) {
        float na = 0.f, nb = 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          na = fmaf(top[i], top[i], na);
          nb = fmaf(bot[i], bot[i], nb);
        }
        int at = 0, ab = 0;  // columns ahead of j0 / j1 in norm order (ties by index)
#pragma unroll 4
        for (int j = 0; j < HP; ++j) {
          const float xa = __shfl_sync(FULL, na, j), xb = __shfl_sync(FULL, nb, j);
          at += (xa > na || (xa == na && j < lane)) ? 1 : 0;
          at += (xb > na) ? 1 : 0;
          ab += (xa >= nb) ? 1 : 0;
          ab += (xb > nb || (xb == nb && j < lane)) ? 1 : 0;
        }
        int ft = (act && at < rk) ? 1 : 0, fb = (act && ab < rk) ? 1 : 0;
        float rmax = 0.f;  // largest ratio over pairs of kept columns
        float2* rb = rot + (size_t)(sweep & 1) * (R - 1) * HP;
        for (int rr = 0; rr < R - 1; ++rr) {
          float g0 = 0.f, g1 = 0.f;
#pragma unroll
          for (int i = 0; i < R; i += 2) {
            g0 = fmaf(top[i], bot[i], g0);
            g1 = fmaf(top[i + 1], bot[i + 1], g1);
          }
          const float gm = g0 + g1;
          float cs = 1.f, sn = 0.f;
          const float rel = (act && na > 0.f && nb > 0.f) ? fabsf(gm) * rsqrtf(na) * rsqrtf(nb) : 0.f;
          if (ft & fb) rmax = fmaxf(rmax, rel);
          if (rel > tol) {
            const float zeta = (nb - na) / (2.f * gm);
            const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            cs = rsqrtf(fmaf(tt, tt, 1.f));
            sn = cs * tt;
#pragma unroll
            for (int i = 0; i + 1 < R; i += 2) {
              const float2 x = make_float2(top[i], top[i + 1]), y = make_float2(bot[i], bot[i + 1]);
              const float2 nt = fmac2(cs, x, -sn, y), nbt = fmac2(sn, x, cs, y);
              top[i] = nt.x;
              top[i + 1] = nt.y;
              bot[i] = nbt.x;
              bot[i + 1] = nbt.y;
            }
            if (R & 1) {
              const float x = top[R - 1], y = bot[R - 1];
              top[R - 1] = fmaf(cs, x, -sn * y);
              bot[R - 1] = fmaf(sn, x, cs * y);
            }
            na = fmaf(-tt, gm, na);
            nb = fmaf(tt, gm, nb);
          }
          if (act) rb[rr * HP + lane] = make_float2(cs, sn);
#pragma unroll
          for (int i = 0; i < R; ++i) ring_step<HP>(top[i], bot[i], lane);
          ring_step<HP>(na, nb, lane);
          ring_step<HP>(ft, fb, lane);
        }
        const bool conv = warp_max(rmax) <= rstop;
        const bool stop = conv || sweep + 1 >= QW_SWEEPS;
        if (lane == 0) {
          ctrl[sweep & 1] = stop ? 1 : 0;
          if (!conv && stop) set_status(status, ST_SWEEP_CAP);
        }
        pair_bar(bar_id);
        if (stop) break;
      }
      pair_bar(bar_id);  // the V warp has applied the last sweep: S1 / S2 are free

      // ---- Z = the kept columns of T V normalised: the rk largest sigma > 0
      float st = 0.f, sb = 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        st = fmaf(top[i], top[i], st);
        sb = fmaf(bot[i], bot[i], sb);
      }
      st = sqrtf(st);
      sb = sqrtf(sb);
      int at = 0, ab = 0;
#pragma unroll 4
      for (int j = 0; j < HP; ++j) {
        const float xa = __shfl_sync(FULL, st, j), xb = __shfl_sync(FULL, sb, j);
        at += (xa > st || (xa == st && j < lane)) ? 1 : 0;
        at += (xb > st) ? 1 : 0;
        ab += (xa >= sb) ? 1 : 0;
        ab += (xb > sb || (xb == sb && j < lane)) ? 1 : 0;
      }
      const float it = (st > 0.f && at < rk) ? 1.f / st : 0.f;
      const float ib = (sb > 0.f && ab < rk) ? 1.f / sb : 0.f;
      if (act) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          S1[i * LD + j0] = top[i] * it;
          S1[i * LD + j1] = bot[i] * ib;
        }
      }
      pair_bar(bar_id);
    } else {
      // ================================ V warp ================================
      float vt[R], vb[R];
      // V0 after one Newton-Schulz step, columns j0 and j1
#pragma unroll
      for (int i = 0; i < R; ++i) {
        float s0 = 0.f, s1 = 0.f;
        if (act) {
          if (Prot) {
#pragma unroll 4
            for (int a = 0; a < R; ++a) {
              const float v = S2[i * LD + a];
              s0 = fmaf(v, S3[a * LD + j0], s0);
              s1 = fmaf(v, S3[a * LD + j1], s1);
            }
            s0 = fmaf(1.5f, S2[i * LD + j0], -0.5f * s0);
            s1 = fmaf(1.5f, S2[i * LD + j1], -0.5f * s1);
          } else {
            s0 = (i == j0) ? 1.f : 0.f;
            s1 = (i == j1) ? 1.f : 0.f;
          }
        }
        vt[i] = s0;
        vb[i] = s1;
      }
      pair_bar(bar_id);
      if (act) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          S3[i * LD + j0] = vt[i];
          S3[i * LD + j1] = vb[i];
        }
      }
      pair_bar(bar_id);
      // ---- apply each sweep's rotations as the T warp publishes them
      for (int sweep = 0;; ++sweep) {
        pair_bar(bar_id);
        const float2* rb = rot + (size_t)(sweep & 1) * (R - 1) * HP;
        const int stop = ctrl[sweep & 1];
        for (int rr = 0; rr < R - 1; ++rr) {
          const float2 p = act ? rb[rr * HP + lane] : make_float2(1.f, 0.f);
          if (p.y != 0.f) {
#pragma unroll
            for (int i = 0; i + 1 < R; i += 2) {
              const float2 x = make_float2(vt[i], vt[i + 1]), y = make_float2(vb[i], vb[i + 1]);
              const float2 nt = fmac2(p.x, x, -p.y, y), nbt = fmac2(p.y, x, p.x, y);
              vt[i] = nt.x;
              vt[i + 1] = nt.y;
              vb[i] = nbt.x;
              vb[i + 1] = nbt.y;
            }
            if (R & 1) {
              const float x = vt[R - 1], y = vb[R - 1];
              vt[R - 1] = fmaf(p.x, x, -p.y * y);
              vb[R - 1] = fmaf(p.y, x, p.x * y);
            }
          }
#pragma unroll
          for (int i = 0; i < R; ++i) ring_step<HP>(vt[i], vb[i], lane);
        }
        if (stop) break;
      }
      __syncwarp();
      pair_bar(bar_id);
      // ---- V into S2 (row-major); Prot_k = V
      if (act) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          S2[i * LD + j0] = vt[i];
          S2[i * LD + j1] = vb[i];
        }
        if (Prot) {
          float* pk = Prot + k * RaRa;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            if (i < Ra && j0 < Ra) pk[i * Ra + j0] = vt[i];
            if (i < Ra && j1 < Ra) pk[i * Ra + j1] = vb[i];
          }
        }
      }
      pair_bar(bar_id);
    }

    // ---- Upol = Z V^T (S3 and global):  Upol(a, c) = sum_i Z(a, i) V(c, i)
    for (int e = pt; e < RR; e += 64) {
      const int a = e / R, c = e % R;
      float s = 0.f;
#pragma unroll 8
      for (int i = 0; i < R; ++i) s = fmaf(S1[a * LD + i], S2[c * LD + i], s);
      S3[a * LD + c] = s;
      if (a < Ra && c < Ra) Upol[k * RaRa + a * Ra + c] = s;
    }
    pair_bar(bar_id);
    // ---- Pi = Upol^T F~_k (S1 and global)
    for (int e = pt; e < RR; e += 64) {
      const int a = e / R, c = e % R;
      float s = 0.f;
#pragma unroll 8
      for (int i = 0; i < R; ++i) s = fmaf(S3[i * LD + a], Fs[i * LD + c], s);
      S1[a * LD + c] = s;
      if (a < Ra && c < Ra) Pi[k * RaRa + a * Ra + c] = s;
    }
    if (want_g1) {
      pair_bar(bar_id);
      // Lemma 1: G1(i, c) += W(k, c) (Pi Psi)(i, c)
      for (int e = pt; e < RR; e += 64) {
        const int i = e / R, c = e % R;
        float s = 0.f;
#pragma unroll 8
        for (int m = 0; m < R; ++m) s = fmaf(S1[i * LD + m], ps[m * LD + c], s);
        slot[e] = fmaf(wks[c], s, slot[e]);
      }
    }
    pair_bar(bar_id);  // wks, Fs and S1 are rewritten by the next slice
  }
  if (!want_g1) return;
  __syncthreads();
  for (int e = threadIdx.x; e < RaRa; e += blockDim.x) {
    const int i = e / Ra, c = e % Ra;
    const float* s0 = sm + 2 * R * LD + 4 * R * LD + i * R + c;
    float s = 0.f;
    for (int q = 0; q < NP; ++q) s += s0[(size_t)q * qw_pair_floats<R>()];
    part[(int64_t)blockIdx.x * pstride + e] = s;
  }
}

template <int R>
static void qwide(const AlsBufs& b, float* part, int pstride, int want_g1, cudaStream_t s, const PreSolve* pre) {
  constexpr int NP = qw_pairs<R>();
  PreSolve p0;
  const int on = pre ? 1 : 0;
  if (pre) p0 = *pre;  // pre_solve_words(R, 64 NP) fits the Q-step's shared memory for R <= 64
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_qstep_wide<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qw_smem<R>());
    attr = true;
  }
  DP2_COUNTED(k_qstep_wide<R><<<b.nq + on, 64 * NP, qw_smem<R>(), s>>>(b.K, b.R, b.Ft, b.Psi, b.W, b.H, b.Upol, b.Pi, part,
                                                             pstride, b.status, want_g1, b.Prot, b.rank, p0, on));
}

// Blocks: one slice per pair of warps, at most `cap` blocks (the blocks loop
// over the slices), so that the Lemma 1 partials stay as many as the other
// partial sums of an iteration.
template <int R>
static int qwide_blocks(int K, int cap) {
  constexpr int NP = qw_pairs<R>();
  return std::max(1, std::min((K + NP - 1) / NP, cap));
}

// Instantiated ranks: 40, 50 exactly; 48, 56, 64 for the others (zero-padded).
int qstep_wide_blocks(int K, int R, int cap) {
  if (R == 40) return qwide_blocks<40>(K, cap);
  if (R == 50) return qwide_blocks<50>(K, cap);
  if (R <= 48) return qwide_blocks<48>(K, cap);
  if (R <= 56) return qwide_blocks<56>(K, cap);
  return qwide_blocks<64>(K, cap);
}

bool launch_qstep_wide(const AlsBufs& b, float* part, int pstride, int want_g1, cudaStream_t s, const PreSolve* pre) {
  if (b.R <= 32 || b.R > 64) return false;
  if (b.R == 40) qwide<40>(b, part, pstride, want_g1, s, pre);
  else if (b.R == 50) qwide<50>(b, part, pstride, want_g1, s, pre);
  else if (b.R <= 48) qwide<48>(b, part, pstride, want_g1, s, pre);
  else if (b.R <= 56) qwide<56>(b, part, pstride, want_g1, s, pre);
  else qwide<64>(b, part, pstride, want_g1, s, pre);
  return true;
}

}  // namespace dp2
