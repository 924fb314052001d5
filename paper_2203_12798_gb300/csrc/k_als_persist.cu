// All ALS iterations of a fit in one persistent launch (Alg. 3 repeat loop;
// Eq. q_k and Lemmas 1-3) for ranks R <= 20.
//
// One block per SM, launched cooperatively so that every block is resident.
// Block 0 is the solver block; blocks 1..nb-1 own fixed lists of slices (the
// register Q-step's groups of G = 32 / R consecutive slices, warp by warp) for
// the whole fit, so that the W_k a block computes at the end of an iteration
// is the one its Q-step reads at the start of the next.  An iteration is three
// phases separated by two grid barriers:
//   A  slice blocks: Q-step of their slices (qstep_warp) and their Lemma 1
//      partial; solver block, meanwhile: the previous iteration's W^T W and
//      e from the Lemma 3 partials (it waits only for those), and the FP64
//      factor (W^T W * V^T V)^-1 of the H update;
//   -- grid barrier --
//   B  every block: the H update (block_h_update; every block forms the same
//      H from the same partials in the same order); slice blocks: Lemma 2
//      partials; solver block, meanwhile: the FP64 factor (W^T W * H^T H)^-1
//      of the V update;
//   -- grid barrier --
//   C  every block: the V update and the W update's FP64 inverse
//      (V^T V * H^T H)^-1; slice blocks: Lemma 3, W_k, and the partials of
//      W^T W and e, then a count the solver block waits on.
// The arithmetic of every phase is that of the three-launch iteration
// (als_phases.cuh); only the slice-to-block assignment, and with it the
// order of the partial sums, differs.  The FP64 factorisations, whose
// instructions issue slowly on this part, overlap the FP32 slice work instead
// of following it, and no launch boundary separates the phases.
//
// Every wait is bounded (2 s of %globaltimer): a wait that runs out raises a
// flag in global memory that every other wait also watches, sets the timeout
// bit of the status word, and every block returns.
#include <algorithm>

#include "als_phases.cuh"
#include "common.cuh"
#include "internal.h"
#include "qstep_reg.cuh"
#include "small_solve.cuh"

namespace dp2 {

namespace {

constexpr unsigned long long kPersistWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long pt_time() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Thread 0: wait until *ctr >= target; false if the wait ran out (raising
// *abort) or another wait already raised it.
__device__ bool wait_count(const unsigned* ctr, unsigned target, int* abort) {
  const unsigned long long t0 = pt_time();
  for (;;) {
    if (ld_acquire_u32(ctr) >= target) return true;
    if (ld_volatile_i32(abort)) return false;
    if (pt_time() - t0 > kPersistWaitNs) {
      atomicExch(abort, 1);
      return false;
    }
    __nanosleep(32);
  }
}

// Whole block: grid barrier number `epoch` (0, 1, ...) on the arrival
// counter ctr (zero before the launch).  Returns false in every thread of
// the block when the barrier was abandoned.
__device__ bool grid_barrier(unsigned* ctr, unsigned epoch, int* abort, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const bool w = wait_count(ctr, (epoch + 1) * gridDim.x, abort);
    if (!w) set_status(status, ST_TIMEOUT);
    __threadfence();
    ok = w;
  }
  __syncthreads();
  return ok != 0;
}

template <int RP>
constexpr int persist_warps() { return RP <= 12 ? 18 : 8; }

}  // namespace

template <int RP>
__global__ void __launch_bounds__(32 * persist_warps<RP>(), 1) k_als_persist(PersistArgs a) {
  constexpr int G = 32 / RP;
  constexpr int PRR = RP * RP;
  extern __shared__ __align__(16) double sd[];
  __shared__ float ered[32][2];
  __shared__ int s_ok;
  const int K = a.K, R = a.R, RR = R * R, T = blockDim.x;
  const int nw = T >> 5, warp = threadIdx.x >> 5;
  const bool solver = blockIdx.x == 0;
  const int nsb = gridDim.x - 1, sb = blockIdx.x - 1;
  const int ps_ = a.pstride;
  // ---- shared memory (persist_smem below sizes this carve-up)
  double* red = sd;           // 4 T (quad reductions)
  double* G1 = red + 4 * T;   // RR
  double* Hn = G1 + RR;       // RR
  double* HtH = Hn + RR;      // RR
  double* Cb = HtH + RR;      // 2 RR
  double* C = Cb + 2 * RR;    // RR
  double* DC = C + RR;        // RR
  double* Gm = DC + RR;       // RR
  double* gi = Gm + RR;       // RR
  double* wtw = gi + RR;      // RR
  double* vtv = wtw + RR;     // RR
  double* W3 = vtv + RR;      // 2 RR + 2
  double* Lw = W3 + 2 * RR + 2;  // RR
  double* Vw = Lw + RR;          // RR
  double* fac = Vw + RR;         // spd_pinv_words(R)
  float* psc = reinterpret_cast<float*>(fac + spd_pinv_words(R));  // Psi, R x R
  float* hsc = psc + RR;      // H
  float* cvs = hsc + RR;      // CV
  float* psp = cvs + RR;      // Psi padded to RP x RP (Q-step)
  float* hsp = psp + PRR;     // H padded
  float* wreg = hsp + PRR;    // nw x a.wstride: per-warp scratch of the phases
  const int wstride = a.wstride;
  float* mine = wreg + (size_t)warp * wstride;
  // Lemma 2 / 3 layout inside `mine`: G x RP^2 group scratch, then G slots of
  // 2 R^2 floats (double-float entries (m, c) of lane c of group gq)
  const int gq = (threadIdx.x & 31) / RP, cq = (threadIdx.x & 31) - gq * RP;
  const bool lane_act = gq < G && cq < R;
  float* gslot2 = mine + G * PRR;

  for (int e = threadIdx.x; e < RR; e += T) {
    psc[e] = (float)a.Psi[e];
    hsc[e] = a.H[e];
    HtH[e] = a.HtH[e];
    wtw[e] = a.WtW[e];
    vtv[e] = a.VtV[e];
  }
  __syncthreads();
  unsigned epoch = 0;
  const int64_t first = (int64_t)sb * nw + warp, step = (int64_t)nsb * nw;
  for (int it = 0; it < a.max_iter; ++it) {
    // ================================================================ A
    if (!solver) {
      for (int e = threadIdx.x; e < PRR; e += T) {
        const int i = e / RP, j = e - i * RP;
        const bool in = i < R && j < R;
        psp[e] = in ? psc[i * R + j] : 0.f;
        hsp[e] = in ? hsc[i * R + j] : 0.f;
      }
      __syncthreads();
      qstep_warp<RP>(K, R, a.Ft, psp, hsp, a.W, a.Upol, a.Pi, a.status, 1, a.Prot, a.rank, mine,
                     mine + G * 3 * PRR, first, step);
      __syncthreads();
      for (int e = threadIdx.x; e < RR; e += T) {  // the block's Lemma 1 partial (warps, then groups)
        const int i = e / R, c = e - i * R;
        float s = 0.f;
        for (int w = 0; w < nw; ++w)
          for (int g = 0; g < G; ++g) s += wreg[(size_t)w * wstride + G * 3 * PRR + g * PRR + i * RP + c];
        a.part1[(int64_t)sb * ps_ + e] = s;
      }
    } else {
      if (it > 0) {
        // the previous iteration's W^T W and e, once every slice block has
        // written its Lemma 3 partial
        if (threadIdx.x == 0) {
          const bool w = wait_count(a.bar + 1, (unsigned)it * nsb, a.abort);
          if (!w) set_status(a.status, ST_TIMEOUT);
          __threadfence();
          s_ok = w;
        }
        __syncthreads();
        if (!s_ok) return;
        par_reduce4_load(a.part3, nsb, ps_, 2 * RR + 2, red);
        __syncthreads();
        par_reduce4_combine(2 * RR + 2, nsb, red, W3);
        __syncthreads();
        for (int e = threadIdx.x; e < RR + 1; e += T) {
          if (e < RR) {
            wtw[e] = W3[e] + W3[RR + e];
            a.WtW[e] = wtw[e];
          } else {
            const double v = W3[2 * RR] + W3[2 * RR + 1];
            a.loss[it - 1] = v;
            if (!isfinite(v)) set_status(a.status, ST_NONFINITE);
          }
        }
        __syncthreads();
      }
      // the H update's factor (W^T W * V^T V)^-1
      for (int e = threadIdx.x; e < RR; e += T) Gm[e] = wtw[e] * vtv[e];
      __syncthreads();
      block_spd_pinv<double, double>(Gm, a.InvH, Lw, Vw, R, fac, a.status);
    }
    if (!grid_barrier(a.bar, epoch++, a.abort, a.status)) return;
    // ================================================================ B
    block_h_update(a.part1, nsb, ps_, a.InvH, R, red, G1, Hn, hsc, HtH, a.status, 1);
    if (solver) {
      for (int e = threadIdx.x; e < RR; e += T) {
        a.H[e] = hsc[e];
        a.HtH[e] = HtH[e];
        Gm[e] = wtw[e] * HtH[e];
      }
      __syncthreads();
      block_spd_pinv<double, double>(Gm, a.InvV, Lw, Vw, R, fac, a.status);
    } else {
      DF acc[RP];
      lemma2_group<RP>(K, R, a.Pi, a.W, hsc, mine, acc, first, step);
      if (lane_act) {
        float* sl = gslot2 + (size_t)gq * 2 * RR;
#pragma unroll
        for (int m = 0; m < RP; ++m)
          if (m < R) {
            sl[m * R + cq] = acc[m].hi;
            sl[RR + m * R + cq] = acc[m].lo;
          }
      }
      __syncthreads();
      block_group_slots_df(wreg, nw, wstride, G * PRR, G, 2 * RR, RR, a.part2 + (int64_t)sb * ps_);
    }
    if (!grid_barrier(a.bar, epoch++, a.abort, a.status)) return;
    // ================================================================ C
    block_v_update(a.part2, nsb, ps_, a.InvV, a.DtD, HtH, R, red, Cb, C, DC, Gm, cvs, psc,
                   solver ? a.VtV : nullptr, a.CV, a.Psi, a.status, 1);
    block_spd_pinv<double, double>(Gm, gi, Lw, Vw, R, fac, a.status);
    if (solver) {
      for (int e = threadIdx.x; e < RR; e += T) {
        a.Ginv[e] = gi[e];
        vtv[e] = a.VtV[e];
      }
      __syncthreads();
    } else {
      DF wtw3[RP], ek;
      lemma3_group<RP>(K, R, a.Pi, psc, hsc, cvs, gi, a.W, mine, wtw3, ek, first, step);
      if (lane_act) {
        float* sl = gslot2 + (size_t)gq * 2 * RR;
#pragma unroll
        for (int m = 0; m < RP; ++m)
          if (m < R) {
            sl[m * R + cq] = wtw3[m].hi;
            sl[RR + m * R + cq] = wtw3[m].lo;
          }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        DF other;
        other.hi = __shfl_xor_sync(0xffffffffu, ek.hi, o);
        other.lo = __shfl_xor_sync(0xffffffffu, ek.lo, o);
        ek = df_add(ek, other);
      }
      if ((threadIdx.x & 31) == 0) {
        ered[warp][0] = ek.hi;
        ered[warp][1] = ek.lo;
      }
      __syncthreads();
      float* dst3 = a.part3 + (int64_t)sb * ps_;
      block_group_slots_df(wreg, nw, wstride, G * PRR, G, 2 * RR, RR, dst3);
      if (threadIdx.x == 0) {
        DF e3 = {0.f, 0.f};
        for (int w = 0; w < nw; ++w) e3 = df_add(e3, DF{ered[w][0], ered[w][1]});
        dst3[2 * RR] = e3.hi;
        dst3[2 * RR + 1] = e3.lo;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.bar + 1, 1u);
      }
    }
  }
}

// ---------------------------------------------------------------- launcher --
// Instantiated ranks: R <= 10 runs as RP = 10, 10 < R <= 20 as RP = 20 (zero
// padded, as the Q-step kernel pads).
static int persist_rp(int R) {
  if (R <= 10) return 10;
  if (R <= 20) return 20;
  return 0;
}

size_t persist_smem(int R, int RP, int nw, int* wstride) {
  const int RR = R * R, PRR = RP * RP, G = 32 / RP;
  const int per_q = G * 4 * PRR;            // Q-step scratch + Lemma 1 slots
  const int per_l = G * (PRR + 2 * RR);     // Lemma 2 / 3 group scratch and slots
  *wstride = round_up(std::max(per_q, per_l), 4);
  const size_t dbl = (size_t)128 * nw + 15 * (size_t)RR + 2 + spd_pinv_words(R);
  const size_t flt = (size_t)3 * RR + 2 * (size_t)PRR + (size_t)nw * *wstride;
  return dbl * sizeof(double) + flt * sizeof(float);
}

template <int RP>
static bool persist_launch(PersistArgs& a, int num_sms, cudaStream_t s) {
  constexpr int nw = persist_warps<RP>();
  const size_t smem = persist_smem(a.R, RP, nw, &a.wstride);
  if (smem > 220 * 1024) return false;
  if (cudaFuncSetAttribute(k_als_persist<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return false;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_als_persist<RP>, 32 * nw, smem) != cudaSuccess ||
      per_sm < 1)
    return false;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)k_als_persist<RP>, dim3((unsigned)num_sms), dim3(32 * nw), args, smem,
                                  s) != cudaSuccess) {
    (void)cudaGetLastError();  // a refused launch configuration: the caller falls back
    return false;
  }
  note_launch();
  return true;
}

bool persist_supported(int R) { return persist_rp(R) != 0; }

// Slices the slice blocks hold with one group of G = 32 / RP slices per warp.
// Past this count warps run several Q-step groups one after the other, and
// the per-iteration launches (whose grids cover any K in waves) are faster
// (measured at R = 10: K = 8154 persistent 3.37 ms, per-iteration 3.70 ms;
// K = 8455 4.90 against 4.10 ms; K = 12000 5.35 against 4.92 ms).
int64_t persist_capacity(int R, int num_sms) {
  const int RP = persist_rp(R);
  if (!RP || num_sms < 2) return 0;
  const int nw = RP <= 12 ? persist_warps<10>() : persist_warps<20>();
  return (int64_t)(num_sms - 1) * nw * (32 / RP);
}

// Launches the whole iteration loop; false when the rank has no
// instantiation or the cooperative launch is not possible (nothing launched
// then, except when the launch itself failed).  a.bar (3 words: barrier
// arrivals, Lemma 3 arrivals, abort flag) is zeroed here.
bool launch_als_persist(PersistArgs& a, int num_sms, cudaStream_t s) {
  const int RP = persist_rp(a.R);
  if (!RP || num_sms < 2) return false;
  if (cudaMemsetAsync(a.bar, 0, 3 * sizeof(unsigned), s) != cudaSuccess) return false;
  a.abort = reinterpret_cast<int*>(a.bar + 2);
  switch (RP) {
    case 10: return persist_launch<10>(a, num_sms, s);
    case 20: return persist_launch<20>(a, num_sms, s);
    default: return false;
  }
}

}  // namespace dp2
