// Stage-1 streaming passes on the 5th-generation tensor cores (sm_103a) for
// 16-bit X (BF16 / FP16 storage and multiplication, FP32 accumulation in TMEM).
//
//   sketch   Y = X Omega                (Alg. 1, "construct Y"; Eq. fstage_svd)
//   project  B1_k = Q1_k^T X_k          (Alg. 1, "construct B") + ||X_k||_F^2
//
// Both kernels are persistent (one CTA per SM) and warp-specialised:
//   warp 0      one thread issues TMA tile loads (cp.async.bulk.tensor) into a
//               ring of shared-memory stages, each guarded by mbarriers;
//   warp 1      allocates TMEM; one thread issues tcgen05.mma for every stage
//               and tcgen05.commit's the stage back to the producer;
//   warps 2-5   epilogue: tcgen05.ld the FP32 accumulator (one TMEM lane per
//               output row), write it out; the accumulator is double-buffered
//               in TMEM so the epilogue of one tile overlaps the next tile's MMAs;
//   warps 6-13  (project only) sum the squares of the staged X tiles, each
//               warp one eighth of every stage.
// Every mbarrier wait is bounded by %globaltimer (kWaitNs); a wait that runs out
// raises a CTA-wide abort flag, every role stops issuing work, waits (bounded)
// for its in-flight copies / MMAs, TMEM is released and the status word gets
// ST_TIMEOUT.
//
// Shared-memory operand layouts are the canonical 128-byte-swizzled ones that
// TMA SWIZZLE_128B produces (8-row atoms of 128-byte rows, 1024-byte aligned):
//   sketch   A = X tile, 128 rows x 64 columns, K-major (K = columns)
//            B = Omega^T chunk, LPN x 64, K-major
//   project  A = X tile seen as M = 128 columns x K = 64 rows: MN-major, two
//            64-column atoms 8 KB apart (leading-dimension offset), 8-row K
//            groups 1 KB apart (stride offset)
//            B = Q1 split into three 16-bit parts (Q1 = hi + mid + lo exactly
//            up to FP32 rounding), 3 LPN x 64 rows, K-major (K = rows), so
//            one MMA per K step yields hi/mid/lo partial products that the
//            epilogue adds: FP32 accuracy from 16-bit operands.
#include <cuda.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace dp2 {
namespace tc {

// --------------------------------------------------------------- sketch ----
constexpr int SK_BM = 128, SK_BK = 64, SK_STAGES = 6;

template <int LPN>
struct SketchSmem {
  static constexpr int A = SK_BM * SK_BK * 2;
  static constexpr int B = LPN * SK_BK * 2;
  static constexpr int BYTES = 1024 + SK_STAGES * (A + B) + 256;
};

template <int LPN>
__global__ void __launch_bounds__(192, 1) k_sketch_tc(const __grid_constant__ CUtensorMap tmX,
                                                      const __grid_constant__ CUtensorMap tmO, int64_t N, int J,
                                                      int LP, float* __restrict__ Y, int bf16, int* status) {
  using S = SketchSmem<LPN>;
  constexpr uint32_t NCOL = 2 * LPN < 32 ? 32 : 2 * LPN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint8_t* sA = base;
  uint8_t* sB = base + SK_STAGES * S::A;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + SK_STAGES * S::B);
  uint64_t* empty = full + SK_STAGES;
  uint64_t* accfull = empty + SK_STAGES;
  uint64_t* accempty = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (N + SK_BM - 1) / SK_BM;
  const int nk = (J + SK_BK - 1) / SK_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SK_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accfull[a], 1);
      mbar_init(&accempty[a], 128);
    }
    *abort_flag = 0;
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    tmem_alloc(tslot, NCOL);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    prefetch_tmap(&tmX);
    prefetch_tmap(&tmO);
    int s = 0;
    uint32_t ph = 0, inflight = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
      for (int kc = 0; kc < nk; ++kc) {
        if (!wait_bounded(&empty[s], ph ^ 1, abort_flag)) break;
        mbar_arrive_expect_tx(&full[s], S::A + S::B);
        tma_load_2d(sA + s * S::A, &tmX, &full[s], kc * SK_BK, (int)(tile * SK_BM));
        tma_load_2d(sB + s * S::B, &tmO, &full[s], kc * SK_BK, 0);
        inflight = 1;
        if (++s == SK_STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    // on abort: wait (bounded) until the last issued stage has landed
    if (*abort_flag && inflight) {
      int ls = (s + SK_STAGES - 1) % SK_STAGES;
      uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&full[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idesc = idesc_f16(SK_BM, LPN, bf16 != 0, false, false);
    int s = 0;
    uint32_t ph = 0;
    int t = 0;
    bool issued = false;
    for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++t) {
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accempty[acc], aph ^ 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * LPN;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc) {
        if (!wait_bounded(&full[s], ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sdesc_sw128(smem_u32(sA + s * S::A), 16, 1024);
        const uint64_t bd = sdesc_sw128(smem_u32(sB + s * S::B), 16, 1024);
#pragma unroll
        for (int kk = 0; kk < SK_BK / 16; ++kk)
          tc_mma(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc | kk) != 0 ? 1u : 0u);
        tc_commit(&empty[s]);
        issued = true;
        if (++s == SK_STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      tc_commit(&accfull[acc]);
    }
    if (*abort_flag && issued) {
      // drain: wait (bounded) for the MMAs behind the last commit
      const int ls = (s + SK_STAGES - 1) % SK_STAGES;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&empty[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    int t = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accfull[acc], aph, abort_flag)) break;
      tc_fence_after();
      float v[LPN];
#pragma unroll
      for (int g = 0; g < LPN / 32; ++g) tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * LPN + g * 32, v + 32 * g);
      tc_fence_before();
      mbar_arrive(&accempty[acc]);
      const int64_t row = tile * SK_BM + q * 32 + lane;
      if (row < N) {
        float4* dst = reinterpret_cast<float4*>(Y + row * LP);
#pragma unroll
        for (int c4 = 0; c4 < LPN / 4; ++c4)
          if (4 * c4 < LP) dst[c4] = make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOL);
  }
  if (threadIdx.x == 0 && *abort_flag) set_status(status, ST_TIMEOUT);
}

// ------------------------------------------------- per-slice sketch ----
// U_k = X_k M_k with a different J x LP right operand per slice (the
// learned-sketch gradient's X_k (X_k^T Y_k G_k^-1) pass).  M_k is given as three
// exact-sum 16-bit parts, stored [k][3 LPN][Jpad] (K-major rows), so one MMA
// per K step yields hi / mid / lo products that the epilogue adds.  Work
// items are (slice, 128-row tile of the slice); rows of a tile past the end of
// its slice are computed against the wrong operand and not written.
template <int LPN>
struct SegSmem {
  static constexpr int NS = 3 * LPN;
  static constexpr int A = SK_BM * SK_BK * 2;
  static constexpr int B = NS * SK_BK * 2;
  static constexpr int STAGES = LPN == 32 ? 6 : 4;
  static constexpr int BYTES = 1024 + STAGES * (A + B) + 256;
};

// slice of work item `item` (toff: K + 1 prefix sums of tiles per slice)
__device__ __forceinline__ int seg_slice(const int64_t* __restrict__ toff, int K, int64_t item) {
  int lo = 0, hi = K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int LPN>
__global__ void __launch_bounds__(192, 1) k_sketch_seg_tc(const __grid_constant__ CUtensorMap tmX,
                                                          const __grid_constant__ CUtensorMap tmM,
                                                          const int64_t* __restrict__ off,
                                                          const int64_t* __restrict__ toff, int K, int J, int LP,
                                                          float* __restrict__ U, int bf16, int* status) {
  using S = SegSmem<LPN>;
  constexpr int ST = S::STAGES;
  constexpr uint32_t NCOL = 2 * S::NS <= 256 ? 256 : 512;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint8_t* sA = base;
  uint8_t* sB = base + ST * S::A;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + ST * S::B);
  uint64_t* empty = full + ST;
  uint64_t* accfull = empty + ST;
  uint64_t* accempty = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nitems = toff[K];
  const int nk = (J + SK_BK - 1) / SK_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accfull[a], 1);
      mbar_init(&accempty[a], 128);
    }
    *abort_flag = 0;
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    tmem_alloc(tslot, NCOL);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    prefetch_tmap(&tmX);
    prefetch_tmap(&tmM);
    int s = 0;
    uint32_t ph = 0, inflight = 0;
    for (int64_t item = blockIdx.x; item < nitems && !*abort_flag; item += gridDim.x) {
      const int k = seg_slice(toff, K, item);
      // the last tile of a slice ends at its last row (overlapping the tile
      // before it) instead of reading rows of the next slice
      const int row0 = (int)min64(off[k] + (item - toff[k]) * SK_BM, off[k + 1] - SK_BM);
      for (int kc = 0; kc < nk; ++kc) {
        if (!wait_bounded(&empty[s], ph ^ 1, abort_flag)) break;
        mbar_arrive_expect_tx(&full[s], S::A + S::B);
        tma_load_2d(sA + s * S::A, &tmX, &full[s], kc * SK_BK, row0);
        tma_load_3d(sB + s * S::B, &tmM, &full[s], kc * SK_BK, 0, k);
        inflight = 1;
        if (++s == ST) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    if (*abort_flag && inflight) {
      const int ls = (s + ST - 1) % ST;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&full[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idesc = idesc_f16(SK_BM, S::NS, bf16 != 0, false, false);
    int s = 0;
    uint32_t ph = 0;
    int t = 0;
    bool issued = false;
    for (int64_t item = blockIdx.x; item < nitems && !*abort_flag; item += gridDim.x, ++t) {
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accempty[acc], aph ^ 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * S::NS;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc) {
        if (!wait_bounded(&full[s], ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sdesc_sw128(smem_u32(sA + s * S::A), 16, 1024);
        const uint64_t bd = sdesc_sw128(smem_u32(sB + s * S::B), 16, 1024);
#pragma unroll
        for (int kk = 0; kk < SK_BK / 16; ++kk)
          tc_mma(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc | kk) != 0 ? 1u : 0u);
        tc_commit(&empty[s]);
        issued = true;
        if (++s == ST) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      tc_commit(&accfull[acc]);
    }
    if (*abort_flag && issued) {
      const int ls = (s + ST - 1) % ST;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&empty[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    int t = 0;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++t) {
      const int k = seg_slice(toff, K, item);
      const int64_t first = off[k] + (item - toff[k]) * SK_BM;  // first row this tile owns
      const int64_t row = min64(first, off[k + 1] - SK_BM) + q * 32 + lane;
      const bool valid = row >= first && row < off[k + 1];
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accfull[acc], aph, abort_flag)) break;
      tc_fence_after();
      const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + acc * S::NS;
#pragma unroll
      for (int g = 0; g < LPN / 32; ++g) {
        float v[32], w[32];
        tmem_ld32(tl + g * 32, v);
        tmem_ld32(tl + LPN + g * 32, w);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += w[i];
        tmem_ld32(tl + 2 * LPN + g * 32, w);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += w[i];
        if (valid) {
          float4* dst = reinterpret_cast<float4*>(U + row * LP + g * 32);
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4)
            if (g * 32 + 4 * c4 < LP) dst[c4] = make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
        }
      }
      tc_fence_before();
      mbar_arrive(&accempty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOL);
  }
  if (threadIdx.x == 0 && *abort_flag) set_status(status, ST_TIMEOUT);
}

// Power of two applied to a slice's Q rows before the 16-bit split: Q has
// orthonormal columns, so its entries are about I_k^-1/2 and at most 1; the
// scale 2^floor(log2 sqrt(I_k)) lifts them towards 1, which keeps the FP16
// middle and low parts out of the subnormal range (exact for both types).
__device__ __forceinline__ float qsplit_scale(int64_t nrows) {
  return ldexpf(1.f, ilogbf(sqrtf((float)(nrows > 0 ? nrows : 1))));
}

// -------------------------------------------------------------- project ----
constexpr int PJ_BM = 128, PJ_BK = 64, PJ_STAGES = 5;
constexpr int PJ_NORM_WARPS = kProjNormWarps;          // warps 6 .. 6 + PJ_NORM_WARPS - 1
constexpr int PJ_THREADS = 32 * (6 + PJ_NORM_WARPS);
constexpr int PJ_NORM_GROUP = 4096;  // bytes of X per FP32 partial sum of squares

template <int NS_, int HV_ = (NS_ <= 64 ? 4 : (NS_ <= 128 ? 2 : 1))>
struct ProjSmem {
  // NS = MMA N: the three 16-bit parts of the Q rows, part t of column c in
  // row t OFF + c (OFF = l rounded up to 4, or 32 / 64), padded to 48, 64, 96
  // or 192.  HV column halves of PJ_BM columns per work item: by default as
  // many as let the double-buffered accumulators (2 HV NS columns) fit TMEM's
  // 512 (wider rows per TMA load, one Q tile per stage for all halves); half
  // as many is the narrower candidate the autotuner also times.
  static constexpr int NS = NS_;
  static constexpr int HV = HV_;
  static_assert(2 * HV * NS <= 512, "double-buffered accumulators within TMEM");
  static constexpr int A = HV * PJ_BM * PJ_BK * 2;  // 2 HV 64-column boxes of 64 rows, 8 KB each
  static constexpr int B = NS * PJ_BK * 2;
  static constexpr int FIT = (227 * 1024 - 1024 - 256) / (A + B);
  static constexpr int STAGES = FIT > PJ_STAGES ? PJ_STAGES : FIT;
  static constexpr int BYTES = 1024 + STAGES * (A + B) + 256;
  static constexpr int COLS = HV * PJ_BM;          // columns of X per work item
};

// 4 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes (no wait)
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int NS, int HV>
__global__ void __launch_bounds__(PJ_THREADS, 1) k_project_tc(const __grid_constant__ CUtensorMap tmX,
                                                       const __grid_constant__ CUtensorMap tmQ,
                                                       const int64_t* __restrict__ off,
                                                       const int64_t* __restrict__ poff, int K, int J, int Jp,
                                                       int LP, int OFF, float* __restrict__ B1,
                                                       double* __restrict__ xpart, int nJb, int bf16, int qscale,
                                                       const int* __restrict__ lptr, const int* __restrict__ items,
                                                       int* status) {
  using S = ProjSmem<NS, HV>;
  constexpr int ST = S::STAGES;
  constexpr uint32_t NCOL = 2 * S::HV * S::NS <= 256 ? 256 : 512;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint8_t* sA = base;
  uint8_t* sB = base + ST * S::A;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + ST * S::B);
  uint64_t* empty = full + ST;
  uint64_t* accfull = empty + ST;
  uint64_t* accempty = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Work items (slice k, column block jb) numbered k nJb + jb, two schedules:
  //   lptr == null  dealt round-robin over the CTAs;
  //   otherwise     CTA b takes items[lptr[b] .. lptr[b + 1]) in order (a
  //                 schedule the host builds, e.g. longest slices first onto
  //                 the least-loaded CTA).
  const int64_t it0 = lptr ? (int64_t)lptr[blockIdx.x] : (int64_t)blockIdx.x;
  const int64_t its = lptr ? 1 : (int64_t)gridDim.x;
  const int64_t itn = lptr ? (int64_t)lptr[blockIdx.x + 1] : (int64_t)K * nJb;
#define PJ_ITEM(it) const int64_t item_ = lptr ? (int64_t)items[it] : (it); \
  const int k = (int)(item_ / nJb); const int jb = (int)(item_ % nJb); (void)jb

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + PJ_NORM_WARPS);  // MMA commit + one arrival per norm warp
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accfull[a], 1);
      mbar_init(&accempty[a], 128);
    }
    *abort_flag = 0;
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    tmem_alloc(tslot, NCOL);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    prefetch_tmap(&tmX);
    prefetch_tmap(&tmQ);
    const uint64_t pol_x = policy_evict_first(), pol_q = policy_evict_last();
    int s = 0;
    uint32_t ph = 0;
    bool inflight = false;
    for (int64_t it = it0; it < itn && !*abort_flag; it += its) {
      PJ_ITEM(it);
      const int64_t r0 = off[k], r1 = off[k + 1], p0 = poff[k];
      const int nch = (int)((r1 - r0 + PJ_BK - 1) / PJ_BK);
      bool ok = true;
      for (int c = 0; c < nch; ++c) {
        if (!wait_bounded(&empty[s], ph ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[s], S::A + S::B);
        uint8_t* a = sA + s * S::A;
        // the last chunk ends at the slice's last row (it overlaps the chunk
        // before it, whose rows its Q rows zero) instead of reading past it;
        // the chunk before it is kept in L2 for that second read
        const int row = (int)(c + 1 < nch ? r0 + (int64_t)c * PJ_BK : r1 - PJ_BK);
        const uint64_t pol = (c + 2 == nch && (r1 - r0) % PJ_BK != 0) ? pol_q : pol_x;
#pragma unroll
        for (int bx = 0; bx < 2 * S::HV; ++bx)
          tma_load_2d_hint(a + bx * 8192, &tmX, &full[s], jb * S::COLS + 64 * bx, row, pol);
        tma_load_3d_hint(sB + s * S::B, &tmQ, &full[s], 0, 0, (int)(p0 / PJ_BK + c), pol_q);
        inflight = true;
        if (++s == ST) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
    }
    if (*abort_flag && inflight) {
      const int ls = (s + ST - 1) % ST;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&full[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idesc = idesc_f16(PJ_BM, S::NS, bf16 != 0, true, false);
    int s = 0;
    uint32_t ph = 0;
    int t = 0;
    bool issued = false;
    for (int64_t it = it0; it < itn && !*abort_flag; it += its, ++t) {
      PJ_ITEM(it);
      const int64_t nrows = off[k + 1] - off[k];
      const int nch = (int)((nrows + PJ_BK - 1) / PJ_BK);
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accempty[acc], aph ^ 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * S::HV * S::NS;
      bool ok = true;
      for (int c = 0; c < nch; ++c) {
        if (!wait_bounded(&full[s], ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // B: K-major, 8-row groups 1 KB apart
        const uint64_t bd = sdesc_sw128(smem_u32(sB + s * S::B), 16, 1024);
#pragma unroll
        for (int h = 0; h < S::HV; ++h) {
          // A (half h): MN-major, 64-column atoms 8 KB apart, 8-row K groups 1 KB apart
          const uint64_t ad = sdesc_sw128(smem_u32(sA + s * S::A + h * 16384), 8192, 1024);
#pragma unroll
          for (int kk = 0; kk < PJ_BK / 16; ++kk)
            tc_mma(d + h * S::NS, ad + (uint64_t)(kk * 128), bd + (uint64_t)(kk * 2), idesc,
                   (c | kk) != 0 ? 1u : 0u);
        }
        tc_commit(&empty[s]);
        issued = true;
        if (++s == ST) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      tc_commit(&accfull[acc]);
    }
    if (*abort_flag && issued) {
      const int ls = (s + ST - 1) % ST;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&empty[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= 2 && warp <= 5) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    int t = 0;
    for (int64_t it = it0; it < itn; it += its, ++t) {
      PJ_ITEM(it);
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      // the split Q rows of this slice were scaled by qsplit_scale(I_k)
      const float inv = qscale ? 1.f / qsplit_scale(off[k + 1] - off[k]) : 1.f;
      if (!wait_bounded(&accfull[acc], aph, abort_flag)) break;
      tc_fence_after();
      for (int h = 0; h < S::HV; ++h) {
        const int j = jb * S::COLS + h * PJ_BM + q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + acc * S::HV * S::NS + h * S::NS;
        if constexpr (NS >= 96) {
          // parts 32 or 64 columns apart (OFF = NS / 3): whole 32-column loads
          for (int g = 0; g < OFF / 32; ++g) {
            float v[32], w[32];
            tmem_ld32(tl + g * 32, v);
            tmem_ld32(tl + OFF + g * 32, w);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += w[i];
            tmem_ld32(tl + 2 * OFF + g * 32, w);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += w[i];
            if (j < Jp) {
              float* dst = B1 + ((int64_t)k * LP + g * 32) * Jp + j;
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (g * 32 + i < LP) dst[(int64_t)i * Jp] = v[i] * inv;
            }
          }
        } else {
          // compact parts (OFF <= 21, a multiple of 4): the three parts of
          // column c sit at c, OFF + c and 2 OFF + c, inside this half's NS columns
#pragma unroll
          for (int g = 0; g < 2; ++g) {  // 16 output rows at a time
            float a[16], b[16];
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              if (16 * g + 4 * q4 < OFF) {
                tmem_ld4(tl + 16 * g + 4 * q4, a + 4 * q4);
                tmem_ld4(tl + OFF + 16 * g + 4 * q4, b + 4 * q4);
              }
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] += b[i];
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              if (16 * g + 4 * q4 < OFF) tmem_ld4(tl + 2 * OFF + 16 * g + 4 * q4, b + 4 * q4);
            tmem_wait_ld();
            if (j < Jp) {
              float* dst = B1 + ((int64_t)k * LP + 16 * g) * Jp + j;
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (16 * g + i < LP) dst[(int64_t)i * Jp] = 16 * g + i < OFF ? (a[i] + b[i]) * inv : 0.f;
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&accempty[acc]);
    }
  } else if (warp >= 6) {
    // ------------------------------------------------------------ ||X_k||^2
    // Norm warp nw scans bytes [nw * BYTES_PER, (nw + 1) * BYTES_PER) of every
    // staged X tile (2 HV 8 KB boxes of 64 rows x 128 bytes), rows of the
    // current slice only, and writes its own partial sum per work item
    // (xpart is K x nJb x PJ_NORM_WARPS; a later kernel adds them in order).
    constexpr int BYTES_PER = S::A / PJ_NORM_WARPS;
    constexpr int GROUP = BYTES_PER < PJ_NORM_GROUP ? BYTES_PER : PJ_NORM_GROUP;
    static_assert(BYTES_PER % GROUP == 0, "norm groups");
    const int nw = warp - 6;
    int s = 0;
    uint32_t ph = 0;
    for (int64_t it = it0; it < itn; it += its) {
      PJ_ITEM(it);
      const int64_t nrows = off[k + 1] - off[k];
      const int nch = (int)((nrows + PJ_BK - 1) / PJ_BK);
      // per lane: eight independent FP32 accumulators (one per element of a
      // 16-byte load, 64 squares each per staged chunk, so no accumulator grows
      // far beyond its terms), combined pairwise and added in FP64 per chunk
      double acc = 0.0;
      bool ok = true;
      for (int c = 0; c < nch; ++c) {
        if (!wait_bounded(&full[s], ph, abort_flag)) {
          ok = false;
          break;
        }
        // rows of this slice in the staged box: the last `valid` ones (the
        // last chunk is aligned to the slice's end)
        const int valid = (int)min64(PJ_BK, nrows - (int64_t)c * PJ_BK);
        const uint8_t* a = sA + s * S::A + nw * BYTES_PER;
        // FP32 sums over fixed 4 KB groups (32 rows of a 64-column box), so
        // that both work-item widths form the same group sums
#pragma unroll
        for (int g0 = 0; g0 < BYTES_PER; g0 += GROUP) {
          float a8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) a8[e] = 0.f;
#pragma unroll
          for (int it = g0 / 512; it < (g0 + GROUP) / 512; ++it) {
            const int byte = nw * BYTES_PER + it * 512 + lane * 16;
            const int row = (byte % 8192) / 128;
            if (row >= PJ_BK - valid) {
              const uint4 u = *reinterpret_cast<const uint4*>(a + it * 512 + lane * 16);
              float f[8];
              if (bf16) Vec16<__nv_bfloat16>::unpack(u, f);
              else Vec16<__half>::unpack(u, f);
#pragma unroll
              for (int e = 0; e < 8; ++e) a8[e] = fmaf(f[e], f[e], a8[e]);
            }
          }
          acc += (double)(((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7])));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == ST) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      acc = warp_sum(acc);
      if (lane == 0) xpart[((int64_t)k * nJb + jb) * PJ_NORM_WARPS + nw] = acc;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOL);
  }
  if (threadIdx.x == 0 && *abort_flag) set_status(status, ST_TIMEOUT);
}

#undef PJ_ITEM

// ------------------------------------------------------------- operands ----
// Omega^T in 16-bit (LPN x Jpad) from the padded FP32 Omega (Jpad x LP).
__global__ void k_omega_t16(const float* __restrict__ om, int Jpad, int LP, int LPN, int bf16, void* out) {
  const int64_t n = (int64_t)LPN * Jpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / Jpad), j = (int)(i % Jpad);
    const float v = c < LP ? om[(int64_t)j * LP + c] : 0.f;
    if (bf16) reinterpret_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16_rn(v);
    else reinterpret_cast<__half*>(out)[i] = __float2half_rn(v);
  }
}

// Q1 rows (N x LP FP32) -> three exact-sum 16-bit parts, transposed to
// NSQ x Npad with every slice padded to a multiple of 64 rows; part t of
// column c is row t OFF + c (rows from 3 OFF on are zero).
// Layout of the split: 64-row chunks of all NSQ rows stored contiguously,
// element (p, r) at ((p / 64) NSQ + r) 64 + p % 64, so that one chunk (the B
// operand of one projection stage) is a single contiguous NSQ x 128-byte block.
// The last chunk of a slice holds the slice's last 64 rows (the projection
// reads X there from the slice's end backwards), zeros where they repeat
// rows of the chunk before it.
__global__ void k_qsplit(const float* __restrict__ Q, int LP, int NSQ, int OFF, const int64_t* __restrict__ off,
                         const int64_t* __restrict__ poff, int K, int64_t Npad, int bf16, void* out) {
  const int k = blockIdx.y;
  const int64_t p0 = poff[k], p1 = poff[k + 1], r0 = off[k], nr = off[k + 1] - r0;
  const int64_t last0 = p1 - p0 - PJ_BK;  // first padded row of the last chunk
  const float sc = qsplit_scale(nr);
  for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = p - p0;
    bool in = i < nr;
    if (i >= last0) {  // last chunk: box row b holds slice row nr - 64 + b
      const int64_t b = i - last0;
      i = nr - PJ_BK + b;
      in = i >= last0;
    }
    const int64_t cb = (p / PJ_BK) * NSQ * PJ_BK + (p % PJ_BK);  // element (p, 0)
    for (int c = 0; c < OFF; ++c) {
      const float qv = (in && c < LP) ? Q[(r0 + i) * LP + c] * sc : 0.f;
      if (bf16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(qv);
        const float r1 = qv - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
        __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + cb;
        o[(int64_t)c * PJ_BK] = h;
        o[(int64_t)(OFF + c) * PJ_BK] = m;
        o[(int64_t)(2 * OFF + c) * PJ_BK] = l;
      } else {
        const __half h = __float2half_rn(qv);
        const float r1 = qv - __half2float(h);
        const __half m = __float2half_rn(r1);
        const __half l = __float2half_rn(r1 - __half2float(m));
        __half* o = reinterpret_cast<__half*>(out) + cb;
        o[(int64_t)c * PJ_BK] = h;
        o[(int64_t)(OFF + c) * PJ_BK] = m;
        o[(int64_t)(2 * OFF + c) * PJ_BK] = l;
      }
    }
    for (int r = 3 * OFF; r < NSQ; ++r) {  // padding rows of the chunk
      if (bf16) reinterpret_cast<__nv_bfloat16*>(out)[cb + (int64_t)r * PJ_BK] = __float2bfloat16_rn(0.f);
      else reinterpret_cast<__half*>(out)[cb + (int64_t)r * PJ_BK] = __float2half_rn(0.f);
    }
  }
}

}  // namespace tc

// ---------------------------------------------------------------- host side --
bool tc_available() { return encode_fn() != nullptr; }

int tc_lpn(int ell) { return ell <= 32 ? 32 : 64; }

bool launch_sketch_tc(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const void* omT16, int Jpad,
                      int LPN, int LP, float* Y, int num_sms, int* status, cudaStream_t s) {
  const bool bf = dt == DPAR2_BF16;
  CUtensorMap mx, mo;
  if (!make_map(&mx, X, bf, (uint64_t)J, (uint64_t)N, (uint64_t)ldx, tc::SK_BK, tc::SK_BM)) return false;
  if (!make_map(&mo, omT16, bf, (uint64_t)Jpad, (uint64_t)LPN, (uint64_t)Jpad, tc::SK_BK, (uint32_t)LPN)) return false;
  const int64_t ntiles = (N + tc::SK_BM - 1) / tc::SK_BM;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  if (LPN == 32) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tc::k_sketch_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SketchSmem<32>::BYTES);
      attr = true;
    }
    DP2_COUNTED(tc::k_sketch_tc<32><<<grid, 192, tc::SketchSmem<32>::BYTES, s>>>(mx, mo, N, J, LP, Y, bf ? 1 : 0, status));
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tc::k_sketch_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SketchSmem<64>::BYTES);
      attr = true;
    }
    DP2_COUNTED(tc::k_sketch_tc<64><<<grid, 192, tc::SketchSmem<64>::BYTES, s>>>(mx, mo, N, J, LP, Y, bf ? 1 : 0, status));
  }
  return true;
}

bool launch_sketch_seg_tc(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const int64_t* d_off,
                          const int64_t* d_toff, int64_t ntiles, int K, const void* Ms, int Jpad, int LPN, int LP,
                          float* U, int num_sms, int* status, cudaStream_t s) {
  const bool bf = dt == DPAR2_BF16;
  CUtensorMap mx, mm;
  if (!make_map(&mx, X, bf, (uint64_t)J, (uint64_t)N, (uint64_t)ldx, tc::SK_BK, tc::SK_BM)) return false;
  if (!make_map3_box(&mm, Ms, bf, (uint64_t)Jpad, (uint64_t)(3 * LPN), (uint64_t)K, tc::SK_BK)) return false;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  if (grid <= 0) return true;
  if (LPN == 32) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tc::k_sketch_seg_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::SegSmem<32>::BYTES);
      attr = true;
    }
    DP2_COUNTED(tc::k_sketch_seg_tc<32><<<grid, 192, tc::SegSmem<32>::BYTES, s>>>(mx, mm, d_off, d_toff, K, J, LP, U,
                                                                      bf ? 1 : 0, status));
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tc::k_sketch_seg_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::SegSmem<64>::BYTES);
      attr = true;
    }
    DP2_COUNTED(tc::k_sketch_seg_tc<64><<<grid, 192, tc::SegSmem<64>::BYTES, s>>>(mx, mm, d_off, d_toff, K, J, LP, U,
                                                                      bf ? 1 : 0, status));
  }
  return true;
}

void project_lpt_lists(const int64_t* off, int K, int nJb, int nlists, std::vector<int>& lptr,
                       std::vector<int>& items) {
  std::vector<int> order(K);
  for (int k = 0; k < K; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
  // an item costs its slice's rows plus one 64-row chunk of fixed overhead
  using Load = std::pair<int64_t, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int c = 0; c < nlists; ++c) heap.push({0, c});
  std::vector<std::vector<int>> lists(nlists);
  for (int k : order) {
    const int64_t cost = off[k + 1] - off[k] + 64;
    for (int jb = 0; jb < nJb; ++jb) {
      Load l = heap.top();
      heap.pop();
      lists[l.second].push_back(k * nJb + jb);
      heap.push({l.first + cost, l.second});
    }
  }
  lptr.assign(nlists + 1, 0);
  items.clear();
  items.reserve((size_t)K * nJb);
  for (int c = 0; c < nlists; ++c) {
    items.insert(items.end(), lists[c].begin(), lists[c].end());
    lptr[c + 1] = (int)items.size();
  }
}

void proj_layout(int ell, int* NS, int* OFF) {
  if (ell > 32) {
    *NS = 192;
    *OFF = 64;
    return;
  }
  // compact (parts OFF = l rounded up to 4 apart) where that saves MMA width,
  // else parts 32 rows apart
  const int o = (ell + 3) / 4 * 4;
  *OFF = 3 * o <= 64 ? o : 32;
  *NS = 3 * o <= 48 ? 48 : (3 * o <= 64 ? 64 : 96);
}

int project_hv_default(int NS) { return NS <= 64 ? 4 : (NS <= 128 ? 2 : 1); }
// the narrower width only where a norm warp's share of a stage stays a whole
// number of 4 KB groups (so that ||X_k||^2 does not depend on the width)
int project_hv_alt(int NS) { return NS <= 64 ? project_hv_default(NS) / 2 : 0; }

int project_tc_cols(int NS, int hv) { return (hv > 0 ? hv : project_hv_default(NS)) * tc::PJ_BM; }

template <int NS, int HV>
static void project_launch(const CUtensorMap& mx, const CUtensorMap& mq, int grid, const int64_t* d_off,
                           const int64_t* d_poff, int K, int J, int Jp, int LP, int OFF, float* B1, double* xpart,
                           int nJb, int bf, int qs, const int* lptr, const int* items, int* status, cudaStream_t s) {
  using S = tc::ProjSmem<NS, HV>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_project_tc<NS, HV>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    attr = true;
  }
  DP2_COUNTED(tc::k_project_tc<NS, HV><<<grid, tc::PJ_THREADS, S::BYTES, s>>>(mx, mq, d_off, d_poff, K, J, Jp, LP, OFF,
                                                                             B1, xpart, nJb, bf, qs, lptr, items,
                                                                             status));
}

bool launch_project_tc(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, const int64_t* d_off,
                       const int64_t* d_poff, int K, int J, int Jp, const void* Qs, int64_t Npad, int NS, int OFF,
                       int LP, float* B1, double* xpart, int nJb, bool qscale, int num_sms, int* status,
                       cudaStream_t s, const int* lptr, const int* items, int nlists, int hv) {
  const bool bf = dt == DPAR2_BF16;
  if (hv <= 0) hv = project_hv_default(NS);
  if (hv != project_hv_default(NS) && hv != project_hv_alt(NS)) return false;
  CUtensorMap mx, mq;
  // no L2 promotion: a box row (128 bytes) of X starts anywhere on a 16-byte
  // boundary, so 256-byte promotion fetches neighbouring columns that belong to
  // another work item (measured: 5% more DRAM reads, same time)
  if (!make_map(&mx, X, bf, (uint64_t)J, (uint64_t)N, (uint64_t)ldx, 64, tc::PJ_BK,
                (int)CU_TENSOR_MAP_L2_PROMOTION_NONE))
    return false;
  if (!make_map3(&mq, Qs, bf, (uint64_t)tc::PJ_BK, (uint64_t)NS, (uint64_t)(Npad / tc::PJ_BK))) return false;
  const int grid = lptr ? nlists : (int)std::min<int64_t>((int64_t)K * nJb, num_sms);
  const int bfi = bf ? 1 : 0, qs = qscale ? 1 : 0;
#define DP2_PJ(NSV, HVV) \
  project_launch<NSV, HVV>(mx, mq, grid, d_off, d_poff, K, J, Jp, LP, OFF, B1, xpart, nJb, bfi, qs, lptr, items, status, s)
  switch (NS * 8 + hv) {
    case 48 * 8 + 4: DP2_PJ(48, 4); break;
    case 48 * 8 + 2: DP2_PJ(48, 2); break;
    case 64 * 8 + 4: DP2_PJ(64, 4); break;
    case 64 * 8 + 2: DP2_PJ(64, 2); break;
    case 96 * 8 + 2: DP2_PJ(96, 2); break;
    case 96 * 8 + 1: DP2_PJ(96, 1); break;
    case 192 * 8 + 1: DP2_PJ(192, 1); break;
    default: return false;
  }
#undef DP2_PJ
  return true;
}

void launch_omega_t16(const float* om_pad, int Jpad, int LP, int LPN, dpar2_dtype dt, void* out, cudaStream_t s) {
  const int64_t n = (int64_t)LPN * Jpad;
  DP2_COUNTED(tc::k_omega_t16<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(om_pad, Jpad, LP, LPN,
                                                                                     dt == DPAR2_BF16 ? 1 : 0, out));
}

void launch_qsplit(const float* Q, int LP, int NS, int OFF, const int64_t* d_off, const int64_t* d_poff, int K,
                   int64_t Npad, int64_t maxPad, dpar2_dtype dt, void* out, cudaStream_t s) {
  dim3 grid((unsigned)std::max<int64_t>(1, (maxPad + 127) / 128), K);
  DP2_COUNTED(tc::k_qsplit<<<grid, 128, 0, s>>>(Q, LP, NS, OFF, d_off, d_poff, K, Npad, dt == DPAR2_BF16 ? 1 : 0, out));
}

}  // namespace dp2
