// Stage-2 passes over M = [C_1 B_1 ... C_K B_K] (J x KR; Sec. III-B, the
// randomized SVD of the matricized stage-1 factors) on the tensor cores:
//   sketch      Y2 (J x l)    = M Omega2   (reduction over the KR columns of M)
//   projection  B2^T (KR x l) = M^T Q2     (reduction over the J rows of M)
// M is held as M^T (KR x Jq, Jq = J rounded up to 64, zero columns past J) in
// three BF16 parts whose sum is M exactly (written by the M-block kernels);
// the FP32 right operand (Omega2 or Q2) is split the same way, its parts
// stacked as rows p LP + c of an NB x K-extent BF16 matrix (NB = 3 LP rounded
// up to 16).  Per K step, three MMAs (one per part of M) accumulate all nine
// part products into one FP32 accumulator of NB columns, and the epilogue adds
// the three column groups: FP32 accuracy from 16-bit operands, M read once per
// pass (6 bytes per element).
//
// One kernel serves both passes (template MNA):
//   sketch      MMA M = 128 columns j of M, K = rows kr of M^T: each part's A
//               tile is M^T rows seen MN-major (two 64-column atoms 8 KB
//               apart, 8-row K groups 1 KB apart); B = split Omega2^T rows.
//   projection  MMA M = 128 rows kr of M^T, K = columns j: A K-major; B =
//               split Q2^T rows.
// Work item = (M tile, chunk of K steps); the item writes its partial output
// rows (LP floats each) to part[chunk], and a fixed-order sum over the chunks
// follows.  Warp roles as in the stage-1 passes: warp 0 issues the TMA loads,
// warp 1 the MMAs (TMEM accumulator double buffered across items), warps 2-5
// drain the accumulator.  Every mbarrier wait is bounded; on a timeout every
// role stops, waits (bounded) for its copies / MMAs in flight, TMEM is freed
// and the status word gets ST_TIMEOUT.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace dp2 {
namespace tc {

constexpr int S2T_BM = 128, S2T_BK = 64, S2T_ST = 3, S2T_THREADS = 192;
constexpr int S2T_PART = S2T_BM * S2T_BK * 2;  // one part's A tile: 16 KB

template <int NB>
struct S2Smem {
  static constexpr int A = 3 * S2T_PART;
  static constexpr int B = NB * S2T_BK * 2;
  static constexpr int ACC = (NB + 31) / 32 * 32;  // TMEM columns per accumulator
  static constexpr uint32_t NCOL = 2 * ACC <= 64 ? 64 : (2 * ACC <= 128 ? 128 : (2 * ACC <= 256 ? 256 : 512));
  static constexpr int BYTES = 1024 + S2T_ST * (A + B) + 256;
  static_assert(B % 1024 == 0, "B tiles must stay 1024-byte aligned");
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

// Item `it` -> (M tile, first and last K step).
__device__ __forceinline__ void s2t_item(int64_t it, int nmt, int nks, int nchunk, int* mt, int* k0, int* k1) {
  *mt = (int)(it % nmt);
  const int c = (int)(it / nmt);
  *k0 = (int)((int64_t)c * nks / nchunk);
  *k1 = (int)((int64_t)(c + 1) * nks / nchunk);
}

template <bool MNA, int LP>
__global__ void __launch_bounds__(S2T_THREADS, 1) k_s2_tc(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, int nrows,
                                                          int nmt, int nks, int nchunk, float* __restrict__ part,
                                                          int* status) {
  constexpr int NB = (3 * LP + 15) / 16 * 16;
  using S = S2Smem<NB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint8_t* sA = base;
  uint8_t* sB = base + S2T_ST * S::A;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + S2T_ST * S::B);
  uint64_t* empty = full + S2T_ST;
  uint64_t* accfull = empty + S2T_ST;
  uint64_t* accempty = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nitems = (int64_t)nmt * nchunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S2T_ST; ++s) {
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
    tmem_alloc(tslot, S::NCOL);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    const uint64_t pol_a = policy_evict_first();  // M: streamed once
    const uint64_t pol_b = policy_evict_last();   // right operand: shared by every M tile
    int s = 0;
    uint32_t ph = 0, inflight = 0;
    for (int64_t it = blockIdx.x; it < nitems && !*abort_flag; it += gridDim.x) {
      int mt, k0, k1;
      s2t_item(it, nmt, nks, nchunk, &mt, &k0, &k1);
      for (int kc = k0; kc < k1; ++kc) {
        if (!wait_bounded(&empty[s], ph ^ 1, abort_flag)) break;
        mbar_arrive_expect_tx(&full[s], S::A + S::B);
        uint8_t* a = sA + s * S::A;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if (MNA) {
            // M^T rows kc*64 .. +63, columns mt*128 .. +127 as two 64-column boxes
            tma_load_3d_hint(a + p * S2T_PART, &tmA, &full[s], mt * S2T_BM, kc * S2T_BK, p, pol_a);
            tma_load_3d_hint(a + p * S2T_PART + S2T_PART / 2, &tmA, &full[s], mt * S2T_BM + 64, kc * S2T_BK, p,
                             pol_a);
          } else {
            // M^T rows mt*128 .. +127, columns kc*64 .. +63
            tma_load_3d_hint(a + p * S2T_PART, &tmA, &full[s], kc * S2T_BK, mt * S2T_BM, p, pol_a);
          }
        }
        tma_load_2d_hint(sB + s * S::B, &tmB, &full[s], kc * S2T_BK, 0, pol_b);
        inflight = 1;
        if (++s == S2T_ST) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    if (*abort_flag && inflight) {
      const int ls = (s + S2T_ST - 1) % S2T_ST;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&full[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idesc = idesc_f16(S2T_BM, NB, true, MNA, false);
    int s = 0;
    uint32_t ph = 0;
    int t = 0;
    bool issued = false;
    for (int64_t it = blockIdx.x; it < nitems && !*abort_flag; it += gridDim.x, ++t) {
      int mt, k0, k1;
      s2t_item(it, nmt, nks, nchunk, &mt, &k0, &k1);
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accempty[acc], aph ^ 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * S::ACC;
      bool ok = true;
      for (int kc = k0; kc < k1; ++kc) {
        if (!wait_bounded(&full[s], ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t bd = sdesc_sw128(smem_u32(sB + s * S::B), 16, 1024);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const uint32_t aaddr = smem_u32(sA + s * S::A + p * S2T_PART);
          const uint64_t ad = MNA ? sdesc_sw128(aaddr, 8192, 1024) : sdesc_sw128(aaddr, 16, 1024);
#pragma unroll
          for (int kk = 0; kk < S2T_BK / 16; ++kk)
            tc_mma(d, ad + (uint64_t)(MNA ? kk * 128 : kk * 2), bd + (uint64_t)(kk * 2), idesc,
                   (kc != k0 || p != 0 || kk != 0) ? 1u : 0u);
        }
        tc_commit(&empty[s]);
        issued = true;
        if (++s == S2T_ST) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      tc_commit(&accfull[acc]);
    }
    if (*abort_flag && issued) {
      const int ls = (s + S2T_ST - 1) % S2T_ST;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&empty[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    int t = 0;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x, ++t) {
      int mt, k0, k1;
      s2t_item(it, nmt, nks, nchunk, &mt, &k0, &k1);
      const int acc = t & 1;
      const uint32_t aph = (t >> 1) & 1;
      if (!wait_bounded(&accfull[acc], aph, abort_flag)) break;
      tc_fence_after();
      // column p LP + c holds the products with part p of the right operand
      float o[LP];
#pragma unroll
      for (int c = 0; c < LP; ++c) o[c] = 0.f;
#pragma unroll
      for (int g = S::ACC / 32 - 1; g >= 0; --g) {  // lo parts first
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * S::ACC + g * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (g * 32 + i < 3 * LP) o[(g * 32 + i) % LP] += v[i];
      }
      tc_fence_before();
      mbar_arrive(&accempty[acc]);
      const int row = mt * S2T_BM + q * 32 + lane;
      const int c = (int)(it / nmt);
      if (row < nrows) {
        float4* dst = reinterpret_cast<float4*>(part + ((int64_t)c * nrows + row) * LP);
#pragma unroll
        for (int c4 = 0; c4 < LP / 4; ++c4) dst[c4] = make_float4(o[4 * c4], o[4 * c4 + 1], o[4 * c4 + 2], o[4 * c4 + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, S::NCOL);
  }
  if (threadIdx.x == 0 && *abort_flag) set_status(status, ST_TIMEOUT);
}

// Right operand split: F (nf x LP FP32, row-major) -> Bs (NB x bcols BF16),
// row p LP + c = part p of column c of F (F = part 0 + part 1 + part 2
// exactly), columns past nf and rows past 3 LP zero.  One thread per row of F.
__global__ void k_s2_split_rhs(const float* __restrict__ F, int64_t nf, int LP, int NB, int64_t bcols,
                               __nv_bfloat16* __restrict__ Bs) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < bcols; x += (int64_t)gridDim.x * blockDim.x) {
    for (int c4 = 0; c4 < LP / 4; ++c4) {
      const float4 v = x < nf ? reinterpret_cast<const float4*>(F + x * LP)[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float w[4] = {v.x, v.y, v.z, v.w};
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * c4 + u;
        __nv_bfloat16 h, m, l;
        split3_bf16(w[u], &h, &m, &l);
        Bs[(int64_t)c * bcols + x] = h;
        Bs[(int64_t)(LP + c) * bcols + x] = m;
        Bs[(int64_t)(2 * LP + c) * bcols + x] = l;
      }
    }
    for (int r = 3 * LP; r < NB; ++r) Bs[(int64_t)r * bcols + x] = __float2bfloat16_rn(0.f);
  }
}

// M (K x J x R FP32, block k = C_k B_k) from its three BF16 parts of M^T.
__global__ void k_ms_to_m(const __nv_bfloat16* __restrict__ Ms, int64_t pstride, int K, int J, int Jq, int R,
                          float* __restrict__ M) {
  const int64_t n = (int64_t)K * J * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / ((int64_t)J * R);
    const int j = (int)((i / R) % J), r = (int)(i % R);
    const int64_t e = (k * R + r) * Jq + j;
    M[i] = (__bfloat162float(Ms[e + 2 * pstride]) + __bfloat162float(Ms[e + pstride])) + __bfloat162float(Ms[e]);
  }
}

}  // namespace tc

// Chunks of the K steps: the fewest that keep the slowest CTA's share of K
// steps (rounds of items x steps per item, plus one step of overhead per item)
// near the even split over the SMs.
int s2_chunks(int nmt, int nks, int num_sms) {
  int best = 1;
  int64_t bestc = INT64_MAX;
  for (int S = 1; S <= std::min(nks, 64); ++S) {
    const int64_t items = (int64_t)nmt * S;
    const int64_t rounds = (items + num_sms - 1) / num_sms;
    const int64_t cost = rounds * ((nks + S - 1) / S + 1);
    if (cost < bestc) {
      bestc = cost;
      best = S;
    }
  }
  return best;
}

template <bool MNA, int LP>
static void s2_launch(const CUtensorMap& ma, const CUtensorMap& mb, int grid, int nrows, int nmt, int nks, int nch,
                      float* part, int* status, cudaStream_t s) {
  constexpr int NB = (3 * LP + 15) / 16 * 16;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_s2_tc<MNA, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::S2Smem<NB>::BYTES);
    attr = true;
  }
  DP2_COUNTED(tc::k_s2_tc<MNA, LP><<<grid, tc::S2T_THREADS, tc::S2Smem<NB>::BYTES, s>>>(ma, mb, nrows, nmt, nks, nch,
                                                                                        part, status));
}

int s2_nb(int LP) { return (3 * LP + 15) / 16 * 16; }

bool launch_s2_tc(bool sketch, const void* Ms, int64_t KR, int J, int Jq, const void* Bs, int64_t bcols, int LP,
                  float* part, int nch, int num_sms, int* status, cudaStream_t s) {
  CUtensorMap ma, mb;
  const int NB = s2_nb(LP);
  if (!make_map3_rows(&ma, Ms, (uint64_t)Jq, (uint64_t)KR, 3, 64, sketch ? 64 : 128)) return false;
  if (!make_map(&mb, Bs, true, (uint64_t)bcols, (uint64_t)NB, (uint64_t)bcols, 64, (uint32_t)NB)) return false;
  const int nrows = sketch ? J : (int)KR;
  const int nmt = (nrows + tc::S2T_BM - 1) / tc::S2T_BM;
  const int nks = (int)((sketch ? KR : (int64_t)Jq) + tc::S2T_BK - 1) / tc::S2T_BK;
  const int grid = (int)std::min<int64_t>((int64_t)nmt * nch, num_sms);
  bool ok = false;
  DP2_LP_SWITCH(LP, (sketch ? s2_launch<true, L>(ma, mb, grid, nrows, nmt, nks, nch, part, status, s)
                            : s2_launch<false, L>(ma, mb, grid, nrows, nmt, nks, nch, part, status, s),
                     ok = true));
  return ok;
}

int s2_tc_chunks(bool sketch, int64_t KR, int J, int Jq, int num_sms) {
  const int nrows = sketch ? J : (int)KR;
  const int nmt = (nrows + tc::S2T_BM - 1) / tc::S2T_BM;
  const int nks = (int)((sketch ? KR : (int64_t)Jq) + tc::S2T_BK - 1) / tc::S2T_BK;
  return s2_chunks(nmt, nks, num_sms);
}

void launch_s2_split_rhs(const float* F, int64_t nf, int LP, int64_t bcols, void* Bs, cudaStream_t s) {
  const int64_t g = std::min<int64_t>((bcols + 255) / 256, 4096);
  DP2_COUNTED(tc::k_s2_split_rhs<<<(unsigned)std::max<int64_t>(g, 1), 256, 0, s>>>(
      F, nf, LP, s2_nb(LP), bcols, static_cast<__nv_bfloat16*>(Bs)));
}

void launch_ms_to_m(const void* Ms, int64_t pstride, int K, int J, int Jq, int R, float* M, cudaStream_t s) {
  const int64_t n = (int64_t)K * J * R;
  const int64_t g = std::min<int64_t>((n + 255) / 256, 8192);
  DP2_COUNTED(tc::k_ms_to_m<<<(unsigned)std::max<int64_t>(g, 1), 256, 0, s>>>(
      static_cast<const __nv_bfloat16*>(Ms), pstride, K, J, Jq, R, M));
}

}  // namespace dp2
