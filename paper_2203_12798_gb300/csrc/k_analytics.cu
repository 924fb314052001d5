// Post-fit analyses of the discovery section (Sec. IV-E) on the fitted
// factors:
//   similarity  S(i, j) = exp(-gamma ||U_i - U_j||_F^2) between slices of one
//               length (Eq. similarity), through the Gram matrix of the
//               flattened U_i: ||U_i - U_j||^2 = n_i + n_j - 2 <U_i, U_j>;
//   top-k       the k largest entries of each row of a score matrix, one
//               index left out per row (k-nearest neighbours, RWR ranking);
//   RWR         random walks with restarts on the similarity graph,
//               r <- (1 - c) A~^T r + c q, A = S without its diagonal, A~ its
//               row-normalised form, for several queries at once;
//   PCC         Pearson correlation coefficients between the rows of V.
//
// The Gram matrix is the one dense contraction here (K^2 L multiply-adds for
// K slices of L = I R entries): it runs on the tensor cores.  The FP32 U is
// split into three bf16 parts, U = P0 + P1 + P2 up to FP32 rounding, and the
// six products Pa Pb^T with a + b <= 2 are accumulated in FP32 in TMEM, which
// leaves the FP32 level of the inputs (the dropped products are below 2^-24
// of the terms).  The kernel is persistent over the tiles of the upper
// triangle (i-block <= j-block) and warp-specialised as the stage-1 passes:
// warp 0 issues TMA loads of the six 128 x 64 bf16 tiles of a K step into a
// two-stage ring, warp 1 issues tcgen05.mma into a double-buffered 128 x 128
// FP32 accumulator, warps 2-5 read it back (one row per thread), form S and
// store the tile and its mirror image.  Every mbarrier wait is bounded.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace dp2 {
namespace tc {

constexpr int SM_BM = 128, SM_BK = 64, SM_STAGES = 2;
constexpr int SM_TILE = SM_BM * SM_BK * 2;  // bytes of one 128 x 64 bf16 tile
constexpr int SM_STAGE = 6 * SM_TILE;       // A0 A1 A2 B0 B1 B2
constexpr int SM_SMEM = 1024 + SM_STAGES * SM_STAGE + 256;

// (bi, bj), bi <= bj, of tile t of the upper triangle of nb x nb blocks, row by row
__device__ __forceinline__ void tri_tile(int64_t t, int nb, int& bi, int& bj) {
  int i = 0;
  int64_t rem = t;
  while (rem >= nb - i) {
    rem -= nb - i;
    ++i;
  }
  bi = i;
  bj = i + (int)rem;
}

__global__ void __launch_bounds__(192, 1) k_sim_tc(const __grid_constant__ CUtensorMap m0,
                                                   const __grid_constant__ CUtensorMap m1,
                                                   const __grid_constant__ CUtensorMap m2, int K, int L,
                                                   const double* __restrict__ nrm, float gamma, float* __restrict__ S,
                                                   int64_t lds, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + SM_STAGES * SM_STAGE);
  uint64_t* empty = full + SM_STAGES;
  uint64_t* accfull = empty + SM_STAGES;
  uint64_t* accempty = accfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = (K + SM_BM - 1) / SM_BM;
  const int64_t ntiles = (int64_t)nb * (nb + 1) / 2;
  const int nk = (L + SM_BK - 1) / SM_BK;
  constexpr uint32_t NCOL = 256;  // two 128-column FP32 accumulators

  if (threadIdx.x == 0) {
    for (int s = 0; s < SM_STAGES; ++s) {
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
    prefetch_tmap(&m0);
    prefetch_tmap(&m1);
    prefetch_tmap(&m2);
    const CUtensorMap* maps[3] = {&m0, &m1, &m2};
    int s = 0;
    uint32_t ph = 0, inflight = 0;
    for (int64_t t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
      int bi, bj;
      tri_tile(t, nb, bi, bj);
      for (int kc = 0; kc < nk; ++kc) {
        if (!wait_bounded(&empty[s], ph ^ 1, abort_flag)) break;
        mbar_arrive_expect_tx(&full[s], SM_STAGE);
        uint8_t* st = base + s * SM_STAGE;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          tma_load_2d(st + p * SM_TILE, maps[p], &full[s], kc * SM_BK, bi * SM_BM);
          tma_load_2d(st + (3 + p) * SM_TILE, maps[p], &full[s], kc * SM_BK, bj * SM_BM);
        }
        inflight = 1;
        if (++s == SM_STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    if (*abort_flag && inflight) {
      const int ls = (s + SM_STAGES - 1) % SM_STAGES;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&full[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idesc = idesc_f16(SM_BM, SM_BM, true, false, false);
    int s = 0;
    uint32_t ph = 0;
    int tl = 0;
    bool issued = false;
    for (int64_t t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tl) {
      const int acc = tl & 1;
      const uint32_t aph = (tl >> 1) & 1;
      if (!wait_bounded(&accempty[acc], aph ^ 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * SM_BM;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc) {
        if (!wait_bounded(&full[s], ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(base + s * SM_STAGE);
        uint64_t da[3], db[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          da[p] = sdesc_sw128(st + p * SM_TILE, 16, 1024);
          db[p] = sdesc_sw128(st + (3 + p) * SM_TILE, 16, 1024);
        }
#pragma unroll
        for (int kk = 0; kk < SM_BK / 16; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);  // 16 bf16 = 32 bytes along K
          tc_mma(d, da[0] + o, db[0] + o, idesc, (kc | kk) != 0 ? 1u : 0u);
          tc_mma(d, da[0] + o, db[1] + o, idesc, 1u);
          tc_mma(d, da[1] + o, db[0] + o, idesc, 1u);
          tc_mma(d, da[0] + o, db[2] + o, idesc, 1u);
          tc_mma(d, da[2] + o, db[0] + o, idesc, 1u);
          tc_mma(d, da[1] + o, db[1] + o, idesc, 1u);
        }
        tc_commit(&empty[s]);
        issued = true;
        if (++s == SM_STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      tc_commit(&accfull[acc]);
    }
    if (*abort_flag && issued) {
      const int ls = (s + SM_STAGES - 1) % SM_STAGES;
      const uint32_t lph = (s == 0) ? (ph ^ 1) : ph;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&empty[ls], lph) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31
    int tl = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      int bi, bj;
      tri_tile(t, nb, bi, bj);
      const int acc = tl & 1;
      const uint32_t aph = (tl >> 1) & 1;
      if (!wait_bounded(&accfull[acc], aph, abort_flag)) break;
      tc_fence_after();
      const int i = bi * SM_BM + q * 32 + lane;
      const double ni = i < K ? nrm[i] : 0.0;
      for (int g = 0; g < SM_BM / 32; ++g) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * SM_BM + g * 32, v);
        const int j0 = bj * SM_BM + g * 32;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int j = j0 + c;
          float sv = 0.f;
          if (i < K && j < K) {
            const double d2 = fmax(ni + nrm[j] - 2.0 * (double)v[c], 0.0);
            sv = (i == j) ? 1.f : expf(-gamma * (float)d2);
          }
          v[c] = sv;
        }
        // a diagonal tile writes its upper triangle and mirrors it (the MMA
        // sums G(i, j) and G(j, i) in different orders), so S is symmetric
        if (i < K) {
          float* row = S + (int64_t)i * lds + j0;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (j0 + c < K && (bi != bj || j0 + c >= i)) row[c] = v[c];
        }
        // the mirror: column i of rows j (a warp writes 32 consecutive i)
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int j = j0 + c;
          if (i < K && j < K && (bi != bj || j > i)) S[(int64_t)j * lds + i] = v[c];
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

}  // namespace tc

// ---------------------------------------------------------------- split ----
// Row i of U (L floats, pitch ldu) -> three bf16 parts (pitch ldp, zero past
// L) with u = p0 + p1 + p2 up to FP32 rounding, and n_i = sum_l u_il^2 (FP64).
// One block per row.
__global__ void k_sim_split(const float* __restrict__ U, int64_t ldu, int L, int ldp, __nv_bfloat16* __restrict__ P0,
                            __nv_bfloat16* __restrict__ P1, __nv_bfloat16* __restrict__ P2,
                            double* __restrict__ nrm) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  const float* u = U + i * ldu;
  double s = 0.0;
  for (int l = threadIdx.x; l < ldp; l += blockDim.x) {
    const float x = l < L ? u[l] : 0.f;
    const __nv_bfloat16 a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);
    P0[i * ldp + l] = a;
    P1[i * ldp + l] = b;
    P2[i * ldp + l] = __float2bfloat16_rn(r2);
    s = fma((double)x, (double)x, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    nrm[i] = t;
  }
}

// ---------------------------------------------------------------- top-k ----
// Block per row: the k largest scores (ties: lower index first) among the
// columns j != exclude[row] (exclude may be null or hold -1).  Every thread
// keeps its own top-k of a strided share of the row (insertion into a sorted
// register list), then k rounds of a block-wide argmax over the threads' list
// heads pick the result in order.
constexpr int TOPK_MAX = 16;
constexpr int TOPK_THREADS = 256;

__device__ __forceinline__ bool topk_better(float va, int ia, float vb, int ib) {
  return va > vb || (va == vb && ia < ib);
}

__global__ void __launch_bounds__(TOPK_THREADS) k_topk(const float* __restrict__ sc, int64_t ld, int n,
                                                        const int* __restrict__ exclude, int k, int* __restrict__ idx,
                                                        float* __restrict__ val) {
  __shared__ float hv[TOPK_THREADS];
  __shared__ int hi[TOPK_THREADS], ht[TOPK_THREADS];
  __shared__ float lv[TOPK_THREADS * TOPK_MAX];
  __shared__ int li[TOPK_THREADS * TOPK_MAX];
  const int row = blockIdx.x, t = threadIdx.x;
  const float* r = sc + (int64_t)row * ld;
  const int ex = exclude ? exclude[row] : -1;
  float v[TOPK_MAX];
  int ix[TOPK_MAX];
  int cnt = 0;
  for (int j = t; j < n; j += TOPK_THREADS) {
    if (j == ex) continue;
    const float x = r[j];
    if (cnt == k && !topk_better(x, j, v[k - 1], ix[k - 1])) continue;
    int pos = cnt < k ? cnt++ : k - 1;
    while (pos > 0 && topk_better(x, j, v[pos - 1], ix[pos - 1])) {
      v[pos] = v[pos - 1];
      ix[pos] = ix[pos - 1];
      --pos;
    }
    v[pos] = x;
    ix[pos] = j;
  }
  for (int u = 0; u < cnt; ++u) {
    lv[t * TOPK_MAX + u] = v[u];
    li[t * TOPK_MAX + u] = ix[u];
  }
  int head = 0;
  for (int out = 0; out < k; ++out) {
    hv[t] = head < cnt ? lv[t * TOPK_MAX + head] : -INFINITY;
    hi[t] = head < cnt ? li[t * TOPK_MAX + head] : 0x7fffffff;
    ht[t] = t;
    __syncthreads();
    for (int w = TOPK_THREADS / 2; w > 0; w >>= 1) {
      if (t < w && topk_better(hv[t + w], hi[t + w], hv[t], hi[t])) {
        hv[t] = hv[t + w];
        hi[t] = hi[t + w];
        ht[t] = ht[t + w];
      }
      __syncthreads();
    }
    if (t == 0) {
      idx[(int64_t)row * k + out] = hi[0] == 0x7fffffff ? -1 : hi[0];
      val[(int64_t)row * k + out] = hv[0];
    }
    const int win = ht[0];
    __syncthreads();
    if (t == win) ++head;
  }
}

// ------------------------------------------------------------------ RWR ----
// Degrees d_i = sum_{j != i} S(i, j) (FP64 sum per row, warp per row).
__global__ void k_rwr_degree(int K, const float* __restrict__ S, int64_t lds, double* __restrict__ deg) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= K) return;
  const float* r = S + (int64_t)w * lds;
  double s = 0.0;
  for (int j = lane; j < K; j += 32)
    if (j != w) s += (double)r[j];
  s = warp_sum(s);
  if (lane == 0) deg[w] = s;
}

// The iterates are kept query-fastest, y[j][q] with NQ = 4 NQ4 floats per
// column j (nq <= NQ queries, the rest zero), so that one column of all
// queries is NQ4 float4 loads.
constexpr int RWR_MAXQ = 16;
constexpr int RWR_ROWS = 4;   // rows of S per block (the y loads serve all of them)
constexpr int RWR_WARPS = 8;  // warps per block, splitting the columns

// y[j][q] = r[q][j] / d_j for the starting vector r = q (one-hot at the target);
// r is written query-major (nq x K) as the output.
__global__ void k_rwr_init(int K, int nq, int NQ, const int* __restrict__ tgt, const double* __restrict__ deg,
                           float* __restrict__ r, float* __restrict__ y) {
  const int64_t n = (int64_t)K * NQ;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / NQ), q = (int)(e - (int64_t)j * NQ);
    const float v = (q < nq && j == tgt[q]) ? 1.f : 0.f;
    if (q < nq) r[(int64_t)q * K + j] = v;
    y[e] = deg[j] > 0.0 ? (float)(v / deg[j]) : 0.f;
  }
}

// One step for every query: r'(q, i) = (1 - c) sum_{j != i} S(i, j) y(q, j) +
// c [i == t_q], since A~^T r = A D^-1 r for the symmetric A; then
// y'(q, i) = r'(q, i) / d_i.  A block takes RWR_ROWS rows; its threads walk
// the columns j (two at a time), load y(:, j) once and apply it to every row;
// the partial sums meet through warp shuffles and shared memory.
template <int NQ4>
__global__ void __launch_bounds__(32 * RWR_WARPS) k_rwr_step(int K, int nq, const float* __restrict__ S, int64_t lds,
                                                            const int* __restrict__ tgt,
                                                            const double* __restrict__ deg, float c,
                                                            const float* __restrict__ y, float* __restrict__ rn,
                                                            float* __restrict__ yn) {
  constexpr int NQ = 4 * NQ4;
  __shared__ float part[RWR_WARPS][RWR_ROWS * NQ];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, T = blockDim.x;
  const int i0 = blockIdx.x * RWR_ROWS;
  float acc[RWR_ROWS][NQ];
#pragma unroll
  for (int a = 0; a < RWR_ROWS; ++a)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[a][q] = 0.f;
  const float4* y4 = reinterpret_cast<const float4*>(y);
  auto column = [&](int j) {
    float sv[RWR_ROWS];
#pragma unroll
    for (int a = 0; a < RWR_ROWS; ++a) {
      const int i = i0 + a;
      sv[a] = (i < K && j != i) ? S[(int64_t)i * lds + j] : 0.f;
    }
    float4 t[NQ4];
#pragma unroll
    for (int u = 0; u < NQ4; ++u) t[u] = y4[(int64_t)j * NQ4 + u];
#pragma unroll
    for (int a = 0; a < RWR_ROWS; ++a)
#pragma unroll
      for (int u = 0; u < NQ4; ++u) {
        acc[a][4 * u] = fmaf(sv[a], t[u].x, acc[a][4 * u]);
        acc[a][4 * u + 1] = fmaf(sv[a], t[u].y, acc[a][4 * u + 1]);
        acc[a][4 * u + 2] = fmaf(sv[a], t[u].z, acc[a][4 * u + 2]);
        acc[a][4 * u + 3] = fmaf(sv[a], t[u].w, acc[a][4 * u + 3]);
      }
  };
  int j = threadIdx.x;
  for (; j + T < K; j += 2 * T) {
    column(j);
    column(j + T);
  }
  if (j < K) column(j);
#pragma unroll
  for (int a = 0; a < RWR_ROWS; ++a)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float v = warp_sum(acc[a][q]);
      if (lane == 0) part[warp][a * NQ + q] = v;
    }
  __syncthreads();
  if (threadIdx.x < RWR_ROWS * NQ) {
    const int a = threadIdx.x / NQ, q = threadIdx.x - a * NQ, i = i0 + a;
    float s = 0.f;
    for (int w = 0; w < RWR_WARPS; ++w) s += part[w][threadIdx.x];
    if (i < K) {
      const float v = q < nq ? (1.f - c) * s + (i == tgt[q] ? c : 0.f) : 0.f;
      if (q < nq) rn[(int64_t)q * K + i] = v;
      yn[(int64_t)i * NQ + q] = deg[i] > 0.0 ? (float)(v / deg[i]) : 0.f;
    }
  }
}

// ------------------------------------------------------------------ PCC ----
// Rows of V centred and scaled to unit norm (FP64 mean and norm), one warp per row.
__global__ void k_pcc_rows(int J, int R, const float* __restrict__ V, float* __restrict__ Vn) {
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (a >= J) return;
  double m = 0.0;
  for (int r = lane; r < R; r += 32) m += (double)V[(int64_t)a * R + r];
  m = warp_sum(m) / R;
  double n2 = 0.0;
  for (int r = lane; r < R; r += 32) {
    const double d = (double)V[(int64_t)a * R + r] - m;
    n2 += d * d;
  }
  n2 = warp_sum(n2);
  const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : __longlong_as_double(0x7ff8000000000000ll);
  for (int r = lane; r < R; r += 32) Vn[(int64_t)a * R + r] = (float)(((double)V[(int64_t)a * R + r] - m) * inv);
}

// C(a, b) = sum_r Vn(a, r) Vn(b, r): 16 x 16 tiles, FP32 products summed in FP64.
__global__ void k_pcc_gram(int J, int R, const float* __restrict__ Vn, float* __restrict__ C) {
  const int a = blockIdx.y * 16 + threadIdx.y, b = blockIdx.x * 16 + threadIdx.x;
  if (a >= J || b >= J) return;
  double s = 0.0;
  for (int r = 0; r < R; ++r) s = fma((double)Vn[(int64_t)a * R + r], (double)Vn[(int64_t)b * R + r], s);
  C[(int64_t)a * J + b] = (float)s;
}

// ---------------------------------------------------------------- launchers --
bool launch_similarity(int K, int L, const float* U, int64_t ldu, double gamma, float* S, int64_t lds, void* parts,
                       int ldp, double* nrm, int num_sms, int* status, cudaStream_t s) {
  __nv_bfloat16* pb = static_cast<__nv_bfloat16*>(parts);
  __nv_bfloat16* P[3] = {pb, pb + (size_t)K * ldp, pb + (size_t)2 * K * ldp};
  DP2_COUNTED(k_sim_split<<<K, 128, 0, s>>>(U, ldu, L, ldp, P[0], P[1], P[2], nrm));
  CUtensorMap m[3];
  for (int p = 0; p < 3; ++p)
    if (!make_map(&m[p], P[p], true, (uint64_t)ldp, (uint64_t)K, (uint64_t)ldp, tc::SM_BK, tc::SM_BM)) return false;
  const int nb = (K + tc::SM_BM - 1) / tc::SM_BM;
  const int64_t ntiles = (int64_t)nb * (nb + 1) / 2;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_sim_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SM_SMEM);
    attr = true;
  }
  DP2_COUNTED(tc::k_sim_tc<<<grid, 192, tc::SM_SMEM, s>>>(m[0], m[1], m[2], K, ldp, nrm, (float)gamma, S, lds, status));
  return true;
}

void launch_topk(int nrows, int n, const float* sc, int64_t ld, const int* exclude, int k, int* idx, float* val,
                 cudaStream_t s) {
  DP2_COUNTED(k_topk<<<nrows, TOPK_THREADS, 0, s>>>(sc, ld, n, exclude, k, idx, val));
}

int rwr_max_queries() { return RWR_MAXQ; }

// r (nq x K) <- the scores after `iters` steps from r = q; y0, y1: K x 16
// floats of scratch for the degree-scaled iterates, deg: K doubles.
void launch_rwr(int K, const float* S, int64_t lds, int nq, const int* tgt, double c, int iters, double* deg,
                float* r, float* y0, float* y1, cudaStream_t s) {
  const int wpb = 8;
  DP2_COUNTED(k_rwr_degree<<<(unsigned)((K + wpb - 1) / wpb), 32 * wpb, 0, s>>>(K, S, lds, deg));
  const int nq4 = (nq + 3) / 4;
  DP2_COUNTED(k_rwr_init<<<256, 256, 0, s>>>(K, nq, 4 * nq4, tgt, deg, r, y0));
  const unsigned gs = (unsigned)((K + RWR_ROWS - 1) / RWR_ROWS);
  float* ya = y0;
  float* yb = y1;
  for (int it = 0; it < iters; ++it) {
    switch (nq4) {
      case 1: DP2_COUNTED(k_rwr_step<1><<<gs, 32 * RWR_WARPS, 0, s>>>(K, nq, S, lds, tgt, deg, (float)c, ya, r, yb)); break;
      case 2: DP2_COUNTED(k_rwr_step<2><<<gs, 32 * RWR_WARPS, 0, s>>>(K, nq, S, lds, tgt, deg, (float)c, ya, r, yb)); break;
      case 3: DP2_COUNTED(k_rwr_step<3><<<gs, 32 * RWR_WARPS, 0, s>>>(K, nq, S, lds, tgt, deg, (float)c, ya, r, yb)); break;
      default: DP2_COUNTED(k_rwr_step<4><<<gs, 32 * RWR_WARPS, 0, s>>>(K, nq, S, lds, tgt, deg, (float)c, ya, r, yb)); break;
    }
    std::swap(ya, yb);
  }
}

void launch_feature_pcc(int J, int R, const float* V, float* Vn, float* C, cudaStream_t s) {
  DP2_COUNTED(k_pcc_rows<<<(unsigned)((J + 7) / 8), 256, 0, s>>>(J, R, V, Vn));
  DP2_COUNTED(k_pcc_gram<<<dim3((unsigned)((J + 15) / 16), (unsigned)((J + 15) / 16)), dim3(16, 16), 0, s>>>(J, R, Vn, C));
}

}  // namespace dp2
