// Stage-2 passes over M = [C_1 B_1 ... C_K B_K] (J x KR; Sec. III-B, the
// randomized SVD of the matricized stage-1 factors):
//   sketch      Y2 (J x l)   = M Omega2   = sum_k M_k Omega2_k,
//   projection  B2^T (KR x l) = M^T Q2,   block k = M_k^T Q2,
// with M stored as K blocks M_k (J x R, row-major).  Both are tall-skinny
// FP32 GEMMs bound by the single read of M; they run on CUDA cores with
// register tiles (4 rows x l/4 columns per thread) fed by a cp.async
// double-buffered shared-memory pipeline.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace dp2 {

constexpr int S2_THREADS = 128;
constexpr int S2_JT = 128;  // sketch: rows j per block
constexpr int S2_PJ = 32;   // projection: j per pipeline stage

// ---- sketch: block (j-tile, chunk of kchunk slices) -> Y2p[chunk] (J x LP) ----
// smem per stage: As[R][S2_JT] (M_k tile, transposed), Bs[R][LP] (Omega2_k).
template <int LP>
__global__ void __launch_bounds__(S2_THREADS) k_s2_sketch(const float* __restrict__ Mblk, int K, int J, int R,
                                                          const float* __restrict__ om2, int kchunk,
                                                          float* __restrict__ Y2p) {
  constexpr int CG = LP / 4;
  extern __shared__ __align__(16) float s2sm[];
  // stage b: As(b) = s2sm + b R S2_JT, Bs(b) = s2sm + 2 R S2_JT + b R LP
  float* const as0 = s2sm;
  float* const bs0 = s2sm + 2 * R * S2_JT;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * S2_JT;
  const int ch = blockIdx.y;
  const int k0 = ch * kchunk, k1 = min(K, k0 + kchunk);
  const int jg = tid >> 2, cg = tid & 3;
  float acc[4][CG];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CG; ++c) acc[a][c] = 0.f;
  // element e = tid + q S2_THREADS of a slice tile is (jj, r) = divmod(e, R);
  // stepping q advances it by divmod(S2_THREADS, R)
  const int dq = S2_THREADS / R, dr = S2_THREADS - dq * R;
  const int jj0 = tid / R, r0 = tid - jj0 * R;
  auto stage = [&](int k, int buf) {
    // M_k rows j0 .. j0 + S2_JT - 1 (R floats each, contiguous) -> As[r][jj]
    const float* src = Mblk + ((int64_t)k * J + j0) * R;
    float* dst = as0 + buf * R * S2_JT;
    int jj = jj0, r = r0;
    for (int e = tid; e < S2_JT * R; e += S2_THREADS) {
      const bool ok = j0 + jj < J;
      cp_async4(dst + r * S2_JT + jj, ok ? src + e : Mblk, ok ? 4 : 0);
      jj += dq;
      r += dr;
      if (r >= R) {
        r -= R;
        ++jj;
      }
    }
    const float* osrc = om2 + (int64_t)k * R * LP;
    for (int e = tid; e < R * LP / 4; e += S2_THREADS) cp_async16(bs0 + buf * R * LP + 4 * e, osrc + 4 * e, 16);
    cp_async_commit();
  };
  if (k0 < k1) stage(k0, 0);
  for (int k = k0; k < k1; ++k) {
    const int buf = (k - k0) & 1;
    if (k + 1 < k1) {
      stage(k + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* as = as0 + buf * R * S2_JT;
    const float* bs = bs0 + buf * R * LP;
    for (int r = 0; r < R; ++r) {
      const float4 a4 = *reinterpret_cast<const float4*>(as + r * S2_JT + 4 * jg);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      float bv[CG];
#pragma unroll
      for (int c = 0; c < CG; ++c) bv[c] = bs[r * LP + cg * CG + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
    }
    __syncthreads();
  }
  float* dst = Y2p + (int64_t)ch * J * LP;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int j = j0 + 4 * jg + a;
    if (j < J) {
#pragma unroll
      for (int c = 0; c < CG; ++c) dst[(int64_t)j * LP + cg * CG + c] = acc[a][c];
    }
  }
}

// ---- projection: block of spb slices (rows (k, r)) -> B2p rows ----
// smem per stage: As[S2_PJ][128] (M rows j for the block's (k, r) columns),
// Bs[S2_PJ][LP] (Q2 rows).
template <int LP>
__global__ void __launch_bounds__(S2_THREADS) k_s2_project(const float* __restrict__ Mblk, int K, int J, int R,
                                                           const float* __restrict__ Q2, int spb,
                                                           float* __restrict__ B2p) {
  constexpr int CG = LP / 4;
  extern __shared__ __align__(16) float s2sm[];
  // stage b: As(b) = s2sm + b S2_PJ 128, Bs(b) = s2sm + 2 S2_PJ 128 + b S2_PJ LP
  float* const as0 = s2sm;
  float* const bs0 = s2sm + 2 * S2_PJ * 128;
  const int tid = threadIdx.x;
  const int kb = blockIdx.x * spb;
  const int nk = min(spb, K - kb);
  const int rows = nk * R;  // <= 128
  const int rg = tid >> 2, cg = tid & 3;
  float acc[4][CG];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CG; ++c) acc[a][c] = 0.f;
  // element w = tid + q S2_THREADS of one slice's tile is (jj, r) = divmod(w, R);
  // stepping q advances it by divmod(S2_THREADS, R)
  const int dq = S2_THREADS / R, dr = S2_THREADS - dq * R;
  const int jj0 = tid / R, r0 = tid - jj0 * R;
  auto stage = [&](int j0, int buf) {
    // for every slice s of the block: M_k rows j0 .. j0 + S2_PJ - 1 -> As[jj][s R + r]
    float* dst = as0 + buf * S2_PJ * 128;
    for (int s = 0; s < nk; ++s) {
      const float* src = Mblk + ((int64_t)(kb + s) * J + j0) * R;
      int jj = jj0, r = r0;
      for (int w = tid; w < S2_PJ * R; w += S2_THREADS) {
        const bool ok = j0 + jj < J;
        cp_async4(dst + jj * 128 + s * R + r, ok ? src + w : Mblk, ok ? 4 : 0);
        jj += dq;
        r += dr;
        if (r >= R) {
          r -= R;
          ++jj;
        }
      }
    }
    for (int e = tid; e < S2_PJ * LP / 4; e += S2_THREADS) {
      const int jj = (4 * e) / LP;
      const bool ok = j0 + jj < J;
      cp_async16(bs0 + buf * S2_PJ * LP + 4 * e, ok ? Q2 + (int64_t)j0 * LP + 4 * e : Q2, ok ? 16 : 0);
    }
    cp_async_commit();
  };
  const int nt = (J + S2_PJ - 1) / S2_PJ;
  stage(0, 0);
  for (int t = 0; t < nt; ++t) {
    const int buf = t & 1;
    if (t + 1 < nt) {
      stage((t + 1) * S2_PJ, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* as = as0 + buf * S2_PJ * 128;
    const float* bs = bs0 + buf * S2_PJ * LP;
#pragma unroll 4
    for (int jj = 0; jj < S2_PJ; ++jj) {
      const float4 a4 = *reinterpret_cast<const float4*>(as + jj * 128 + 4 * rg);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      float bv[CG];
#pragma unroll
      for (int c = 0; c < CG; ++c) bv[c] = bs[jj * LP + cg * CG + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int row = 4 * rg + a;
    if (row < rows) {
      float* dst = B2p + ((int64_t)kb * R + row) * LP + cg * CG;
#pragma unroll
      for (int c = 0; c < CG; ++c) dst[c] = acc[a][c];
    }
  }
}

// Chunk of slices per sketch block: about twelve resident blocks per SM, so
// that enough tiles are in flight to cover the memory latency.
int s2_sketch_chunk(int K, int J, int num_sms) {
  const int jt = (J + S2_JT - 1) / S2_JT;
  const int want_chunks = std::max(1, (12 * num_sms + jt - 1) / jt);
  return std::max(1, (K + want_chunks - 1) / want_chunks);
}

template <typename F>
static void set_smem_attr(F* f, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_s2_sketch(const float* Mblk, int K, int J, int R, const float* om2, int LP, float* Y2p, int kchunk,
                      cudaStream_t s) {
  const int nch = (K + kchunk - 1) / kchunk;
  dim3 grid((J + S2_JT - 1) / S2_JT, nch);
  const size_t smem = (size_t)2 * (R * S2_JT + R * LP) * sizeof(float);
  DP2_LP_SWITCH(LP, (set_smem_attr(k_s2_sketch<L>, smem),
                     DP2_COUNTED(k_s2_sketch<L><<<grid, S2_THREADS, smem, s>>>(Mblk, K, J, R, om2, kchunk, Y2p))));
}

void launch_s2_project(const float* Mblk, int K, int J, int R, const float* Q2, int LP, float* B2p, cudaStream_t s) {
  const int spb = std::max(1, 128 / R);
  const size_t smem = (size_t)2 * (S2_PJ * 128 + S2_PJ * LP) * sizeof(float);
  DP2_LP_SWITCH(LP, (set_smem_attr(k_s2_project<L>, smem),
                     DP2_COUNTED(k_s2_project<L><<<(unsigned)((K + spb - 1) / spb), S2_THREADS, smem, s>>>(Mblk, K, J, R, Q2,
                                                                                              spb, B2p))));
}

}  // namespace dp2
