// Stage-2 passes over M = [C_1 B_1 ... C_K B_K] (J x KR; Sec. III-B, the
// randomized SVD of the matricized stage-1 factors):
//   sketch      Y2 (J x l)   = M Omega2   = sum_k M_k Omega2_k,
//   projection  B2^T (KR x l) = M^T Q2,   block k = M_k^T Q2,
// with M stored as K blocks M_k (J x R, row-major).  Both are tall-skinny
// FP32 GEMMs bound by the single read of M (about 2 l FMAs per element); they
// run on CUDA cores with packed FP32 FMAs (two per instruction): the sketch
// one row of Y2 per thread, the projection register tiles (4 rows x l/4
// columns per thread) fed by a cp.async double-buffered shared-memory
// pipeline.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace dp2 {

constexpr int S2_THREADS = 128;
constexpr int S2_PJ = 32;   // projection: j per pipeline stage

// ---- sketch: block (j-tile, chunk of kchunk slices) -> Y2p[chunk] (J x LP) ----
// Thread = row j of Y2 (LP accumulators as float2 pairs).  Each warp copies
// the rows of its 32 j's of the next slices' M_k (32 R contiguous floats per
// slice) into a ring of S2_RING shared-memory buffers with cp.async, S2_RING
// - 1 slices ahead of the one it multiplies, so that the loads of M overlap
// the packed FP32 FMAs; the Omega2_k rows of sg slices at a time are staged
// for the whole block and read by every thread (broadcast).
constexpr int S2_ROWS = 128;  // rows j per sketch block (4 warps)
constexpr int S2_RING = 4;    // M_k row buffers per warp

template <int LP>
__global__ void __launch_bounds__(S2_ROWS) k_s2_sketch(const float* __restrict__ Mblk, int K, int J, int R,
                                                       const float* __restrict__ om2, int kchunk, int sg,
                                                       float* __restrict__ Y2p) {
  extern __shared__ __align__(16) float s2s[];  // sg x R x LP Omega2 rows, then 4 x S2_RING x 32 R M rows
  float* oms = s2s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ring = s2s + sg * R * LP + warp * (S2_RING * 32 * R);
  const int jw = blockIdx.x * S2_ROWS + warp * 32;  // first row of this warp
  const int j = jw + lane;
  const int ch = blockIdx.y;
  const int k0 = ch * kchunk, k1 = min(K, k0 + kchunk);
  const bool even = (R & 1) == 0;
  const int nrows = max(0, min(32, J - jw));
  float2 acc[LP / 2];
#pragma unroll
  for (int c = 0; c < LP / 2; ++c) acc[c] = make_float2(0.f, 0.f);
  // copy of slice k's rows jw .. jw + 31 (zero past J) into ring buffer b
  auto issue = [&](int k, int b) {
    const float* src = Mblk + ((int64_t)k * J + jw) * R;
    float* dst = ring + b * 32 * R;
    const int nv = nrows * R;
    if (even) {
      for (int e = lane; e < 16 * R; e += 32) {
        const bool ok = 2 * e < nv;
        cp_async8(dst + 2 * e, ok ? src + 2 * e : Mblk, ok ? 8 : 0);
      }
    } else {
      for (int e = lane; e < 32 * R; e += 32) {
        const bool ok = e < nv;
        cp_async4(dst + e, ok ? src + e : Mblk, ok ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  for (int kg = k0; kg < k1; kg += sg) {
    const int ng = min(sg, k1 - kg);
    __syncthreads();  // every warp is done with the previous group's Omega2 rows
    const float4* src = reinterpret_cast<const float4*>(om2 + (int64_t)kg * R * LP);
    for (int e = threadIdx.x; e < ng * R * LP / 4; e += S2_ROWS) reinterpret_cast<float4*>(oms)[e] = src[e];
    for (int s = 0; s < min(S2_RING - 1, ng); ++s) issue(kg + s, s);
    __syncthreads();
    for (int s = 0; s < ng; ++s) {
      if (s + S2_RING - 1 < ng) {
        issue(kg + s + S2_RING - 1, (s + S2_RING - 1) % S2_RING);
        cp_async_wait<S2_RING - 1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const float* mrow = ring + (s % S2_RING) * 32 * R + lane * R;
      const float* om = oms + s * R * LP;
      if (even) {
        for (int r = 0; r < R; r += 2) {
          const float2 mv = *reinterpret_cast<const float2*>(mrow + r);
          const float2 m0 = make_float2(mv.x, mv.x), m1 = make_float2(mv.y, mv.y);
          const float4* o0 = reinterpret_cast<const float4*>(om + r * LP);
          const float4* o1 = reinterpret_cast<const float4*>(om + (r + 1) * LP);
#pragma unroll
          for (int c4 = 0; c4 < LP / 4; ++c4) {
            const float4 w0 = o0[c4], w1 = o1[c4];
            acc[2 * c4] = ffma2(m0, make_float2(w0.x, w0.y), acc[2 * c4]);
            acc[2 * c4 + 1] = ffma2(m0, make_float2(w0.z, w0.w), acc[2 * c4 + 1]);
            acc[2 * c4] = ffma2(m1, make_float2(w1.x, w1.y), acc[2 * c4]);
            acc[2 * c4 + 1] = ffma2(m1, make_float2(w1.z, w1.w), acc[2 * c4 + 1]);
          }
        }
      } else {
        for (int r = 0; r < R; ++r) {
          const float mv = mrow[r];
          const float2 m2 = make_float2(mv, mv);
          const float4* o4 = reinterpret_cast<const float4*>(om + r * LP);
#pragma unroll
          for (int c4 = 0; c4 < LP / 4; ++c4) {
            const float4 w = o4[c4];
            acc[2 * c4] = ffma2(m2, make_float2(w.x, w.y), acc[2 * c4]);
            acc[2 * c4 + 1] = ffma2(m2, make_float2(w.z, w.w), acc[2 * c4 + 1]);
          }
        }
      }
      __syncwarp();  // every lane is done with this buffer before it is refilled
    }
  }
  if (j < J) {
    float4* dst = reinterpret_cast<float4*>(Y2p + ((int64_t)ch * J + j) * LP);
#pragma unroll
    for (int c4 = 0; c4 < LP / 4; ++c4)
      dst[c4] = make_float4(acc[2 * c4].x, acc[2 * c4].y, acc[2 * c4 + 1].x, acc[2 * c4 + 1].y);
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
  float2 acc[4][CG / 2];  // packed pairs of columns (CG = LP / 4 is even)
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CG / 2; ++c) acc[a][c] = make_float2(0.f, 0.f);
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
      float2 bv[CG / 2];
#pragma unroll
      for (int c = 0; c < CG / 2; ++c) bv[c] = *reinterpret_cast<const float2*>(bs + jj * LP + cg * CG + 2 * c);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float2 m2 = make_float2(av[a], av[a]);
#pragma unroll
        for (int c = 0; c < CG / 2; ++c) acc[a][c] = ffma2(m2, bv[c], acc[a][c]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int row = 4 * rg + a;
    if (row < rows) {
      float* dst = B2p + ((int64_t)kb * R + row) * LP + cg * CG;
#pragma unroll
      for (int c = 0; c < CG / 2; ++c) {
        dst[2 * c] = acc[a][c].x;
        dst[2 * c + 1] = acc[a][c].y;
      }
    }
  }
}

// Chunk of slices per sketch block: about twelve resident blocks per SM, so
// that enough rows are in flight to cover the memory latency.
int s2_sketch_chunk(int K, int J, int num_sms) {
  const int jt = (J + S2_ROWS - 1) / S2_ROWS;
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
  dim3 grid((J + S2_ROWS - 1) / S2_ROWS, nch);
  // Omega2 rows of up to 16 slices per staging round, within 24 KB; the
  // M row rings of the four warps
  const int sg = std::max(1, std::min(16, (24 * 1024) / (R * LP * (int)sizeof(float))));
  const size_t smem = ((size_t)sg * R * LP + (size_t)4 * S2_RING * 32 * R) * sizeof(float);
  DP2_LP_SWITCH(LP, (set_smem_attr(k_s2_sketch<L>, smem),
                     DP2_COUNTED(k_s2_sketch<L><<<grid, S2_ROWS, smem, s>>>(Mblk, K, J, R, om2, kchunk, sg, Y2p))));
}

void launch_s2_project(const float* Mblk, int K, int J, int R, const float* Q2, int LP, float* B2p, cudaStream_t s) {
  const int spb = std::max(1, 128 / R);
  const size_t smem = (size_t)2 * (S2_PJ * 128 + S2_PJ * LP) * sizeof(float);
  DP2_LP_SWITCH(LP, (set_smem_attr(k_s2_project<L>, smem),
                     DP2_COUNTED(k_s2_project<L><<<(unsigned)((K + spb - 1) / spb), S2_THREADS, smem, s>>>(Mblk, K, J, R, Q2,
                                                                                              spb, B2p))));
}

}  // namespace dp2
