// Stage 1 of the two-stage compression (Sec. III-B, Eq. fstage_svd), CUDA-core
// kernels: the sketch pass Y = X Omega (Alg. 1, "construct Y") and the
// projection pass B = Q^T X (Alg. 1, "construct B"), both streaming X from HBM
// with 16-byte loads.  All K slices run in one launch (rows of every slice
// are tiled together in the sketch; one block per (slice, column block) in
// the projection).  These kernels serve FP32 X and any X whose rows are not
// 16-byte aligned for the tensor-core path.
#include "common.cuh"
#include "internal.h"

namespace dp2 {

// ------------------------------------------------------------------ sketch --
// Y (N x LP) = X (N x J) * Omega_pad (Jpad x LP).  One thread owns RPT rows
// and all LP outputs of each; X is staged through shared memory in chunks
// of 64 bytes per row (cp.async double buffering), Omega rows are read as
// warp-uniform (broadcast) vectors.
constexpr int SK_THREADS = 256;
constexpr int SK_ROWB = 64;   // bytes of a row per chunk
constexpr int SK_PITCH = 80;  // smem row pitch (bytes): 5 x 16 -> conflict-free 16B reads

template <typename T, int LP>
struct SkCfg {
  static constexpr int RPT = LP <= 32 ? 2 : 1;
  static constexpr int ROWS = SK_THREADS * RPT;
  static constexpr int JC = SK_ROWB / (int)sizeof(T);  // elements per chunk
  static constexpr int VN = 16 / (int)sizeof(T);       // elements per 16-byte vector
  static constexpr int XS_BYTES = ROWS * SK_PITCH;
  static constexpr int OS_BYTES = JC * LP * 4;
  static constexpr int SMEM = 2 * (XS_BYTES + OS_BYTES);
};

template <typename T, int LP>
__global__ void __launch_bounds__(SK_THREADS) k_sketch(const T* __restrict__ X, int64_t ldx, int64_t N, int J,
                                                       const float* __restrict__ om, float* __restrict__ Y,
                                                       const int64_t* __restrict__ d_off, int64_t om_stride) {
  using C = SkCfg<T, LP>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* xs[2] = {smem, smem + C::XS_BYTES};
  float* os[2] = {reinterpret_cast<float*>(smem + 2 * C::XS_BYTES),
                  reinterpret_cast<float*>(smem + 2 * C::XS_BYTES + C::OS_BYTES)};
  const int tid = threadIdx.x;

  // Row range of this block: flat tiling over all slices, or (per-slice Omega)
  // block (bx, k) covers rows of slice k only.
  int64_t row0, rowEnd;
  if (d_off) {
    const int k = blockIdx.y;
    row0 = d_off[k] + (int64_t)blockIdx.x * C::ROWS;
    rowEnd = d_off[k + 1];
    if (row0 >= rowEnd) return;
    om += (int64_t)k * om_stride;
  } else {
    row0 = (int64_t)blockIdx.x * C::ROWS;
    rowEnd = N;
  }
  const int nchunk = (J + C::JC - 1) / C::JC;

  auto load_chunk = [&](int ch, int buf) {
    const int j0 = ch * C::JC;
    // X: ROWS rows x 4 pieces of 16 bytes
#pragma unroll
    for (int i = 0; i < (C::ROWS * 4) / SK_THREADS; ++i) {
      const int p = tid + i * SK_THREADS;
      const int r = p >> 2, part = p & 3;
      const int64_t grow = row0 + r;
      const int jj = j0 + part * C::VN;
      const T* src = X + (grow < rowEnd ? grow : row0) * ldx + (jj < J ? jj : 0);
      const int nbytes = (grow < rowEnd && jj < J) ? 16 : 0;
      cp_async16(xs[buf] + r * SK_PITCH + part * 16, src, nbytes);
    }
    // Omega chunk: JC rows x LP floats, contiguous
    const float* osrc = om + (int64_t)j0 * LP;
    for (int p = tid; p < C::JC * LP / 4; p += SK_THREADS) cp_async16(os[buf] + p * 4, osrc + p * 4, 16);
    cp_async_commit();
  };

  float acc[C::RPT][LP];
#pragma unroll
  for (int r = 0; r < C::RPT; ++r)
#pragma unroll
    for (int c = 0; c < LP; ++c) acc[r][c] = 0.f;

  const int warp = tid >> 5, lane = tid & 31;
  const int rloc0 = warp * 32 * C::RPT + lane;  // my rows: rloc0 + 32 * r

  load_chunk(0, 0);
  for (int ch = 0; ch < nchunk; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunk) {
      load_chunk(ch + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int j0 = ch * C::JC;
    const bool tail = j0 + C::JC > J;
#pragma unroll
    for (int v = 0; v < C::JC / C::VN; ++v) {
      float xv[C::RPT][C::VN];
#pragma unroll
      for (int r = 0; r < C::RPT; ++r) {
        uint4 u = *reinterpret_cast<const uint4*>(xs[buf] + (rloc0 + 32 * r) * SK_PITCH + v * 16);
        Vec16<T>::unpack(u, xv[r]);
        if (tail) {
#pragma unroll
          for (int e = 0; e < C::VN; ++e)
            if (j0 + v * C::VN + e >= J) xv[r][e] = 0.f;
        }
      }
#pragma unroll
      for (int e = 0; e < C::VN; ++e) {
        const float4* orow = reinterpret_cast<const float4*>(os[buf] + (v * C::VN + e) * LP);
#pragma unroll
        for (int c4 = 0; c4 < LP / 4; ++c4) {
          const float4 o = orow[c4];
#pragma unroll
          for (int r = 0; r < C::RPT; ++r) {
            acc[r][4 * c4 + 0] = fmaf(xv[r][e], o.x, acc[r][4 * c4 + 0]);
            acc[r][4 * c4 + 1] = fmaf(xv[r][e], o.y, acc[r][4 * c4 + 1]);
            acc[r][4 * c4 + 2] = fmaf(xv[r][e], o.z, acc[r][4 * c4 + 2]);
            acc[r][4 * c4 + 3] = fmaf(xv[r][e], o.w, acc[r][4 * c4 + 3]);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < C::RPT; ++r) {
    const int64_t grow = row0 + rloc0 + 32 * r;
    if (grow < rowEnd) {
      float4* dst = reinterpret_cast<float4*>(Y + grow * LP);
#pragma unroll
      for (int c4 = 0; c4 < LP / 4; ++c4)
        dst[c4] = make_float4(acc[r][4 * c4], acc[r][4 * c4 + 1], acc[r][4 * c4 + 2], acc[r][4 * c4 + 3]);
    }
  }
}

// -------------------------------------------------------------- projection --
// B1[k] (LP x Jp) = Q_k^T X_k, and partial ||X_k||^2 per (k, column block).
// Block (jb, k); thread owns JPT consecutive columns and all LP outputs.
constexpr int PJ_THREADS = 64;
constexpr int PJ_QROWS = 64;

template <typename T, int JPT>
__device__ inline void load_cols(const T* p, float* f);
template <>
__device__ inline void load_cols<float, 4>(const float* p, float* f) { load4<float>(p, f); }
template <>
__device__ inline void load_cols<__nv_bfloat16, 4>(const __nv_bfloat16* p, float* f) { load4<__nv_bfloat16>(p, f); }
template <>
__device__ inline void load_cols<__half, 4>(const __half* p, float* f) { load4<__half>(p, f); }
template <>
__device__ inline void load_cols<float, 2>(const float* p, float* f) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  f[0] = v.x; f[1] = v.y;
}
template <>
__device__ inline void load_cols<__nv_bfloat16, 2>(const __nv_bfloat16* p, float* f) {
  uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(p));
  f[0] = __uint_as_float(v << 16); f[1] = __uint_as_float(v & 0xffff0000u);
}
template <>
__device__ inline void load_cols<__half, 2>(const __half* p, float* f) {
  uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(p));
  float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v));
  f[0] = a.x; f[1] = a.y;
}

template <typename T, int LP>
__global__ void __launch_bounds__(PJ_THREADS) k_project(const T* __restrict__ X, int64_t ldx,
                                                        const int64_t* __restrict__ d_off, int J, int Jp,
                                                        const float* __restrict__ Q, float* __restrict__ B1,
                                                        double* __restrict__ xpart) {
  constexpr int JPT = LP <= 32 ? 4 : 2;
  __shared__ __align__(16) float qs[PJ_QROWS * LP];
  __shared__ double red[PJ_THREADS / 32];
  const int k = blockIdx.y, tid = threadIdx.x;
  const int j0 = (blockIdx.x * PJ_THREADS + tid) * JPT;
  const bool jv = j0 < J;
  const int64_t r0 = d_off[k], r1 = d_off[k + 1];
  float acc[JPT][LP];
#pragma unroll
  for (int a = 0; a < JPT; ++a)
#pragma unroll
    for (int c = 0; c < LP; ++c) acc[a][c] = 0.f;
  // ||X_k||^2 of this thread's columns: one FP32 accumulator per column over
  // a row chunk (at most PJ_QROWS squares each), chunks added in FP64
  float nrm[JPT];
  double nrd = 0.0;
  const T* xcol = X + (jv ? j0 : 0);

  for (int64_t rs = r0; rs < r1; rs += PJ_QROWS) {
#pragma unroll
    for (int a = 0; a < JPT; ++a) nrm[a] = 0.f;
    const int nr = (int)min64(PJ_QROWS, r1 - rs);
    __syncthreads();
    for (int p = tid; p < nr * LP / 4; p += PJ_THREADS)
      reinterpret_cast<float4*>(qs)[p] = __ldg(reinterpret_cast<const float4*>(Q + rs * LP) + p);
    __syncthreads();
    int i = 0;
    for (; i + 4 <= nr; i += 4) {
      float x[4][JPT];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (jv) {
          load_cols<T, JPT>(xcol + (rs + i + u) * ldx, x[u]);
        } else {
#pragma unroll
          for (int a = 0; a < JPT; ++a) x[u][a] = 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int a = 0; a < JPT; ++a) {
          if (j0 + a >= J) x[u][a] = 0.f;
          nrm[a] = fmaf(x[u][a], x[u][a], nrm[a]);
        }
        const float4* qrow = reinterpret_cast<const float4*>(qs + (i + u) * LP);
#pragma unroll
        for (int c4 = 0; c4 < LP / 4; ++c4) {
          const float4 q = qrow[c4];
#pragma unroll
          for (int a = 0; a < JPT; ++a) {
            acc[a][4 * c4 + 0] = fmaf(x[u][a], q.x, acc[a][4 * c4 + 0]);
            acc[a][4 * c4 + 1] = fmaf(x[u][a], q.y, acc[a][4 * c4 + 1]);
            acc[a][4 * c4 + 2] = fmaf(x[u][a], q.z, acc[a][4 * c4 + 2]);
            acc[a][4 * c4 + 3] = fmaf(x[u][a], q.w, acc[a][4 * c4 + 3]);
          }
        }
      }
    }
    for (; i < nr; ++i) {
      float x[JPT];
      if (jv) {
        load_cols<T, JPT>(xcol + (rs + i) * ldx, x);
      } else {
#pragma unroll
        for (int a = 0; a < JPT; ++a) x[a] = 0.f;
      }
#pragma unroll
      for (int a = 0; a < JPT; ++a) {
        if (j0 + a >= J) x[a] = 0.f;
        nrm[a] = fmaf(x[a], x[a], nrm[a]);
      }
      const float4* qrow = reinterpret_cast<const float4*>(qs + i * LP);
#pragma unroll
      for (int c4 = 0; c4 < LP / 4; ++c4) {
        const float4 q = qrow[c4];
#pragma unroll
        for (int a = 0; a < JPT; ++a) {
          acc[a][4 * c4 + 0] = fmaf(x[a], q.x, acc[a][4 * c4 + 0]);
          acc[a][4 * c4 + 1] = fmaf(x[a], q.y, acc[a][4 * c4 + 1]);
          acc[a][4 * c4 + 2] = fmaf(x[a], q.z, acc[a][4 * c4 + 2]);
          acc[a][4 * c4 + 3] = fmaf(x[a], q.w, acc[a][4 * c4 + 3]);
        }
      }
    }
    float cs = 0.f;
#pragma unroll
    for (int a = 0; a < JPT; ++a) cs += nrm[a];
    nrd += (double)cs;
  }
  if (j0 < Jp) {
    float* dst = B1 + (int64_t)k * LP * Jp + j0;
#pragma unroll
    for (int c = 0; c < LP; ++c) {
      if (JPT == 4) *reinterpret_cast<float4*>(dst + (int64_t)c * Jp) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
      else *reinterpret_cast<float2*>(dst + (int64_t)c * Jp) = make_float2(acc[0][c], acc[JPT > 1 ? 1 : 0][c]);
    }
  }
  if (xpart) {
    nrd = warp_sum(nrd);
    if ((tid & 31) == 0) red[tid >> 5] = nrd;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < PJ_THREADS / 32; ++w) s += red[w];
      xpart[(int64_t)k * gridDim.x + blockIdx.x] = s;
    }
  }
}

// --------------------------------------------------------------- dispatch --
template <typename T, int LP>
static void sketch_t(const void* X, int64_t ldx, int64_t N, int J, const float* om, float* Y,
                     const int64_t* d_off, int K, int maxI, int64_t om_stride, cudaStream_t s) {
  using C = SkCfg<T, LP>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sketch<T, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    attr = true;
  }
  dim3 grid;
  if (d_off) grid = dim3((unsigned)((maxI + C::ROWS - 1) / C::ROWS), (unsigned)K);
  else grid = dim3((unsigned)((N + C::ROWS - 1) / C::ROWS));
  if (grid.x == 0) return;
  DP2_COUNTED(k_sketch<T, LP><<<grid, SK_THREADS, C::SMEM, s>>>(reinterpret_cast<const T*>(X), ldx, N, J, om, Y, d_off,
                                                    om_stride));
}

template <int LP>
static void sketch_lp(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const float* om, float* Y,
                      const int64_t* d_off, int K, int maxI, int64_t om_stride, cudaStream_t s) {
  if (dt == DPAR2_F32) sketch_t<float, LP>(X, ldx, N, J, om, Y, d_off, K, maxI, om_stride, s);
  else if (dt == DPAR2_BF16) sketch_t<__nv_bfloat16, LP>(X, ldx, N, J, om, Y, d_off, K, maxI, om_stride, s);
  else sketch_t<__half, LP>(X, ldx, N, J, om, Y, d_off, K, maxI, om_stride, s);
}

void launch_sketch_generic(const void* X, dpar2_dtype dt, int64_t ldx, int64_t N, int J, const float* om_pad,
                           int LP, float* Y, cudaStream_t s) {
  DP2_LP_SWITCH(LP, (sketch_lp<L>(X, dt, ldx, N, J, om_pad, Y, nullptr, 0, 0, 0, s)));
}

void launch_sketch_generic_per_slice(const void* X, dpar2_dtype dt, int64_t ldx, const int64_t* d_off, int K,
                                     int maxI, int J, const float* om_k, int Jpad, int LP, float* Y,
                                     cudaStream_t s) {
  DP2_LP_SWITCH(LP, (sketch_lp<L>(X, dt, ldx, 0, J, om_k, Y, d_off, K, maxI, (int64_t)Jpad * LP, s)));
}

template <typename T, int LP>
static void project_t(const void* X, int64_t ldx, const int64_t* d_off, int K, int J, int Jp, const float* Q,
                      float* B1, double* xpart, int* nJb_out, cudaStream_t s) {
  constexpr int JPT = LP <= 32 ? 4 : 2;
  const int nJb = (Jp + PJ_THREADS * JPT - 1) / (PJ_THREADS * JPT);
  if (nJb_out) *nJb_out = nJb;
  DP2_COUNTED(k_project<T, LP><<<dim3(nJb, K), PJ_THREADS, 0, s>>>(reinterpret_cast<const T*>(X), ldx, d_off, J, Jp, Q, B1,
                                                       xpart));
}

void launch_project_generic(const void* X, dpar2_dtype dt, int64_t ldx, const int64_t* d_off, int K, int J,
                            int Jp, const float* Q, int LP, float* B1, double* xpart, int* nJb_out,
                            cudaStream_t s) {
  if (dt == DPAR2_F32) {
    DP2_LP_SWITCH(LP, (project_t<float, L>(X, ldx, d_off, K, J, Jp, Q, B1, xpart, nJb_out, s)));
  } else if (dt == DPAR2_BF16) {
    DP2_LP_SWITCH(LP, (project_t<__nv_bfloat16, L>(X, ldx, d_off, K, J, Jp, Q, B1, xpart, nJb_out, s)));
  } else {
    DP2_LP_SWITCH(LP, (project_t<__half, L>(X, ldx, d_off, K, J, Jp, Q, B1, xpart, nJb_out, s)));
  }
}

int project_blocks(int Jp, int LP) {
  const int JPT = LP <= 32 ? 4 : 2;
  return (Jp + PJ_THREADS * JPT - 1) / (PJ_THREADS * JPT);
}

}  // namespace dp2
