// Learned sketch: the range-finder loss of a trainable test matrix Omega
// (J x l) and its gradient.  Alg. 1 replaces X_k by Q_k Q_k^T X_k with Q_k an
// orthonormal basis of Y_k = X_k Omega; what it leaves out of slice k is
//   f_k(Omega) = ||X_k - Y_k Y_k^+ X_k||_F^2 = ||X_k||^2 - tr(G_k^-1 Y_k^T X_k X_k^T Y_k),
// G_k = Y_k^T Y_k, and the loss is L = (1/K) sum_k f_k / ||X_k||^2.
//
// The forward pass reuses the stage-1 passes: Y = X Omega, CholeskyQR2
// (Q1_k = Y_k M1_k, Q_k = Q1_k M2_k, M1 = R1^-1, M2 = R2^-1), B1_k = Q1_k^T X_k
// with ||X_k||^2, GB_k = B1_k B1_k^T, so that ||Q_k^T X_k||^2 = tr(M2^T GB M2).
//
// Gradient.  With Y = Q R (R^-1 = M1 M2), B = Q^T X and A = X X^T, the
// derivative of tr(G^-1 Y^T A Y) with respect to Y is 2 (A Y G^-1 - Y G^-1 N G^-1),
// N = Y^T A Y.  Both terms simplify through Y = Q R:
//   X^T Y G^-1 = B^T R^-T =: Mk (J x l),   Y G^-1 N G^-1 = Q B Mk,
// so  df_k/dOmega = -2 X_k^T (X_k Mk - Q_k B_k Mk) = -2 X_k^T (I - Q_k Q_k^T) X_k Mk.
// In stored quantities: Mk = B1^T P with P = M2 M2^T M1^T, and
// Q B Mk = Q1 S with S = M2 M2^T GB P.  The backward pass therefore runs
//   pass 3  V_k = X_k B1_k^T                  (per-slice right operand)
//   W_k = c_k (V_k P_k - Q1_k S_k),  c_k = -2 dL / (K ||X_k||^2)   (V_k P_k = X_k Mk)
// (P_k and S_k are formed by the forward pass).
//   pass 4  dL/dOmega^T = sum_k W_k^T X_k      (one reduction over all rows)
// which are two more streams of X: four per training step.
#include "common.cuh"
#include "internal.h"

namespace dp2 {

// --------------------------------------------------- per-slice small work --
// One block per slice, FP32 l x l products in shared memory (rows padded to
// LP + 1 floats: conflict-free column walks):
//   N2 = M2 M2^T,  ||Q_k^T X_k||^2 = sum_ab GB_ab N2_ab (FP64 sum),
//   ratio_k = (||X_k||^2 - ||Q_k^T X_k||^2) / ||X_k||^2,
//   P_k = N2 M1^T,  S_k = N2 GB P_k  (what the backward pass needs),
// all zero outside l x l.
template <int LP>
__global__ void __launch_bounds__(256) k_sl_small(const float* __restrict__ M1, const float* __restrict__ M2,
                                                  const double* __restrict__ GB, const double* __restrict__ xn,
                                                  int ell, double* __restrict__ ratio, float* __restrict__ Pout,
                                                  float* __restrict__ Sout) {
  constexpr int LQ = LP + 1, LL = LP * LP;
  extern __shared__ float sm[];
  float* m1 = sm;
  float* m2 = m1 + LP * LQ;
  float* gb = m2 + LP * LQ;
  float* n2 = gb + LP * LQ;
  float* pp = n2 + LP * LQ;
  float* tt = pp + LP * LQ;
  __shared__ double red[8];
  const int k = blockIdx.x;
  const double* g = GB + (int64_t)k * LL;
  for (int e = threadIdx.x; e < LL; e += blockDim.x) {
    const int a = e / LP, c = e - a * LP;
    const bool in = a < ell && c < ell;
    m1[a * LQ + c] = in ? M1[(int64_t)k * LL + e] : 0.f;
    m2[a * LQ + c] = in ? M2[(int64_t)k * LL + e] : 0.f;
    gb[a * LQ + c] = in ? (float)g[e] : 0.f;
  }
  __syncthreads();
  double q = 0.0;
  for (int e = threadIdx.x; e < LL; e += blockDim.x) {  // N2 = M2 M2^T and sum GB o N2
    const int a = e / LP, b = e - a * LP;
    float t = 0.f;
    for (int c = 0; c < ell; ++c) t = fmaf(m2[a * LQ + c], m2[b * LQ + c], t);
    n2[a * LQ + b] = t;
    if (a < ell && b < ell) q = fma(g[e], (double)t, q);
  }
  q = warp_sum(q);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const double x = xn[k];
    ratio[k] = x > 0.0 ? (x - t) / x : 0.0;
  }
  for (int e = threadIdx.x; e < LL; e += blockDim.x) {  // P = N2 M1^T
    const int a = e / LP, c = e - a * LP;
    float t = 0.f;
    for (int b = 0; b < ell; ++b) t = fmaf(n2[a * LQ + b], m1[c * LQ + b], t);
    pp[a * LQ + c] = t;
    Pout[(int64_t)k * LL + e] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < LL; e += blockDim.x) {  // T = GB P
    const int a = e / LP, c = e - a * LP;
    float t = 0.f;
    for (int b = 0; b < ell; ++b) t = fmaf(gb[a * LQ + b], pp[b * LQ + c], t);
    tt[a * LQ + c] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < LL; e += blockDim.x) {  // S = N2 T
    const int a = e / LP, c = e - a * LP;
    float t = 0.f;
    for (int b = 0; b < ell; ++b) t = fmaf(n2[a * LQ + b], tt[b * LQ + c], t);
    Sout[(int64_t)k * LL + e] = t;
  }
}

// loss = (1/K) sum_k ratio_k, summed in a fixed order by one block.
__global__ void k_sl_total(const double* __restrict__ ratio, int K, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < K; i += 256) s += ratio[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / (double)K;
}

// power of two that brings m (> 0, finite) into [0.5, 1); 1 otherwise
__device__ __forceinline__ float range_scale(float m) {
  return (m > 0.f && m < 3.0e38f) ? ldexpf(1.f, -(ilogbf(m) + 1)) : 1.f;
}

// three 16-bit parts whose sum is v up to FP32 rounding
template <typename H>
__device__ __forceinline__ void split3(float v, H* o0, H* o1, H* o2);
template <>
__device__ __forceinline__ void split3<__nv_bfloat16>(float v, __nv_bfloat16* o0, __nv_bfloat16* o1,
                                                      __nv_bfloat16* o2) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  *o0 = h;
  *o1 = m;
  *o2 = __float2bfloat16_rn(r1 - __bfloat162float(m));
}
template <>
__device__ __forceinline__ void split3<__half>(float v, __half* o0, __half* o1, __half* o2) {
  const __half h = __float2half_rn(v);
  const float r1 = v - __half2float(h);
  const __half m = __float2half_rn(r1);
  *o0 = h;
  *o1 = m;
  *o2 = __float2half_rn(r1 - __half2float(m));
}

// ------------------------------------------------------ pass-3 operand --
// The right operand of U_k = X_k B1_k^T: row i of B1_k (over j), times r(k, i),
// the power of two that brings max_j |B1_k(i, j)| into [0.5, 1) (rows of B1
// scale with the sketch's singular values; FP16 parts of a small row would
// otherwise sit in the subnormal range).  r is written for the caller to
// divide out (column i of U carries it).  TC: three 16-bit parts stored
// [k][3 LPN][Jpad] (row t LPN + i holds part t of B1 row i); otherwise FP32
// [k][Jpad][LP].  One warp per row of B1, reading it twice (max, then split).
template <typename H>
__device__ __forceinline__ uint2 split4(float4 v, uint2* mid, uint2* lo) {
  H h[4], m[4], l[4];
  split3<H>(v.x, &h[0], &m[0], &l[0]);
  split3<H>(v.y, &h[1], &m[1], &l[1]);
  split3<H>(v.z, &h[2], &m[2], &l[2]);
  split3<H>(v.w, &h[3], &m[3], &l[3]);
  uint2 a, b, c;
  memcpy(&a, h, 8);
  memcpy(&b, m, 8);
  memcpy(&c, l, 8);
  *mid = b;
  *lo = c;
  return a;
}

template <typename H>
__global__ void __launch_bounds__(256) k_sl_rowsplit(const float* __restrict__ B1, int K, int Jp, int J, int Jpad,
                                                     int ell, int LP, int LPN, H* __restrict__ out16,
                                                     float* __restrict__ out32, float* __restrict__ rscale) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int rows = out16 ? LPN : LP;
  if (gw >= (int64_t)K * rows) return;
  const int k = (int)(gw / rows), i = (int)(gw % rows);
  const float* b = B1 + ((int64_t)k * LP + i) * Jp;
  const bool live = i < ell;
  // four columns per lane: B1 rows (pitch Jp, a multiple of 4) and the 16-bit
  // rows (pitch Jpad, a multiple of 32) are 16- and 8-byte aligned
  auto load4 = [&](int j) -> float4 {
    if (!live || j >= J) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (j + 3 < J) return *reinterpret_cast<const float4*>(b + j);
    return make_float4(b[j], j + 1 < J ? b[j + 1] : 0.f, j + 2 < J ? b[j + 2] : 0.f, 0.f);
  };
  float mx = 0.f;
  for (int j = 4 * lane; j < J; j += 128) {
    const float4 v = load4(j);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float r = range_scale(mx);
  if (i < LP && lane == 0) rscale[(int64_t)k * LP + i] = r;
  if (out16) {
    H* o = out16 + (int64_t)k * 3 * LPN * Jpad;
    for (int j = 4 * lane; j < Jpad; j += 128) {
      float4 v = load4(j);
      v.x *= r;
      v.y *= r;
      v.z *= r;
      v.w *= r;
      uint2 mid, lo;
      const uint2 hi = split4<H>(v, &mid, &lo);
      *reinterpret_cast<uint2*>(o + (int64_t)i * Jpad + j) = hi;
      *reinterpret_cast<uint2*>(o + (int64_t)(LPN + i) * Jpad + j) = mid;
      *reinterpret_cast<uint2*>(o + (int64_t)(2 * LPN + i) * Jpad + j) = lo;
    }
  } else {
    for (int j = lane; j < Jpad; j += 32) out32[((int64_t)k * Jpad + j) * LP + i] = (live && j < J) ? b[j] * r : 0.f;
  }
}

// ----------------------------------------------------------- W rows ----
// W_k = c_k (V_k diag(r_k)^-1 P_k - Q1_k S_k) row by row, V_k = X_k B1_k^T diag(r_k)
// from pass 3 (so V_k diag(r_k)^-1 P_k = X_k Mk), c_k = -2 g / (K ||X_k||^2); FP32
// rows N x LP, and each block's largest |W| of every column into
// bmax[block][c] (k_sl_colmax reduces them).  P and S are read from shared
// memory four columns at a time.  Grid (ceil(maxI / 128), K).
template <int LP>
__global__ void __launch_bounds__(128) k_sl_wrows(const float* __restrict__ U, const float* __restrict__ Q1,
                                                  const int64_t* __restrict__ off, const float* __restrict__ P,
                                                  const float* __restrict__ S, const double* __restrict__ xn,
                                                  double gscale, int K, const float* __restrict__ rs,
                                                  float* __restrict__ W, float* __restrict__ bmax) {
  __shared__ __align__(16) float ps[LP * LP];
  __shared__ __align__(16) float ss[LP * LP];
  __shared__ float inv[LP];
  __shared__ float red[4][LP];
  const int k = blockIdx.y;
  for (int e = threadIdx.x; e < LP * LP; e += 128) {
    ps[e] = P[(int64_t)k * LP * LP + e];
    ss[e] = S[(int64_t)k * LP * LP + e];
  }
  if (threadIdx.x < LP) inv[threadIdx.x] = 1.f / rs[(int64_t)k * LP + threadIdx.x];  // exact: powers of two
  __syncthreads();
  const int64_t row = off[k] + (int64_t)blockIdx.x * 128 + threadIdx.x;
  const bool live = row < off[k + 1];
  const double x = xn[k];
  const float c = x > 0.0 ? (float)(-2.0 * gscale / ((double)K * x)) : 0.f;
  float w[LP];
#pragma unroll
  for (int cc = 0; cc < LP; ++cc) w[cc] = 0.f;
  if (live) {
    float v[LP], q[LP];
    const float4* u4 = reinterpret_cast<const float4*>(U + row * LP);
    const float4* q4 = reinterpret_cast<const float4*>(Q1 + row * LP);
#pragma unroll
    for (int i = 0; i < LP / 4; ++i) {
      const float4 a = u4[i], b = q4[i];
      v[4 * i] = a.x * inv[4 * i];
      v[4 * i + 1] = a.y * inv[4 * i + 1];
      v[4 * i + 2] = a.z * inv[4 * i + 2];
      v[4 * i + 3] = a.w * inv[4 * i + 3];
      q[4 * i] = b.x;
      q[4 * i + 1] = b.y;
      q[4 * i + 2] = b.z;
      q[4 * i + 3] = b.w;
    }
    const float4* p4 = reinterpret_cast<const float4*>(ps);
    const float4* s4 = reinterpret_cast<const float4*>(ss);
#pragma unroll
    for (int i = 0; i < LP; ++i) {
#pragma unroll
      for (int c4 = 0; c4 < LP / 4; ++c4) {
        const float4 pv = p4[i * (LP / 4) + c4], sv = s4[i * (LP / 4) + c4];
        w[4 * c4] = fmaf(v[i], pv.x, fmaf(-q[i], sv.x, w[4 * c4]));
        w[4 * c4 + 1] = fmaf(v[i], pv.y, fmaf(-q[i], sv.y, w[4 * c4 + 1]));
        w[4 * c4 + 2] = fmaf(v[i], pv.z, fmaf(-q[i], sv.z, w[4 * c4 + 2]));
        w[4 * c4 + 3] = fmaf(v[i], pv.w, fmaf(-q[i], sv.w, w[4 * c4 + 3]));
      }
    }
#pragma unroll
    for (int cc = 0; cc < LP; ++cc) w[cc] *= c;
    float4* o = reinterpret_cast<float4*>(W + row * LP);
#pragma unroll
    for (int c4 = 0; c4 < LP / 4; ++c4) o[c4] = make_float4(w[4 * c4], w[4 * c4 + 1], w[4 * c4 + 2], w[4 * c4 + 3]);
  }
#pragma unroll
  for (int cc = 0; cc < LP; ++cc) {
    float m = fabsf(w[cc]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][cc] = m;
  }
  __syncthreads();
  if (threadIdx.x < LP) {
    const float m = fmaxf(fmaxf(red[0][threadIdx.x], red[1][threadIdx.x]), fmaxf(red[2][threadIdx.x], red[3][threadIdx.x]));
    bmax[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * LP + threadIdx.x] = m;
  }
}

// wmax[c] = max over the nb block maxima of column c (FP32 bit pattern of a
// non-negative float: atomicMax on it is order-independent).  Each block
// reduces a strided share of the rows, then one atomic per column.
__global__ void k_sl_colmax(const float* __restrict__ bmax, int64_t nb, int LP, unsigned* __restrict__ wmax) {
  __shared__ float red[1024];
  const int c = threadIdx.x % LP, lanes = blockDim.x / LP;
  float m = 0.f;
  if (threadIdx.x < lanes * LP)
    for (int64_t b = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x / LP); b < nb; b += (int64_t)gridDim.x * lanes)
      m = fmaxf(m, bmax[b * LP + c]);
  red[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x < LP) {
    float t = 0.f;
    for (int i = 0; i < lanes; ++i) t = fmaxf(t, red[i * LP + threadIdx.x]);
    if (t > 0.f && t < 3.0e38f) atomicMax(wmax + threadIdx.x, __float_as_uint(t));
  }
}

// W (N x LP FP32), column c scaled by range_scale(wmax[c]) -> three 16-bit
// parts in the 64-row chunked layout of the projection's right operand over
// row ranges that start on multiples of 64: element (p, c) of part t at
// ((p / 64) 3 LPN + t LPN + c) 64 + p % 64, p the global row, except that the
// final chunk holds rows N - 64 .. N - 1 (the projection aligns a range's last
// chunk to its end; the caller zeroes that chunk first).
template <typename H>
__global__ void k_sl_wsplit(const float* __restrict__ W, int64_t N, int LP, int LPN, const unsigned* __restrict__ wmax,
                            H* __restrict__ out16) {
  __shared__ float sc[kMaxEll];
  for (int c = threadIdx.x; c < LP; c += blockDim.x) sc[c] = range_scale(__uint_as_float(wmax[c]));
  __syncthreads();
  const int64_t last = (N + 63) / 64 - 1;  // chunk of rows N - 64 .. N - 1
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < N; row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t chunk = row >= 64 * last ? last : row / 64;
    const int64_t b = row >= 64 * last ? row - (N - 64) : row % 64;
    H* o = out16 + chunk * 3 * LPN * 64 + b;
    for (int c = 0; c < LPN; ++c) {
      const float v = c < LP ? W[row * LP + c] * sc[c] : 0.f;
      split3<H>(v, o + (int64_t)c * 64, o + (int64_t)(LPN + c) * 64, o + (int64_t)(2 * LPN + c) * 64);
    }
  }
}

// ---------------------------------------------------------- gradient ----
// grad(j, c) = sum_p part_p(c, j) over the np row ranges of the last pass, in
// order, with the column scale of the split W divided out (wmax null: none);
// part is np x LP x Jp (the projection's output layout).
__global__ void k_sl_gradsum(const float* __restrict__ part, int np, int LP, int Jp, int J, int ell,
                             const unsigned* __restrict__ wmax, float* __restrict__ grad) {
  const int64_t n = (int64_t)J * ell;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / J), j = (int)(i % J);
    const float inv = wmax ? 1.f / range_scale(__uint_as_float(wmax[c])) : 1.f;  // exact (power of two)
    float s = 0.f;
    for (int p = 0; p < np; ++p) s += part[((int64_t)p * LP + c) * Jp + j];
    grad[(int64_t)j * ell + c] = s * inv;
  }
}

// ---------------------------------------------------------------- host --
template <int LP>
static void sl_small_lp(const float* M1, const float* M2, const double* GB, const double* xn, int K, int ell,
                        double* ratio, float* P, float* S, cudaStream_t s) {
  const size_t sm = (size_t)6 * LP * (LP + 1) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sl_small<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  DP2_COUNTED(k_sl_small<LP><<<K, 256, sm, s>>>(M1, M2, GB, xn, ell, ratio, P, S));
}

void launch_sl_loss(const float* M1, const float* M2, const double* GB, const double* xn, int K, int ell, int LP,
                    double* ratio, float* P, float* S, double* out, cudaStream_t s) {
  DP2_LP_SWITCH(LP, (sl_small_lp<L>(M1, M2, GB, xn, K, ell, ratio, P, S, s)));
  DP2_COUNTED(k_sl_total<<<1, 256, 0, s>>>(ratio, K, out));
}

void launch_sl_rowsplit(const float* B1, int K, int Jp, int J, int Jpad, int ell, int LP, int LPN, dpar2_dtype dt,
                        void* out16, float* out32, float* rscale, cudaStream_t s) {
  const int64_t warps = (int64_t)K * (out16 ? LPN : LP);
  const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
  if (out16 && dt == DPAR2_F16)
    DP2_COUNTED(k_sl_rowsplit<__half><<<grid, 256, 0, s>>>(B1, K, Jp, J, Jpad, ell, LP, LPN, static_cast<__half*>(out16), out32,
                                               rscale));
  else
    DP2_COUNTED(k_sl_rowsplit<__nv_bfloat16><<<grid, 256, 0, s>>>(B1, K, Jp, J, Jpad, ell, LP, LPN,
                                                      static_cast<__nv_bfloat16*>(out16), out32, rscale));
}

template <int LP>
static void sl_wrows_lp(const float* U, const float* Q1, const int64_t* d_off, int K, int64_t maxI, const float* P,
                        const float* S, const double* xn, double gscale, const float* rs, float* W, float* bmax,
                        cudaStream_t s) {
  dim3 grid((unsigned)std::max<int64_t>(1, (maxI + 127) / 128), (unsigned)K);
  DP2_COUNTED(k_sl_wrows<LP><<<grid, 128, 0, s>>>(U, Q1, d_off, P, S, xn, gscale, K, rs, W, bmax));
}

int64_t sl_wrows_blocks(int K, int64_t maxI) { return std::max<int64_t>(1, (maxI + 127) / 128) * K; }

void launch_sl_wrows(const float* U, const float* Q1, const int64_t* d_off, int K, int64_t maxI, int LP,
                     const float* P, const float* S, const double* xn, double gscale, const float* rs, float* W,
                     float* bmax, unsigned* wmax, cudaStream_t s) {
  DP2_LP_SWITCH(LP, (sl_wrows_lp<L>(U, Q1, d_off, K, maxI, P, S, xn, gscale, rs, W, bmax, s)));
  cudaMemsetAsync(wmax, 0, (size_t)LP * sizeof(unsigned), s);
  DP2_COUNTED(k_sl_colmax<<<64, (1024 / LP) * LP, 0, s>>>(bmax, sl_wrows_blocks(K, maxI), LP, wmax));
}

void launch_sl_wsplit(const float* W, int64_t N, int LP, int LPN, const unsigned* wmax, dpar2_dtype dt, void* out16,
                      cudaStream_t s) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 8192));
  if (dt == DPAR2_F16) DP2_COUNTED(k_sl_wsplit<__half><<<grid, 256, 0, s>>>(W, N, LP, LPN, wmax, static_cast<__half*>(out16)));
  else DP2_COUNTED(k_sl_wsplit<__nv_bfloat16><<<grid, 256, 0, s>>>(W, N, LP, LPN, wmax, static_cast<__nv_bfloat16*>(out16)));
}

void launch_sl_gradsum(const float* part, int np, int LP, int Jp, int J, int ell, const unsigned* wmax, float* grad,
                       cudaStream_t s) {
  const int64_t n = (int64_t)J * ell;
  DP2_COUNTED(k_sl_gradsum<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(part, np, LP, Jp, J, ell, wmax,
                                                                                   grad));
}

}  // namespace dp2
