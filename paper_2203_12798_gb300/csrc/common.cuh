// Device helpers shared by the DPar2 kernels (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dpar2.h"

namespace dp2 {

// Bits of the device status word (one int per context).
enum : int {
  ST_NONFINITE = 1,   // a NaN/Inf met in a Gram, loss or solve
  ST_TIMEOUT = 2,     // a bounded wait gave up
  ST_RANK_DROP = 4,   // a CholeskyQR step dropped a dependent column (information)
  ST_SWEEP_CAP = 8,   // a Jacobi solver hit its sweep cap (information)
  ST_PINV = 16,       // a Gram-Hadamard solve fell back to the pseudoinverse (information)
  ST_FATAL_MASK = ST_NONFINITE | ST_TIMEOUT,
};

constexpr int kMaxEll = 64;   // sketch width l = R + p
constexpr int kMaxR = 64;     // target rank

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t round_up64(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Error-free product a*b = p + e (FMA-based TwoProduct, Ogita-Rump-Oishi 2005)
// accumulated into a double-float (hi, lo) pair with Knuth's TwoSum.
struct DF {
  float hi, lo;
};
__device__ inline void df_mac(DF& s, float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  float t = s.hi + p;
  float bp = t - s.hi;
  float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}
__device__ inline double df_value(const DF& s) { return (double)s.hi + (double)s.lo; }

// Packed pairs of FP32 values in one 64-bit register and the f32x2
// arithmetic of the sm_100 family (each half rounded as the scalar op),
// used for two independent double-float accumulations per instruction.
__device__ __forceinline__ uint64_t f2pack(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 f2unpack(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t add_f2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub_f2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul_f2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma_f2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Two double-float accumulators (hi, lo pairs); df_mac2 is df_mac on both
// halves: s += a b with a the packed multiplier and na = -a.
struct DF2 {
  uint64_t hi, lo;
};
__device__ __forceinline__ void df_mac2(DF2& s, uint64_t a, uint64_t na, uint64_t b) {
  const uint64_t p = mul_f2(a, b);
  const uint64_t ne = fma_f2(na, b, p);  // p - a b exactly: minus the rounding error of p
  const uint64_t t = add_f2(s.hi, p);
  const uint64_t bp = sub_f2(t, s.hi);
  const uint64_t err = add_f2(sub_f2(s.hi, sub_f2(t, bp)), sub_f2(p, bp));
  s.hi = t;
  s.lo = add_f2(s.lo, sub_f2(err, ne));
}
// Double-float a + b (TwoSum of the high parts, low parts added, renormalised).
__device__ inline DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);
  e += a.lo + b.lo;
  DF r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}

// ------------------------------------------- warp-parallel small Cholesky ----
// FP64 arithmetic runs at a small fraction of the FP32 rate on this part, so
// the small factorisations below avoid divisions and square roots (one
// reciprocal square root per pivot) and spread every elimination step over
// the 32 lanes of a warp.

// 1/sqrt(d) for d > 0.  Float: the hardware estimate.  Double: the float
// estimate refined by one Newton step for the reciprocal square root,
// y <- y + y (1 - d y^2) / 2, which turns a relative error e into about
// 1.5 e^2 (about 1e-14 here); outside the float range, 1 / sqrt(d) in double.
__device__ inline float rsqrt_nr(float d) { return rsqrtf(d); }
__device__ inline double rsqrt_nr(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  const double y = (double)rsqrtf((float)d);
  const double r = fma(-(d * y), y, 1.0);
  return fma(0.5 * y, r, y);
}

// Upper-triangle index table of an n x n matrix (n <= 255), row-major: entry
// tri_start(c, n) + (e - c) holds (c << 8) | e for c <= e < n.
__host__ __device__ inline int tri_start(int c, int n) { return c * n - c * (c - 1) / 2; }
__device__ inline void warp_pair_table(unsigned short* pairs, int n) {
  const int lane = threadIdx.x & 31;
  for (int c = lane; c < n; c += 32) {
    const int b = tri_start(c, n);
    for (int e = c; e < n; ++e) pairs[b + e - c] = (unsigned short)((c << 8) | e);
  }
  __syncwarp();
}

// Right-looking Cholesky A = R^T R by one warp.  A (n x n, row-major): the
// upper triangle is read and overwritten by R.  The pivot d_j (A_jj after the
// updates of steps < j) is kept when d_j > thr; otherwise (or for every pivot
// when drop_all) row j of R is zero.  rinv[j] = 1 / R_jj, 0 for a dropped
// pivot.  Returns the number of dropped pivots (the same in every lane).
template <typename T>
__device__ int warp_chol_upper(T* A, int n, T thr, bool drop_all, T* rinv, const unsigned short* pairs) {
  const int lane = threadIdx.x & 31;
  const int P = n * (n + 1) / 2;
  int nd = 0;
  for (int j = 0; j < n; ++j) {
    const T d = A[j * n + j];
    const bool drop = drop_all || !(d > thr);
    const T y = drop ? T(0) : rsqrt_nr(d);
    nd += drop;
    for (int c = j + 1 + lane; c < n; c += 32) A[j * n + c] *= y;
    __syncwarp();
    if (lane == 0) {
      A[j * n + j] = drop ? T(0) : d * y;
      rinv[j] = y;
    }
    for (int t = tri_start(j + 1, n) + lane; t < P; t += 32) {
      const int c = pairs[t] >> 8, e = pairs[t] & 255;
      A[c * n + e] -= A[j * n + c] * A[j * n + e];
    }
    __syncwarp();
  }
  return nd;
}

// Mi = R^{-1} for the upper-triangular R of warp_chol_upper (rinv = its
// reciprocal diagonal, 0 at dropped pivots) by back substitution: row m of
// Mi is finished from the bottom up and its contribution pushed to the rows
// above it.  Mi (n x n) must be zero on entry; rows and columns of dropped
// pivots stay zero.
template <typename T>
__device__ void warp_tri_inv(const T* Rm, int n, const T* rinv, T* Mi) {
  const int lane = threadIdx.x & 31;
  for (int m = n - 1; m >= 0; --m) {
    const T ym = rinv[m];
    for (int c = m + lane; c < n; c += 32) Mi[m * n + c] = ((c == m ? T(1) : T(0)) - Mi[m * n + c]) * ym;
    __syncwarp();
    const int w = n - m;
    for (int t = lane; t < m * w; t += 32) {
      const int i = t / w, c = m + (t - i * w);
      Mi[i * n + c] = fma(Rm[i * n + m], Mi[m * n + c], Mi[i * n + c]);
    }
    __syncwarp();
  }
}

// 16-bit element conversions.
template <typename T>
__device__ inline float to_f(T v);
template <>
__device__ inline float to_f<float>(float v) { return v; }
template <>
__device__ inline float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ inline float to_f<__half>(__half v) { return __half2float(v); }

// Unpack a 16-byte vector into floats.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int N = 4;
  __device__ static inline void unpack(const uint4& u, float* f) {
    f[0] = __uint_as_float(u.x);
    f[1] = __uint_as_float(u.y);
    f[2] = __uint_as_float(u.z);
    f[3] = __uint_as_float(u.w);
  }
};
template <>
struct Vec16<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static inline void unpack(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};
template <>
struct Vec16<__half> {
  static constexpr int N = 8;
  __device__ static inline void unpack(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
      float2 v = __half22float2(h);
      f[2 * i] = v.x;
      f[2 * i + 1] = v.y;
    }
  }
};

// 4 consecutive elements -> floats (8- or 16-byte load).
template <typename T>
__device__ inline void load4(const T* p, float* f);
template <>
__device__ inline void load4<float>(const float* p, float* f) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
}
template <>
__device__ inline void load4<__nv_bfloat16>(const __nv_bfloat16* p, float* f) {
  uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  f[0] = __uint_as_float(v.x << 16); f[1] = __uint_as_float(v.x & 0xffff0000u);
  f[2] = __uint_as_float(v.y << 16); f[3] = __uint_as_float(v.y & 0xffff0000u);
}
template <>
__device__ inline void load4<__half>(const __half* p, float* f) {
  uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
}

// Two FP32 fused multiply-adds in one instruction (fma.rn.f32x2, sm_100
// family): d.x = a.x b.x + c.x, d.y = a.y b.y + c.y, each rounded as fmaf.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// Two FP32 products in one instruction (mul.rn.f32x2): d.x = a.x b.x, d.y = a.y b.y.
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// (fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y)) in two packed instructions.
__device__ __forceinline__ float2 fmac2(float a, float2 x, float b, float2 y) {
  return ffma2(make_float2(a, a), x, fmul2(make_float2(b, b), y));
}

// Plane rotation of two entries of a column, x <- cs x + sg y, both rounded as
// fmaf(cs, x, sg * y), two entries per packed instruction.
__device__ __forceinline__ void rot2(float& x0, float& x1, float y0, float y1, float cs, float sg) {
  const float2 r = fmac2(cs, make_float2(x0, x1), sg, make_float2(y0, y1));
  x0 = r.x;
  x1 = r.y;
}

__device__ inline void set_status(int* st, int bits) {
  if (st) atomicOr(st, bits);
}

// cp.async 16-byte copy global -> shared with zero fill of the bytes past src_bytes.
__device__ inline void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
// v = h + m + l exactly (three BF16 parts, each rounded to nearest from the
// remainder of the ones before; exact away from the subnormal range).
__device__ __forceinline__ void split3_bf16(float v, __nv_bfloat16* h, __nv_bfloat16* m, __nv_bfloat16* l) {
  *h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(*h);
  *m = __float2bfloat16_rn(r1);
  *l = __float2bfloat16_rn(r1 - __bfloat162float(*m));
}

// cp.async 8-byte copy with zero fill of the bytes past src_bytes.
__device__ inline void cp_async8(void* smem, const void* gmem, int src_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
// cp.async 4-byte copy with zero fill when src_bytes == 0.
__device__ inline void cp_async4(void* smem, const void* gmem, int src_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

}  // namespace dp2

// Dispatch a runtime sketch width LP (multiple of 8, <= 64) to a template constant L.
// Every kernel launch of the library goes through DP2_COUNTED, which adds one
// to the process-wide launch count (dpar2_kernel_launches) after enqueuing it.
namespace dp2 {
void note_launch();
}
#define DP2_COUNTED(...) ((__VA_ARGS__), ::dp2::note_launch())

#define DP2_LP_SWITCH(LP, CALL)               \
  switch (LP) {                               \
    case 8: { constexpr int L = 8; CALL; } break;   \
    case 16: { constexpr int L = 16; CALL; } break; \
    case 24: { constexpr int L = 24; CALL; } break; \
    case 32: { constexpr int L = 32; CALL; } break; \
    case 40: { constexpr int L = 40; CALL; } break; \
    case 48: { constexpr int L = 48; CALL; } break; \
    case 56: { constexpr int L = 56; CALL; } break; \
    case 64: { constexpr int L = 64; CALL; } break; \
    default: break;                           \
  }

