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

__device__ inline void set_status(int* st, int bits) {
  if (st) atomicOr(st, bits);
}

// cp.async 16-byte copy global -> shared with zero fill of the bytes past src_bytes.
__device__ inline void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

}  // namespace dp2

// Dispatch a runtime sketch width LP (multiple of 8, <= 64) to a template constant L.
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

