// Philox4x32-10 Gaussian streams (test matrices Omega, Omega2 and the initial V).
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw (SC'11): ten
// rounds, multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by 0x9E3779B9 /
// 0xBB67AE85 between rounds.  Stream convention: element n of the stream
// (seed, stream_id) is word n % 4 of the block with counter
// (n/4 lo, n/4 hi, stream_id, 0) and key (seed lo, seed hi).  Gaussians come
// from Box-Muller on the word pairs (0,1) and (2,3) with uniforms
// u = (word + 0.5) / 2^32.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace dp2 {

__device__ inline uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ inline float round16(float v) {
  float r = __bfloat162float(__float2bfloat16_rn(v));
  return fabsf(r) < 6.103515625e-05f ? 0.0f : r;  // 2^-14
}

__global__ void k_gaussian(uint64_t seed, uint32_t sid, int64_t n, float* __restrict__ out, int r16) {
  const int64_t nb = (n + 3) / 4;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    uint4 w = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), sid, 0u), key);
    const float s = 2.3283064365386963e-10f;  // 2^-32
    float u0 = ((float)w.x + 0.5f) * s, u1 = ((float)w.y + 0.5f) * s;
    float u2 = ((float)w.z + 0.5f) * s, u3 = ((float)w.w + 0.5f) * s;
    float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s0, c0, s1, c1;
    sincospif(2.0f * u1, &s0, &c0);
    sincospif(2.0f * u3, &s1, &c1);
    float z[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t idx = 4 * b + i;
      if (idx < n) out[idx] = r16 ? round16(z[i]) : z[i];
    }
  }
}

__global__ void k_philox_words(uint64_t seed, uint32_t sid, int64_t n, uint32_t* __restrict__ out) {
  const int64_t nb = (n + 3) / 4;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    uint4 w = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), sid, 0u), key);
    uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (4 * b + i < n) out[4 * b + i] = v[i];
  }
}

// Omega (J x ell, row-major) -> Jpad x LP zero-padded copy; 16-bit X uses the
// values rounded to its own type (so the MMA and the CUDA-core paths agree).
__global__ void k_pad_omega(const float* __restrict__ om, int J, int ell, int Jpad, int LP, int dt,
                            float* __restrict__ out) {
  int64_t n = (int64_t)Jpad * LP;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int j = (int)(i / LP), c = (int)(i % LP);
    float v = (j < J && c < ell) ? om[(int64_t)j * ell + c] : 0.0f;
    if (dt == DPAR2_BF16) v = __bfloat162float(__float2bfloat16_rn(v));
    if (dt == DPAR2_F16) v = __half2float(__float2half_rn(v));
    out[i] = v;
  }
}

// Packed rows (J elements of es bytes each) -> rows of ldx elements, the
// columns J .. ldx - 1 zeroed; one warp per row, 2- or 4-byte elements.
__global__ void k_repitch(const uint8_t* __restrict__ src, int64_t rows, int J, int es, uint8_t* __restrict__ dst,
                          int64_t ldx) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    if (es == 2) {
      const uint16_t* sr = reinterpret_cast<const uint16_t*>(src) + r * J;
      uint16_t* dr = reinterpret_cast<uint16_t*>(dst) + r * ldx;
      for (int64_t j = lane; j < ldx; j += 32) dr[j] = j < J ? sr[j] : (uint16_t)0;
    } else {
      const uint32_t* sr = reinterpret_cast<const uint32_t*>(src) + r * J;
      uint32_t* dr = reinterpret_cast<uint32_t*>(dst) + r * ldx;
      for (int64_t j = lane; j < ldx; j += 32) dr[j] = j < J ? sr[j] : 0u;
    }
  }
}

static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 65535 * 4 ? 65535 * 4 : g));
}

void launch_gaussian(uint64_t seed, uint32_t sid, int64_t n, float* out, int r16, cudaStream_t s) {
  DP2_COUNTED(k_gaussian<<<grid_for((n + 3) / 4, 256), 256, 0, s>>>(seed, sid, n, out, r16));
}
void launch_philox_words(uint64_t seed, uint32_t sid, int64_t n, uint32_t* out, cudaStream_t s) {
  DP2_COUNTED(k_philox_words<<<grid_for((n + 3) / 4, 256), 256, 0, s>>>(seed, sid, n, out));
}
void launch_repitch(const void* src, int64_t rows, int J, int es, void* dst, int64_t ldx, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((rows + 7) / 8, 65535);
  DP2_COUNTED(k_repitch<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, s>>>(static_cast<const uint8_t*>(src), rows, J, es,
                                                                   static_cast<uint8_t*>(dst), ldx));
}

void launch_pad_omega(const float* om, int J, int ell, int Jpad, int LP, dpar2_dtype dt, float* out,
                      cudaStream_t s) {
  DP2_COUNTED(k_pad_omega<<<grid_for((int64_t)Jpad * LP, 256), 256, 0, s>>>(om, J, ell, Jpad, LP, (int)dt, out));
}

}  // namespace dp2
