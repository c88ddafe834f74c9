// The float32 form's operand representation for the tensor cores: two power-of-two-scaled fp16
// parts per value (used by the packing kernel and the tcgen05 kernels).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace n2f {

// A tensor with largest magnitude m is multiplied by the power of two s = 2^k that puts m just
// below 2^14 (k from m's exponent; clamped to the normal range) and split as x s = hi + lo,
// hi = fp16(x s), lo = fp16(x s - hi); x s - hi is exact in fp32. Products hi*hi + hi*lo + lo*hi
// (the lo*lo term is dropped) carry about 22 significant bits, as 3xTF32 does, but at the fp16
// tensor rate. Every value within 2^-17 of m keeps both parts normal; below that the absolute
// error stays under m 2^-39. The scaled values never exceed 2^14, so no part overflows.
__host__ __device__ __forceinline__ int f16_scale_exp(unsigned mbits) {
  if (mbits == 0u) return 0;
  const int e = (int)((mbits >> 23) & 0xffu);  // m < 2^(e - 126)
  int k = 140 - e;
  return k < -126 ? -126 : (k > 126 ? 126 : k);
}
__host__ __device__ __forceinline__ float pow2f(int k) {  // k in [-126, 127]
  union {
    unsigned u;
    float f;
  } c;
  c.u = (unsigned)(127 + k) << 23;
  return c.f;
}
__device__ __forceinline__ float f16_scale(const unsigned* m) { return pow2f(f16_scale_exp(*m)); }
__device__ __forceinline__ float f16_unscale(const unsigned* m) { return pow2f(-f16_scale_exp(*m)); }

// Two values (a in the low half) -> their scaled hi and lo fp16 parts, packed in pairs.
__device__ __forceinline__ void split_f16_pair(float a, float b, float s, uint32_t& hi,
                                               uint32_t& lo) {
  const float x = a * s, y = b * s;
  const __half2 h = __floats2half2_rn(x, y);
  const float2 f = __half22float2(h);
  const __half2 l = __floats2half2_rn(x - f.x, y - f.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Eight fp32 values (two float4 groups) -> one 16-byte group of hi parts and one of lo parts.
__device__ __forceinline__ void split_f16_group(const float4 u, const float4 v, float s, uint4& hi,
                                                uint4& lo) {
  split_f16_pair(u.x, u.y, s, hi.x, lo.x);
  split_f16_pair(u.z, u.w, s, hi.y, lo.y);
  split_f16_pair(v.x, v.y, s, hi.z, lo.z);
  split_f16_pair(v.z, v.w, s, hi.w, lo.w);
}

// Largest |v| of the calling lanes' values raised into *dst (float bits; non-negative floats
// order as their bit patterns): one atomic per warp.
__device__ __forceinline__ void warp_absmax_to(float m, unsigned* dst) {
  const unsigned mask = __activemask();
  const unsigned b = __reduce_max_sync(mask, __float_as_uint(fabsf(m)));
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1 && b) atomicMax(dst, b);
}

// Block-wide: every thread of the block (a multiple of 32) calls it; one global atomic per block.
__device__ __forceinline__ void block_absmax_to(float m, unsigned* dst) {
  __shared__ unsigned sm;
  if (threadIdx.x == 0) sm = 0u;
  __syncthreads();
  const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(m)));
  if ((threadIdx.x & 31) == 0 && b) atomicMax(&sm, b);
  __syncthreads();
  if (threadIdx.x == 0 && sm) atomicMax(dst, sm);
}

}  // namespace n2f
