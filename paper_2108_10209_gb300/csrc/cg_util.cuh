// Channel-grouped ("CG") activation layout helpers: act[g][pixel][k], c = g * G + k, one
// 16-byte group per (pixel, g): G = 4 float32 or G = 8 bfloat16 channels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace n2f {

template <typename T>
struct CGTraits;
template <>
struct CGTraits<float> {
  static constexpr int G = 4;
  __device__ __forceinline__ static float from_float(float v) { return v; }
  __device__ __forceinline__ static float to_float(float v) { return v; }
};
template <>
struct CGTraits<__nv_bfloat16> {
  static constexpr int G = 8;
  __device__ __forceinline__ static __nv_bfloat16 from_float(float v) {
    return __float2bfloat16_rn(v);
  }
  __device__ __forceinline__ static float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// Loads / stores the 16-byte group number `idx` (= g * npx + pixel) as floats.
template <typename T>
__device__ __forceinline__ void load_group(const T* base, size_t idx, float* v);
template <>
__device__ __forceinline__ void load_group<float>(const float* base, size_t idx, float* v) {
  const float4 q = reinterpret_cast<const float4*>(base)[idx];
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load_group<__nv_bfloat16>(const __nv_bfloat16* base, size_t idx,
                                                          float* v) {
  const uint4 q = reinterpret_cast<const uint4*>(base)[idx];
  const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
// The same conversion from a 16-byte group already in registers (e.g. loaded ahead of use).
template <typename T>
__device__ __forceinline__ void group_from_raw(uint4 q, float* v);
template <>
__device__ __forceinline__ void group_from_raw<float>(uint4 q, float* v) {
  v[0] = __uint_as_float(q.x); v[1] = __uint_as_float(q.y);
  v[2] = __uint_as_float(q.z); v[3] = __uint_as_float(q.w);
}
template <>
__device__ __forceinline__ void group_from_raw<__nv_bfloat16>(uint4 q, float* v) {
  const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

template <typename T>
__device__ __forceinline__ void store_group(T* base, size_t idx, const float* v);
template <>
__device__ __forceinline__ void store_group<float>(float* base, size_t idx, const float* v) {
  reinterpret_cast<float4*>(base)[idx] = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store_group<__nv_bfloat16>(__nv_bfloat16* base, size_t idx,
                                                           const float* v) {
  unsigned w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const unsigned*>(&h);
  }
  reinterpret_cast<uint4*>(base)[idx] = make_uint4(w[0], w[1], w[2], w[3]);
}

// Stores 4 consecutive channels starting at element offset `off` (a multiple of 4).
template <typename T>
__device__ __forceinline__ void store4(T* base, size_t off, const float* v);
template <>
__device__ __forceinline__ void store4<float>(float* base, size_t off, const float* v) {
  *reinterpret_cast<float4*>(base + off) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16* base, size_t off,
                                                      const float* v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
  const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
  *reinterpret_cast<uint2*>(base + off) =
      make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
}

}  // namespace n2f
