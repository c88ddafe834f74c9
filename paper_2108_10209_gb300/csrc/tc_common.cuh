// Helpers shared by the tcgen05 kernel files: TF32 rounding, alignment and the channel-grouped
// TMA tensor maps (cuTensorMapEncodeTiled resolved from the driver once per process).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <mutex>

namespace n2f {
namespace {

// Round to the nearest TF32 value (10 explicit mantissa bits; ties away from zero) by adding
// half a unit of the 13 dropped bits before clearing them. The 3xTF32 split x = hi + lo uses
// it for both parts, so hi and lo are exact TF32 numbers and the dropped lo*lo term and the
// rounding of lo are unbiased, about 2^-22 of x.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void split4(float4 v, float4& h, float4& l) {
  h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
  l = make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y), tf32_round(v.z - h.z),
                  tf32_round(v.w - h.w));
}

__host__ __device__ constexpr uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// ---- tensor maps ----------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// A channel-grouped map act[g][y][x][GE] seen as a 4-D tensor (GE * pu, W / pu, H, C / GE),
// innermost first: `pu` consecutive pixels form one unit, so a box row is pu * 16 bytes (TMA
// moves whole 32-byte sectors: 16-byte rows would fetch every sector twice). The box is
// (GE * pu, bx units, by rows, bg groups); outside the tensor it reads zeros. W must be a
// multiple of pu.
cudaError_t make_map(CUtensorMap* m, const void* base, int bf16, int C, int H, int W, int bx,
                     int by, int bg, int pu = 1) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (pu < 1 || W % pu) return cudaErrorInvalidValue;
  const int GE = bf16 ? 8 : 4;
  cuuint64_t dims[4] = {(cuuint64_t)(GE * pu), (cuuint64_t)(W / pu), (cuuint64_t)H,
                        (cuuint64_t)(C / GE)};
  cuuint64_t strides[3] = {(cuuint64_t)pu * 16, (cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
  cuuint32_t box[4] = {(cuuint32_t)(GE * pu), (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bg};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace
}  // namespace n2f
