// Helpers shared by the tcgen05 kernel files: the float32 form's scaled fp16 split, alignment
// and the channel-grouped TMA tensor maps (cuTensorMapEncodeTiled resolved from the driver once
// per process).
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>

#include "f16_split.cuh"

namespace n2f {
namespace {

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

// A float32 channel-grouped map act[g][y][x][4] seen as a 3-D tensor (4 W, H, C / 4): a box
// row is a run of bx whole pixels of one group and image row (bx * 16 bytes, at most 256
// floats), so a halo tile costs no extra units at its ends. The box is (4 bx, by rows, bg
// groups); outside the tensor it reads zeros. The innermost start coordinate is 4 x (a whole
// pixel, 16 bytes).
cudaError_t make_map_rows(CUtensorMap* m, const void* base, int C, int H, int W, int bx, int by,
                          int bg) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (4 * bx > 256 || C % 4) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)(4 * W), (cuuint64_t)H, (cuuint64_t)(C / 4)};
  cuuint64_t strides[2] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
  cuuint32_t box[3] = {(cuuint32_t)(4 * bx), (cuuint32_t)by, (cuuint32_t)bg};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace
}  // namespace n2f
