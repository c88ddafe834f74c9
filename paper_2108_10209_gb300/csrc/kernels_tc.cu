// tcgen05 / TMEM implicit-GEMM convolution kernels (sm_103a). Placeholder until the
// tensor-core path lands: no shape is covered, so every layer runs on the SIMT kernels.
#include "n2f_internal.h"
#include "tc_layout.cuh"

namespace n2f {

bool tc_supported(int, int) { return false; }
size_t tc_weight_elems(int cin, int cout) { return (size_t)cin * cout * 9; }
cudaError_t launch_conv_tc(int, int, const void*, int, int, int, int, const void*, const float*,
                           const void*, void*, const int*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_wgrad_tc(int, const void*, const void*, int, int, int, int, float*, size_t,
                            float*, float*, const int*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace n2f
