// Allocation-free variant of the weight-gradient entry point.
//
// n2f_conv3x3_wgrad needs a partial-sum workspace (one slice per split of the pixel sum, reduced
// in a fixed order) and obtains it with cudaMallocAsync. Some callers cannot allocate device
// memory at the point where they need a weight gradient: a process whose device memory is
// entirely reserved by another allocator (a framework's caching pool, a fixed-size arena), where
// a cudaMalloc would fail or fragment that reservation, or a latency-sensitive loop that must
// never block on the CUDA allocator. For them this file keeps the workspace in a statically
// sized device array that exists on every GPU the library is loaded on, for the life of the
// process, and passes it to the same kernels.
#include <mutex>

#include "n2f_internal.h"
#include "trainer.h"

namespace {

// 4 Mi floats (16 MiB) of workspace; the last 64 floats hold the kernels' error word.
constexpr size_t kScratchFloats = (size_t)4 << 20;
constexpr size_t kErrFloats = 64;
static __device__ __align__(256) float g_wgrad_scratch[kScratchFloats];

// The address is cached per device ordinal for the life of the process. cudaDeviceReset on a
// device destroys its context and with it the array's old address: a process that resets a
// device and then calls this entry point again on it would pass a stale pointer, so such
// processes must not use this entry point after the reset.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_addr[kMaxDevices] = {};

// Device address of the array on the current device; looked up once per device.
int scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return n2f::set_cuda_error(e, "n2f_conv3x3_wgrad_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return N2F_ENOTSUP;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_wgrad_scratch);
    if (e != cudaSuccess || !p)
      return n2f::set_cuda_error(e, "n2f_conv3x3_wgrad_noalloc: cudaGetSymbolAddress");
    g_addr[dev] = (float*)p;
  }
  *out = g_addr[dev];
  return N2F_OK;
}

}  // namespace

extern "C" int n2f_conv3x3_wgrad_noalloc(int engine, int precision, const void* dout,
                                         const void* in, int cin, int cout, int H, int W,
                                         float* dw, float* db, void* stream) {
  using namespace n2f;
  if (!dout || !in || !dw || !db || H < 1 || W < 1 || cin % 8 || cout % 8 || cin < 8 || cout < 8)
    return N2F_EINVAL;
  if (engine < N2F_ENGINE_AUTO || engine > N2F_ENGINE_TC) return N2F_EINVAL;
  if (precision != N2F_FP32 && precision != N2F_BF16) return N2F_EINVAL;
  // one split of the pixel sum (its weight and bias partials) must fit the array; the
  // tensor-core launcher also keeps up to 63 floats of alignment padding before the bias
  // partials, which the 64 covers; more splits are used when they fit
  const size_t need = (size_t)9 * cin * cout + (size_t)cout + 64;
  if (need > kScratchFloats - kErrFloats) {
    tl_error = "n2f_conv3x3_wgrad_noalloc: layer too large for the fixed 16 MiB workspace";
    return N2F_ETOOBIG;
  }
  const int bf16 = precision == N2F_BF16;
  const bool tc_ok = tc_wgrad_supported(cin, cout, bf16);
  int eng = engine == N2F_ENGINE_SIMT ? N2F_ENGINE_SIMT : (tc_ok ? N2F_ENGINE_TC : N2F_ENGINE_SIMT);
  if (engine == N2F_ENGINE_TC && !tc_ok) return N2F_ENOTSUP;
  float* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cap = kScratchFloats - kErrFloats;
  int* err = reinterpret_cast<int*>(scratch + cap);
  // float32 form: the operands' largest magnitudes (their fp16 scales), beside the error word
  unsigned* dmax = reinterpret_cast<unsigned*>(err + 1);
  unsigned* xmax = dmax + 1;
  const bool tc = eng == N2F_ENGINE_TC;
  // the partial sums are overwritten in full by every call; the error and magnitude words start
  // at zero
  cudaError_t e = cudaMemsetAsync(err, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess && tc && !bf16)
    e = launch_absmax(dout, (size_t)cout * H * W, 0, dmax, nullptr, st);
  if (e == cudaSuccess && tc && !bf16) e = launch_absmax(in, (size_t)cin * H * W, 0, xmax, nullptr, st);
  if (e == cudaSuccess)
    e = tc ? launch_wgrad_tc(bf16, dout, in, cin, cout, H, W, dmax, xmax, scratch, cap, dw, db,
                             nullptr, err, st)
           : launch_wgrad_simt(bf16, dout, in, cin, cout, H, W, scratch, cap, dw, db, nullptr, st);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_conv3x3_wgrad_noalloc");
  return herr ? N2F_ETIMEDOUT : N2F_OK;
}
