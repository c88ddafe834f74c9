// Single-tile tcgen05 GEMM on operands given as shared-memory images (the diagnostic entry point
// that pins the descriptor layouts) and tc_prepare, which readies every tensor-core kernel.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "cg_util.cuh"
#include "n2f_internal.h"
#include "tc_common.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"
#include "trainer.h"

namespace n2f {

using namespace tc;

namespace {

// ---- single-tile GEMM with operands given as shared-memory images -------------------------
struct ProbeArgs {
  const uint4* A;
  const uint4* B;
  float* D;
  int N, ksteps, tf32;
  uint32_t a_bytes, b_bytes, a_lbo, a_sbo, b_lbo, b_sbo, a_kstep, b_kstep, id;
  int* err;
};

__global__ void __launch_bounds__(128, 1) k_umma_probe(ProbeArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // A in [0, 100 KB), B in [100 KB, 200 KB) of a fixed 200 KB allocation
  uint8_t* sA = smem;
  uint8_t* sB = smem + 100 * 1024;
  for (uint32_t i = tid; i < a.a_bytes / 16; i += 128) reinterpret_cast<uint4*>(sA)[i] = a.A[i];
  for (uint32_t i = tid; i < a.b_bytes / 16; i += 128) reinterpret_cast<uint4*>(sB)[i] = a.B[i];
  fence_proxy_async();
  if (tid == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  const uint32_t ncols = tmem_cols(a.N);
  if (warp == 0) tmem_alloc(&tslot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  if (tid == 0) {
    for (int s = 0; s < a.ksteps; ++s) {
      const uint64_t da = sdesc(smem_u32(sA) + s * a.a_kstep, a.a_lbo, a.a_sbo);
      const uint64_t db = sdesc(smem_u32(sB) + s * a.b_kstep, a.b_lbo, a.b_sbo);
      if (a.tf32)
        mma_tf32(tbase, da, db, a.id, s > 0);
      else
        mma_f16(tbase, da, db, a.id, s > 0);
    }
    mma_commit(&bar);
  }
  __syncwarp();
  if (!mbar_wait(&bar, 0, &abort_flag, a.err)) mbar_drain(&bar, 0);
  tc_fence_after();
  for (int c = 0; c < a.N; c += 16) {
    uint32_t r[16];
    tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c, r);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; ++j) a.D[(size_t)(warp * 32 + lane) * a.N + c + j] = __uint_as_float(r[j]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// ---- bounded-wait check --------------------------------------------------------------------
// One warp waits on an mbarrier that nothing ever arrives on, with the same bounded wait as
// the tensor-core kernels (here with a caller-given limit): the wait must give up, record the
// time-out in the error word and let the kernel return.
__global__ void k_wait_probe(uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  mbar_wait_for(&bar, 0, &abort_flag, err, limit_ns);
}

}  // namespace

// Resolves the tensor-map encoder and sets the shared-memory limits of every tensor-core kernel
// once per process.
cudaError_t tc_prepare() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    if (!encode_fn()) {
      result = cudaErrorNotSupported;
      return;
    }
    cudaError_t e = conv_tc_prepare();
    if (e == cudaSuccess) e = wgrad_tc_prepare();
    result = e;
  });
  return result;
}

}  // namespace n2f

// ---- diagnostic entry point (declared in n2f.h) ---------------------------------------------
extern "C" int n2f_umma_gemm(int tf32, int N, int K, int a_mn, int b_mn, const void* A,
                             size_t a_bytes, uint32_t a_lbo, uint32_t a_sbo, uint32_t a_kstep,
                             const void* B, size_t b_bytes, uint32_t b_lbo, uint32_t b_sbo,
                             uint32_t b_kstep, float* D, void* stream) {
  using namespace n2f;
  if (!A || !B || !D || N < 16 || N > 256 || N % 16 || K < 1 || a_bytes % 16 || b_bytes % 16)
    return N2F_EINVAL;
  const int kstep = tf32 ? 8 : 16;
  if (K % kstep) return N2F_EINVAL;
  const uint32_t smem = 200 * 1024;
  if (a_bytes > 100 * 1024 || b_bytes > 100 * 1024) return N2F_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaFuncSetAttribute(k_umma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  int* err = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_umma_gemm");
  ProbeArgs a;
  a.A = (const uint4*)A;
  a.B = (const uint4*)B;
  a.D = D;
  a.N = N;
  a.ksteps = K / kstep;
  a.tf32 = tf32;
  a.a_bytes = (uint32_t)a_bytes;
  a.b_bytes = (uint32_t)b_bytes;
  a.a_lbo = a_lbo;
  a.a_sbo = a_sbo;
  a.b_lbo = b_lbo;
  a.b_sbo = b_sbo;
  a.a_kstep = a_kstep;
  a.b_kstep = b_kstep;
  a.id = idesc(tf32 ? 2 : 1, 128, N, a_mn, b_mn);
  a.err = err;
  k_umma_probe<<<1, 128, smem, st>>>(a);
  e = cudaGetLastError();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_umma_gemm");
  return herr ? N2F_ETIMEDOUT : N2F_OK;
}

// ---- diagnostic entry point: the bounded wait gives up (declared in n2f.h) -----------------
extern "C" int n2f_wait_probe(uint32_t limit_ms, void* stream) {
  using namespace n2f;
  if (limit_ms < 1 || limit_ms > 10000) return N2F_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&err, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_wait_probe");
  k_wait_probe<<<1, 32, 0, st>>>((uint64_t)limit_ms * 1000000ull, err);
  e = cudaGetLastError();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (e != cudaSuccess) return set_cuda_error(e, "n2f_wait_probe");
  return herr ? N2F_ETIMEDOUT : N2F_OK;
}
