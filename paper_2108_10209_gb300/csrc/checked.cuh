// Bounds checks of the checked build (compiled with N2F_CHECKED into libn2f_checked.so by
// build.py --checked). In place of a memory checker, the kernels test their computed
// global-memory indexes against the extent of the tensor each addresses (known from the launch
// shapes): an index out of range is counted, the first failing source line is recorded, and
// the access is skipped -- nothing traps, the kernel carries on and the context stays usable.
// The host reads the counts with n2f_check_status. In the normal build every check is the
// constant `true` and compiles away.
#pragma once
#include <cuda_runtime.h>

#ifdef N2F_CHECKED
namespace n2f {
namespace chk {

// One pair of words per translation unit (static: each .cu file's kernels count in their own).
static __device__ unsigned long long g_fails;
static __device__ int g_first_line;

__device__ __noinline__ static bool fail(int line) {
  atomicAdd(&g_fails, 1ull);
  atomicCAS(&g_first_line, 0, line);
  return false;
}

// Host: this translation unit's words on the current device; clear = 1 zeroes them after.
static inline int read(unsigned long long* fails, int* line, int clear) {
  if (cudaMemcpyFromSymbol(fails, g_fails, sizeof(*fails)) != cudaSuccess ||
      cudaMemcpyFromSymbol(line, g_first_line, sizeof(*line)) != cudaSuccess)
    return -1;
  if (clear) {
    const unsigned long long z = 0;
    const int zl = 0;
    if (cudaMemcpyToSymbol(g_fails, &z, sizeof(z)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_first_line, &zl, sizeof(zl)) != cudaSuccess)
      return -1;
  }
  return 0;
}

}  // namespace chk
}  // namespace n2f

// true when 0 <= i < n; otherwise counts a failure (the caller then skips the access)
#define N2F_IN(i, n) \
  ((unsigned long long)(i) < (unsigned long long)(n) || ::n2f::chk::fail(__LINE__))
// defines `int name(unsigned long long*, int*, int clear)` reading this file's words
#define N2F_CHECK_READER(name)                                  \
  int name(unsigned long long* fails, int* line, int clear) {   \
    return ::n2f::chk::read(fails, line, clear);                \
  }
#else
#define N2F_IN(i, n) true
#define N2F_CHECK_READER(name)                                  \
  int name(unsigned long long* fails, int* line, int clear) {   \
    (void)clear;                                                \
    *fails = 0;                                                 \
    *line = 0;                                                  \
    return 0;                                                   \
  }
#endif
