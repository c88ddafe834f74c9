// Global layout of the tensor-core weight operand (written by the Adam/pack kernel, read by
// the tcgen05 convolution kernels with one bulk copy per pipeline stage).
//
// The GEMM of a 3x3 layer is D[px][n] = sum_k A[px][k] * B[n][k] with k = tap * C_in + c.
// B is stored as a sequence of stage images; one stage = NT output rows x 9 taps x KC input
// channels, laid out exactly as the K-major, no-swizzle shared-memory operand expects:
//   [tap][k-slab of 16 bytes][row (NT)][16 bytes]
// so that 8 rows x 16 bytes form one contiguous 128-byte core matrix. Stages are ordered
// (n-tile, channel chunk). Elements are 16-bit: bf16, or in the float32 form the fp16 hi and lo
// parts of the scaled weights, kept in two such arrays.
#pragma once
#include <stddef.h>

namespace n2f {

struct TcCfg {
  int NT;  // output rows (N) per CTA
  int KC;  // input channels per pipeline stage (one 16-element K step)
  int GE;  // elements per 16 bytes
};

// N = 256 in the bf16 form; 128 in the float32 form, whose stage holds two weight parts
__host__ __device__ __forceinline__ TcCfg tc_cfg(int cin, int cout, int bf16) {
  TcCfg c;
  c.GE = 8;
  c.NT = bf16 ? (cout < 256 ? cout : 256) : (cout < 128 ? cout : 128);
  c.KC = 16;
  (void)cin;
  return c;
}

// log2 of a power of two
__host__ __device__ __forceinline__ int log2_pow2(int v) {
#ifdef __CUDA_ARCH__
  return __ffs(v) - 1;
#else
  return __builtin_ctz((unsigned)v);
#endif
}

// Element offset of B[r][tap * cin + c] in the packed array (NT, KC and GE are powers of two
// for every supported shape: the row split is a shift and a mask).
__host__ __device__ __forceinline__ size_t tc_index_cfg(const TcCfg& f, int cin, int r, int tap,
                                                         int c) {
  const int nchunks = cin / f.KC;
  const int nslab = f.KC / f.GE;
  const int lnt = log2_pow2(f.NT);
  const int nt = r >> lnt, rr = r & (f.NT - 1);
  const int chunk = c / f.KC, cc = c % f.KC;
  const int slab = cc / f.GE, e = cc % f.GE;
  const size_t stage = (size_t)nt * nchunks + chunk;
  return (((stage * 9 + tap) * nslab + slab) * f.NT + rr) * f.GE + e;
}

}  // namespace n2f
