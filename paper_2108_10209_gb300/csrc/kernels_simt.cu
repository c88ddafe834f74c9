// CUDA-core implicit-GEMM kernels for the 3x3 layers with C_in >= 8 (the float32 reference
// kernels; also instantiated for bfloat16 storage). Forward and dgrad share one kernel:
//   forward: out(p, o) = ReLU(b_o + sum_{tap, c} W[o][c][tap] in(p + tap, c))
//   dgrad:   out(p, c) = [mask(p, c) > 0] * sum_{tap', o} W[o][c][8 - tap'] in(p + tap', o)
// (the dgrad weight copy already holds the rotated transpose, so both run the same loop).
#include "cg_util.cuh"
#include "checked.cuh"
#include "n2f_internal.h"

namespace n2f {

namespace {

constexpr int TX = 64;  // pixels of one image row per CTA
constexpr int TO = 64;  // output channels per CTA
constexpr int KC = 8;   // input channels per smem stage

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_conv_simt(const T* __restrict__ in, int cin, int cout,
                                                   int H, int W, const float* __restrict__ wk,
                                                   const float* __restrict__ bias,
                                                   const T* __restrict__ mask, T* __restrict__ out,
                                                   const int* skip) {
  if (skip && *skip) return;
  constexpr int G = CGTraits<T>::G;
  __shared__ float sIn[3][KC][TX + 2];
  __shared__ __align__(16) float sW[9][KC][TO];
  const int tid = threadIdx.x, tx = tid & 15, to = tid >> 4;
  const int y = blockIdx.y, x0 = blockIdx.x * TX, o0 = blockIdx.z * TO;
  const size_t npx = (size_t)H * W;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int c0 = 0; c0 < cin; c0 += KC) {
    __syncthreads();
    for (int i = tid; i < 3 * (TX + 2) * (KC / G); i += 256) {
      const int px = i % (TX + 2), r = (i / (TX + 2)) % 3, gg = i / ((TX + 2) * 3);
      const int yy = y + r - 1, xx = x0 + px - 1;
      float v[G];
      if (yy >= 0 && yy < H && xx >= 0 && xx < W &&
          N2F_IN((size_t)(c0 / G + gg) * npx + (size_t)yy * W + xx, (size_t)(cin / G) * npx)) {
        load_group<T>(in, (size_t)(c0 / G + gg) * npx + (size_t)yy * W + xx, v);
      } else {
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < G; ++k) sIn[r][gg * G + k][px] = v[k];
    }
    const float* wsrc = wk + (size_t)(c0 / KC) * 9 * KC * cout;
    for (int i = tid; i < 9 * KC * TO; i += 256) {
      const int oc = i % TO, tk = i / TO;  // tk = tap * KC + cc
      sW[tk / KC][tk % KC][oc] = (o0 + oc < cout) ? wsrc[(size_t)tk * cout + o0 + oc] : 0.f;
    }
    __syncthreads();
#pragma unroll 3
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap % 3;
#pragma unroll
      for (int cc = 0; cc < KC; ++cc) {
        float a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sIn[dy][cc][tx + 16 * i + dx];
        const float4 w4 = *reinterpret_cast<const float4*>(&sW[tap][cc][to * 4]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[i][0] += a[i] * w4.x;
          acc[i][1] += a[i] * w4.y;
          acc[i][2] += a[i] * w4.z;
          acc[i][3] += a[i] * w4.w;
        }
      }
    }
  }
  const int oc0 = o0 + to * 4;
  if (oc0 >= cout) return;
  const int g = oc0 / G, k0 = oc0 % G;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int x = x0 + tx + 16 * i;
    if (x >= W) continue;
    const size_t p = (size_t)y * W + x;
    if (!N2F_IN((size_t)g * npx + p, (size_t)(cout / G) * npx)) continue;
    float mk[G];
    if (MODE == 1) load_group<T>(mask, (size_t)g * npx + p, mk);
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float r = acc[i][j];
      if (MODE == 0) {
        r += bias[oc0 + j];
        r = r > 0.f ? r : 0.f;
      } else {
        r = mk[k0 + j] > 0.f ? r : 0.f;
      }
      v[j] = r;
    }
    // each thread owns 4 channels: a whole float32 group or one 8-byte half of a bf16 group
    store4<T>(out, ((size_t)g * npx + p) * G + k0, v);
  }
}

// Weight gradient: dW[o][c][tap] = sum_p d(p, o) in(p + tap, c), db[o] = sum_p d(p, o).
// CTA (o-tile of 32, c-tile of 32, split s) sums its rows in raster order; partials land in
// part[s][q] with q the canonical flat index, reduced afterwards in ascending s.
constexpr int WTX = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_wgrad_simt(const T* __restrict__ dout,
                                                    const T* __restrict__ in, int cin, int cout,
                                                    int H, int W, int rows, float* __restrict__ part,
                                                    size_t part_cap, const int* skip) {
  if (skip && *skip) return;
  constexpr int G = CGTraits<T>::G;
  __shared__ __align__(16) float sD[WTX][36];
  __shared__ float sA[3][WTX + 2][33];
  const int tid = threadIdx.x, ic = tid & 31, og = tid >> 5;
  const int o0 = blockIdx.x * 32, c0 = blockIdx.y * 32, s = blockIdx.z;
  const int ya = s * rows, yb = min(H, ya + rows);
  const size_t npx = (size_t)H * W;
  float acc[4][9], bacc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    bacc[j] = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[j][t] = 0.f;
  }
  for (int y = ya; y < yb; ++y) {
    for (int x0 = 0; x0 < W; x0 += WTX) {
      __syncthreads();
      for (int i = tid; i < WTX * (32 / G); i += 256) {
        const int px = i % WTX, gg = i / WTX;
        const int x = x0 + px, gi = o0 / G + gg;
        float v[G];
        if (x < W && gi * G < cout) {
          load_group<T>(dout, (size_t)gi * npx + (size_t)y * W + x, v);
        } else {
#pragma unroll
          for (int k = 0; k < G; ++k) v[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < G; ++k) sD[px][gg * G + k] = v[k];
      }
      for (int i = tid; i < 3 * (WTX + 2) * (32 / G); i += 256) {
        const int px = i % (WTX + 2), r = (i / (WTX + 2)) % 3, gg = i / ((WTX + 2) * 3);
        const int yy = y + r - 1, xx = x0 + px - 1, gi = c0 / G + gg;
        float v[G];
        if (yy >= 0 && yy < H && xx >= 0 && xx < W && gi * G < cin) {
          load_group<T>(in, (size_t)gi * npx + (size_t)yy * W + xx, v);
        } else {
#pragma unroll
          for (int k = 0; k < G; ++k) v[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < G; ++k) sA[r][px][gg * G + k] = v[k];
      }
      __syncthreads();
      const int npx_tile = min(WTX, W - x0);
      for (int px = 0; px < npx_tile; ++px) {
        const float4 d = *reinterpret_cast<const float4*>(&sD[px][og * 4]);
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const float a = sA[t / 3][px + t % 3][ic];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j][t] += dv[j] * a;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) bacc[j] += dv[j];
      }
    }
  }
  const size_t Q = (size_t)cout * cin * 9 + cout;
  float* pp = part + (size_t)s * Q;
  const int c = c0 + ic;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = o0 + og * 4 + j;
    if (o >= cout) continue;
    if (c < cin)
#pragma unroll
      for (int t = 0; t < 9; ++t)
        if (N2F_IN(pp + ((size_t)o * cin + c) * 9 + t - part, part_cap))
          pp[((size_t)o * cin + c) * 9 + t] = acc[j][t];
    if (blockIdx.y == 0 && ic == 0 && N2F_IN(pp + (size_t)cout * cin * 9 + o - part, part_cap))
      pp[(size_t)cout * cin * 9 + o] = bacc[j];
  }
}

__global__ void k_reduce_parts(const float* __restrict__ part, int S, size_t Q, size_t nw,
                               float* __restrict__ gw, float* __restrict__ gb, const int* skip) {
  if (skip && *skip) return;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < Q;
       q += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += part[(size_t)k * Q + q];
    if (q < nw)
      gw[q] = s;
    else
      gb[q - nw] = s;
  }
}

}  // namespace

cudaError_t launch_conv_simt(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                             const float* wk, const float* b, const void* mask, void* out,
                             const int* skip, cudaStream_t st) {
  if (cin % 8 || cout % 8) return cudaErrorInvalidValue;
  dim3 grid((W + TX - 1) / TX, H, (cout + TO - 1) / TO);
  if (bf16) {
    using T = __nv_bfloat16;
    if (mode == 0)
      k_conv_simt<T, 0><<<grid, 256, 0, st>>>((const T*)in, cin, cout, H, W, wk, b, nullptr,
                                              (T*)out, skip);
    else
      k_conv_simt<T, 1><<<grid, 256, 0, st>>>((const T*)in, cin, cout, H, W, wk, nullptr,
                                              (const T*)mask, (T*)out, skip);
  } else {
    using T = float;
    if (mode == 0)
      k_conv_simt<T, 0><<<grid, 256, 0, st>>>((const T*)in, cin, cout, H, W, wk, b, nullptr,
                                              (T*)out, skip);
    else
      k_conv_simt<T, 1><<<grid, 256, 0, st>>>((const T*)in, cin, cout, H, W, wk, nullptr,
                                              (const T*)mask, (T*)out, skip);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_wgrad_simt(int bf16, const void* dout, const void* in, int cin, int cout, int H,
                              int W, float* part, size_t part_cap, float* gw, float* gb,
                              const int* skip, cudaStream_t st) {
  if (cin % 8 || cout % 8) return cudaErrorInvalidValue;
  const int tiles = ((cout + 31) / 32) * ((cin + 31) / 32);
  const size_t Q = (size_t)cout * cin * 9 + cout;
  int S = (152 * 4 + tiles - 1) / tiles;
  if (S > H) S = H;
  if ((size_t)S * Q > part_cap) S = (int)(part_cap / Q);
  if (S < 1) return cudaErrorInvalidValue;
  const int rows = (H + S - 1) / S;
  S = (H + rows - 1) / rows;
  dim3 grid((cout + 31) / 32, (cin + 31) / 32, S);
  if (bf16)
    k_wgrad_simt<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)dout,
                                                      (const __nv_bfloat16*)in, cin, cout, H, W,
                                                      rows, part, part_cap, skip);
  else
    k_wgrad_simt<float><<<grid, 256, 0, st>>>((const float*)dout, (const float*)in, cin, cout, H,
                                              W, rows, part, part_cap, skip);
  count_launch();
  unsigned g = (unsigned)((Q + 255) / 256);
  if (g > 152u * 8) g = 152u * 8;
  k_reduce_parts<<<g, 256, 0, st>>>(part, S, Q, (size_t)cout * cin * 9, gw, gb, skip);
  count_launch();
  return cudaGetLastError();
}

N2F_CHECK_READER(check_read_simt)

}  // namespace n2f
