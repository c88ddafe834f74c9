// Memory-bound kernels of the Noise2Fast path: checkerboard gather, weight init, Adam with
// weight packing, CG-layout packing, the one-channel first layer, the head (1x1 conv +
// sigmoid + loss), the FP64 validation reduction, the stopping rule and output averaging.
#include <math.h>

#include "cg_util.cuh"
#include "checked.cuh"
#include "f16_split.cuh"
#include "n2f_internal.h"
#include "tc_layout.cuh"

namespace n2f {

thread_local uint64_t* tl_launch_counter = nullptr;

#define N2F_LAUNCH_CHECK() \
  do {                     \
    count_launch();        \
    return cudaGetLastError(); \
  } while (0)

static inline unsigned nblocks(size_t n, int per) { return (unsigned)((n + per - 1) / per); }

// ---------------------------------------------------------------------------------------------
// Checkerboard downsampling (Theoretical Background Eq. 6-7; Methods, the "left" equations).
// Odd images: the pixels with i+j odd, compacted in order. Pure copies, bit-exact.
__global__ void k_gather(const float* __restrict__ x, int H, int W, float* __restrict__ ue,
                         float* __restrict__ uo, float* __restrict__ le, float* __restrict__ lo) {
  const int hw = W >> 1, hh = H >> 1;
  const size_t nup = (size_t)H * hw, nlf = (size_t)hh * W;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nup + nlf;
       t += (size_t)gridDim.x * blockDim.x) {
    if (t < nup) {
      const int i = (int)(t / hw), j = (int)(t % hw);
      const float* row = x + (size_t)i * W;
      const int je = 2 * j + (i & 1), jo = 2 * j + 1 - (i & 1);
      if (N2F_IN(je, W) && N2F_IN(jo, W)) {
        ue[t] = row[je];
        uo[t] = row[jo];
      }
    } else {
      const size_t u = t - nup;
      const int i = (int)(u / W), j = (int)(u % W);
      const int ie = 2 * i + (j & 1), io = 2 * i + 1 - (j & 1);
      if (N2F_IN(ie, H) && N2F_IN(io, H)) {
        le[u] = x[(size_t)ie * W + j];
        lo[u] = x[(size_t)io * W + j];
      }
    }
  }
}

cudaError_t launch_gather(const float* x, int H, int W, float* ue, float* uo, float* le, float* lo,
                          cudaStream_t st) {
  const size_t n = (size_t)H * (W / 2) + (size_t)(H / 2) * W;
  unsigned g = nblocks(n, 256);
  if (g > 152u * 16) g = 152u * 16;
  k_gather<<<g, 256, 0, st>>>(x, H, W, ue, uo, le, lo);
  N2F_LAUNCH_CHECK();
}

// Ablation Study, "Quad": 2x2 blocks -> the images of their top-left, top-right, bottom-right
// and bottom-left pixels (stored in that order: the training pairs go k -> k+1 mod 4), each
// floor(H/2) x floor(W/2). Pure copies, bit-exact.
__global__ void k_gather_quad(const float* __restrict__ x, int H, int W, float* __restrict__ tl,
                              float* __restrict__ tr, float* __restrict__ br,
                              float* __restrict__ bl) {
  const int hh = H >> 1, hw = W >> 1;
  const size_t n = (size_t)hh * hw;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / hw), j = (int)(t % hw);
    const float* r0 = x + (size_t)(2 * i) * W + 2 * j;
    const float* r1 = r0 + W;
    tl[t] = r0[0];
    tr[t] = r0[1];
    bl[t] = r1[0];
    br[t] = r1[1];
  }
}

cudaError_t launch_gather_quad(const float* x, int H, int W, float* tl, float* tr, float* br,
                               float* bl, cudaStream_t st) {
  const size_t n = (size_t)(H / 2) * (W / 2);
  unsigned g = nblocks(n, 256);
  if (g > 152u * 16) g = 152u * 16;
  k_gather_quad<<<g, 256, 0, st>>>(x, H, W, tl, tr, br, bl);
  N2F_LAUNCH_CHECK();
}

// Ablation Study, "Exact": target = x_tgt - (s_tgt - s_in), the signal difference taken from
// the clean image's sub-images (the s_odd - s_even term of the Theoretical Background).
__global__ void k_exact_target(const float* __restrict__ xt, const float* __restrict__ st_,
                               const float* __restrict__ si, size_t n, float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = xt[i] - (st_[i] - si[i]);
}

cudaError_t launch_exact_target(const float* xt, const float* s_tgt, const float* s_in, size_t n,
                                float* out, cudaStream_t st) {
  unsigned g = nblocks(n, 256);
  if (g > 152u * 16) g = 152u * 16;
  k_exact_target<<<g, 256, 0, st>>>(xt, s_tgt, s_in, n, out);
  N2F_LAUNCH_CHECK();
}

// Maximum projection along Z of independently denoised slices (Methods, fluorescence
// microscopy). vol: Z planes of n floats; four pixels per thread when n and both pointers
// allow 16-byte accesses. Exact (a comparison, no rounding).
__global__ void k_max_project4(const float4* __restrict__ vol, int Z, size_t n4,
                               float4* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x) {
    float4 m = vol[i];
    for (int z = 1; z < Z; ++z) {
      const float4 v = vol[(size_t)z * n4 + i];
      m.x = v.x > m.x ? v.x : m.x;
      m.y = v.y > m.y ? v.y : m.y;
      m.z = v.z > m.z ? v.z : m.z;
      m.w = v.w > m.w ? v.w : m.w;
    }
    out[i] = m;
  }
}

__global__ void k_max_project1(const float* __restrict__ vol, int Z, size_t n,
                               float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float m = vol[i];
    for (int z = 1; z < Z; ++z) {
      const float v = vol[(size_t)z * n + i];
      m = v > m ? v : m;
    }
    out[i] = m;
  }
}

cudaError_t launch_max_project(const float* vol, int Z, size_t n, float* out, cudaStream_t st) {
  const bool v4 = n % 4 == 0 && ((uintptr_t)vol % 16) == 0 && ((uintptr_t)out % 16) == 0;
  const size_t m = v4 ? n / 4 : n;
  unsigned g = nblocks(m, 256);
  if (g > 152u * 8) g = 152u * 8;
  if (v4)
    k_max_project4<<<g, 256, 0, st>>>((const float4*)vol, Z, m, (float4*)out);
  else
    k_max_project1<<<g, 256, 0, st>>>(vol, Z, n, out);
  N2F_LAUNCH_CHECK();
}

__global__ void k_u16(const uint16_t* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i] / 65535.0f;
}

cudaError_t launch_u16_to_f32(const uint16_t* in, float* out, size_t n, cudaStream_t st) {
  unsigned g = nblocks(n, 256);
  if (g > 152u * 16) g = 152u * 16;
  k_u16<<<g, 256, 0, st>>>(in, out, n);
  N2F_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------------------------
// Initial weights: element k of the flat vector is U(-1/sqrt(fan_in), +1/sqrt(fan_in)) drawn
// from output k of SplitMix64 (Steele, Lea & Flood 2014), rounded to float32. Only exact IEEE
// double operations are used, so the values equal any other correct implementation's.
struct InitArgs {
  unsigned long long seg_end[kLayers + 1];  // first index after layer l (weights + bias)
  double bound[kLayers + 1];
  unsigned long long count, seed;
};

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_init(float* __restrict__ theta, InitArgs a) {
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       k < a.count; k += (unsigned long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (l < kLayers && k >= a.seg_end[l]) ++l;
    const double u = (double)(splitmix64_at(a.seed, k) >> 11) * 0x1.0p-53;
    const double v = __dmul_rn(__dsub_rn(__dmul_rn(2.0, u), 1.0), a.bound[l]);
    theta[k] = __double2float_rn(v);
  }
}

cudaError_t launch_init_params(float* theta, const NetShape& net, uint64_t seed, cudaStream_t st) {
  InitArgs a;
  int cin = net.c0;
  for (int l = 0; l <= kLayers; ++l) {
    const int fan = l < kLayers ? cin * 9 : cin;
    a.bound[l] = 1.0 / sqrt((double)fan);
    a.seg_end[l] = l < kLayers ? net.w_off[l + 1] : net.count;
    if (l < kLayers) cin = net.widths[l];
  }
  a.count = net.count;
  a.seed = seed;
  unsigned g = nblocks(net.count, 256);
  if (g > 152u * 8) g = 152u * 8;
  k_init<<<g, 256, 0, st>>>(theta, a);
  N2F_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------------------------
// Writes weight W[o][c][tap] of one layer into every operand copy that is present:
//   SIMT forward  [C_in/8][tap][8][C_out]   (first layer: canonical [C_out][C_0][9])
//   SIMT dgrad    [C_out/8][8 - tap][8][C_in]
//   tensor core   tc_layout.cuh order, forward (rows o, k = tap*C_in + c) and dgrad
//                 (rows c, k = (8 - tap)*C_out + o); bf16, or (float32 form) the fp16 hi and lo
//                 parts of th * s, s the layer's power-of-two weight scale.
__device__ __forceinline__ void pack_one(float* fwd, float* dgr, void* tcf, void* tcd,
                                         void* tcf_lo, void* tcd_lo, int tc_bf16, int first,
                                         int cin, int cout, int o, int c, int tap, float th,
                                         float s) {
  if (first) {
    if (fwd) fwd[((size_t)o * cin + c) * 9 + tap] = th;
    return;
  }
  if (fwd) fwd[(((size_t)(c >> 3) * 9 + tap) * 8 + (c & 7)) * cout + o] = th;
  if (dgr) dgr[(((size_t)(o >> 3) * 9 + (8 - tap)) * 8 + (o & 7)) * cin + c] = th;
  if (tcf) {
    const size_t fi = tc_index_cfg(tc_cfg(cin, cout, tc_bf16), cin, o, tap, c);
    const size_t di = tc_index_cfg(tc_cfg(cout, cin, tc_bf16), cout, c, 8 - tap, o);
    const size_t nw = (size_t)cin * cout * 9;
    if (!N2F_IN(fi, nw) || !N2F_IN(di, nw)) return;
    if (tc_bf16) {
      ((__nv_bfloat16*)tcf)[fi] = __float2bfloat16_rn(th);
      ((__nv_bfloat16*)tcd)[di] = __float2bfloat16_rn(th);
    } else {
      const float x = th * s;
      const __half hi = __float2half_rn(x);
      const __half lo = __float2half_rn(x - __half2float(hi));
      ((__half*)tcf)[fi] = hi;
      ((__half*)tcf_lo)[fi] = lo;
      ((__half*)tcd)[di] = hi;
      ((__half*)tcd_lo)[di] = lo;
    }
  }
}

// Layer of parameter i and whether it is a 3x3 weight (not a bias or the head).
__device__ __forceinline__ int weight_layer(const PackArgs& pa, unsigned long long i) {
  int l = 0;
  while (l < kLayers && i >= pa.w_off[l + 1]) ++l;
  return (l == kLayers || i >= pa.b_off[l]) ? -1 : l;
}

// Weight i (of layer l) into its SIMT copies and / or its tensor-core copies.
__device__ __forceinline__ void pack_param(const PackArgs& pa, int l, unsigned long long i,
                                           float th, bool simt, bool tc, float s) {
  const int cin = l == 0 ? pa.c0 : pa.widths[l - 1], cout = pa.widths[l];
  // 32-bit: a layer holds at most 256 x 256 x 9 weights
  const unsigned j = (unsigned)(i - pa.w_off[l]), cin9 = (unsigned)cin * 9u;
  const int o = (int)(j / cin9);
  const int rem = (int)(j - (unsigned)o * cin9);
  pack_one(simt ? pa.fwd[l] : nullptr, simt ? pa.dgr[l] : nullptr, tc ? pa.tcf[l] : nullptr,
           pa.tcd[l], pa.tcf_lo[l], pa.tcd_lo[l], pa.tc_bf16, l == 0, cin, cout, o, rem / 9,
           rem % 9, th, s);
}

// Adam (Kingma & Ba, Algorithm 1; Methods: lr 0.001), fused with writing the CUDA-core weight
// copies (the layers that have them). update = 0 only packs (after init / set_theta). The
// tensor-core copies follow in k_pack_tc; in the float32 form they need each layer's largest
// weight first: this kernel collects it (pa.sw->wnew, by step parity); it also clears the
// activation and delta words for the next pass and the other parity's weight words.
__global__ void k_adam(PackArgs pa, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, AdamConsts k, const DevState* __restrict__ state,
                       int update) {
  if (update && state->stopped) return;
  __shared__ unsigned smax[kLayers];
  ScaleWords* sw = pa.sw;
  if (threadIdx.x < kLayers) smax[threadIdx.x] = 0u;
  __syncthreads();
  float bc1 = 1.f, bc2 = 1.f;
  if (update) {
    bc1 = state->bc1;
    bc2 = state->bc2;
  }
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i0 = blockIdx.x * (unsigned long long)blockDim.x; i0 < pa.count;
       i0 += stride) {
    const unsigned long long i = i0 + threadIdx.x;
    int lw = -1;  // tensor-core layer of a float32-form weight
    float aw = 0.f;
    if (i < pa.count) {
      float th = pa.theta[i];
      if (update) {
        const float g = grad[i];
        const float mi = k.b1 * m[i] + k.omb1 * g;
        const float vi = k.b2 * v[i] + k.omb2 * g * g;
        m[i] = mi;
        v[i] = vi;
        th -= k.lr * (mi / bc1) / (sqrtf(vi / bc2) + k.eps);
        pa.theta[i] = th;
      }
      const int l = weight_layer(pa, i);
      if (l >= 0) {
        pack_param(pa, l, i, th, true, false, 1.f);  // tensor-core copies: k_pack_tc
        if (pa.tcf[l] && sw) {
          lw = l;
          aw = fabsf(th);
        }
      }
    }
    if (sw) {  // one shared-memory atomic per warp when its lanes share a layer
      const unsigned b = __float_as_uint(aw);
      const int l0 = __shfl_sync(0xffffffffu, lw, 0);
      if (__all_sync(0xffffffffu, lw == l0)) {
        const unsigned mx = __reduce_max_sync(0xffffffffu, b);
        if ((threadIdx.x & 31) == 0 && l0 >= 0) atomicMax(&smax[l0], mx);
      } else if (lw >= 0) {
        atomicMax(&smax[lw], b);
      }
    }
  }
  if (!sw) return;
  __syncthreads();
  const int slot = state->t & 1;
  if (threadIdx.x < kLayers && smax[threadIdx.x]) atomicMax(&sw->wnew[slot][threadIdx.x], smax[threadIdx.x]);
  if (blockIdx.x == 0 && threadIdx.x < kLayers) {
    sw->wnew[slot ^ 1][threadIdx.x] = 0u;
    sw->act[threadIdx.x] = 0u;
    sw->delta[threadIdx.x] = 0u;
  }
}

// The tensor-core copies of every tensor-core layer (bf16; float32 form: fp16 hi / lo parts
// scaled by the power of two that the layer's largest weight, collected by k_adam, gives), for
// the forward (rows o, K = tap x C_in + c) and the dgrad (rows c, K = (8 - tap) x C_out + o).
// A block packs one tile of 32 rows for one 16-channel K chunk: it reads the weights
// those rows need, contiguous in theta ([o][c][tap]), into shared memory, then writes each
// (tap, 8-channel slab) run of the packed stage, 8 x rows contiguous elements, in order, so
// both its reads and its writes are coalesced (element by element in theta order the packed
// positions scatter: one store per sector). Block 0 also records the largest weights in sw->w
// for the convolution kernels.
struct PackTcPlan {
  int start[2 * kLayers + 1];  // first block of (layer l, direction d) at 2 l + d
};

constexpr int kPackRows = 32;  // rows per k_pack_tc block (every tensor-core layer has >= 32)

__global__ void __launch_bounds__(256) k_pack_tc(PackArgs pa, PackTcPlan plan,
                                                 const DevState* __restrict__ state, int update) {
  if (update && state->stopped) return;
  constexpr int TR = kPackRows, N = 16 * TR * 9, PER = N / 256;
  __shared__ float buf[N];
  ScaleWords* sw = pa.sw;
  const int slot = state->t & 1;
  if (sw && blockIdx.x == 0 && threadIdx.x < kLayers) sw->w[threadIdx.x] = sw->wnew[slot][threadIdx.x];
  int q = 0;
  while (q < 2 * kLayers && (int)blockIdx.x >= plan.start[q + 1]) ++q;
  const int l = q >> 1, dir = q & 1;
  const int cin = l == 0 ? pa.c0 : pa.widths[l - 1], cout = pa.widths[l];
  const int Kc = dir ? cout : cin;  // K-side channels
  const int NT = dir ? tc_cfg(cout, cin, pa.tc_bf16).NT : tc_cfg(cin, cout, pa.tc_bf16).NT;
  const int nchunks = Kc / 16;
  const int b = (int)blockIdx.x - plan.start[q];
  const int tile = b / nchunks, chunk = b - tile * nchunks;
  const int r0 = tile * TR, nt = r0 / NT, rr0 = r0 % NT;
  const float* th = pa.theta + pa.w_off[l];
  float s = 1.f;
  if (!pa.tc_bf16) s = pow2f(f16_scale_exp(sw->wnew[slot][l]));
  // theta[o][c][tap]: forward, rows o = r0.., channels c = 16 chunk..: 144 floats per row;
  // dgrad, rows c = r0.., channels o = 16 chunk..: TR x 9 floats per channel o
  float v[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {  // all loads in flight before any store
    const int u = threadIdx.x + 256 * k;
    if (!dir) {
      const int rl = u / 144, j = u - rl * 144;
      v[k] = th[((size_t)(r0 + rl) * cin + chunk * 16) * 9 + j];
    } else {
      const int ol = u / (TR * 9), j = u - ol * (TR * 9);
      v[k] = th[((size_t)(chunk * 16 + ol) * cin + r0) * 9 + j];
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) buf[threadIdx.x + 256 * k] = v[k];
  __syncthreads();
  void* dhi = dir ? pa.tcd[l] : pa.tcf[l];
  void* dlo = dir ? pa.tcd_lo[l] : pa.tcf_lo[l];
  const size_t stage = (size_t)nt * nchunks + chunk;
  const size_t nw = (size_t)cin * cout * 9;
  (void)nw;  // the checked build's bound
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    // u = ((tap x 2 + slab) x TR + rl) x 8 + e: the stage's element order within this tile
    const int u = threadIdx.x + 256 * k;
    const int e = u & 7, rl = (u >> 3) % TR, ts = (u >> 3) / TR, slab = ts & 1, tap = ts >> 1;
    const int kc = slab * 8 + e;  // K-side channel within the chunk
    const float x0 = !dir ? buf[rl * 144 + kc * 9 + tap] : buf[kc * (TR * 9) + rl * 9 + (8 - tap)];
    const size_t idx = (((stage * 9 + tap) * 2 + slab) * NT + rr0 + rl) * 8 + e;
    if (!N2F_IN(idx, nw)) continue;
    if (pa.tc_bf16) {
      ((__nv_bfloat16*)dhi)[idx] = __float2bfloat16_rn(x0);
    } else {
      const float x = x0 * s;
      const __half hi = __float2half_rn(x);
      ((__half*)dhi)[idx] = hi;
      ((__half*)dlo)[idx] = __float2half_rn(x - __half2float(hi));
    }
  }
}

// Packs one canonical [C_out][C_in][3][3] weight tensor into the kernels' operand copies
// (float32 form: scaled by the largest weight, *wmax).
__global__ void k_pack_layer(const float* __restrict__ w, int cin, int cout, float* fwd,
                             float* dgr, void* tcf, void* tcd, void* tcf_lo, void* tcd_lo,
                             int tc_bf16, const unsigned* wmax) {
  const size_t n = (size_t)cout * cin * 9;
  const float s = (tc_bf16 || !wmax) ? 1.f : f16_scale(wmax);
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
       j += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(j / ((size_t)cin * 9));
    const int rem = (int)(j % ((size_t)cin * 9));
    pack_one(fwd, dgr, tcf, tcd, tcf_lo, tcd_lo, tc_bf16, cin == 1, cin, cout, o, rem / 9,
             rem % 9, w[j], s);
  }
}

template <typename T>
__global__ void k_absmax(const T* __restrict__ x, size_t n, unsigned* out, const int* skip) {
  if (skip && *skip) return;
  float mx = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    mx = fmaxf(mx, fabsf((float)x[i]));
  warp_absmax_to(mx, out);
}

cudaError_t launch_absmax(const void* x, size_t n, int bf16, unsigned* out, const int* skip,
                          cudaStream_t st) {
  unsigned g = nblocks(n, 256);
  if (g > 152u * 4) g = 152u * 4;
  if (g == 0) g = 1;
  if (bf16)
    k_absmax<__nv_bfloat16><<<g, 256, 0, st>>>((const __nv_bfloat16*)x, n, out, skip);
  else
    k_absmax<float><<<g, 256, 0, st>>>((const float*)x, n, out, skip);
  N2F_LAUNCH_CHECK();
}

cudaError_t launch_pack_layer(const float* w, int cin, int cout, float* fwd, float* dgr, void* tcf,
                              void* tcd, void* tcf_lo, void* tcd_lo, int tc_bf16, unsigned* wmax,
                              cudaStream_t st) {
  const size_t n = (size_t)cout * cin * 9;
  if (tcf && !tc_bf16) {
    if (!wmax) return cudaErrorInvalidValue;
    const cudaError_t e = launch_absmax(w, n, 0, wmax, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  unsigned g = nblocks(n, 256);
  if (g > 152u * 8) g = 152u * 8;
  k_pack_layer<<<g, 256, 0, st>>>(w, cin, cout, fwd, dgr, tcf, tcd, tcf_lo, tcd_lo, tc_bf16, wmax);
  N2F_LAUNCH_CHECK();
}

AdamConsts adam_consts(double lr, double b1, double b2, double eps) {
  AdamConsts k;
  k.lr = (float)lr;
  k.b1 = (float)b1;
  k.omb1 = (float)(1.0 - b1);  // formed in double: 1 - float(b) would round b first
  k.b2 = (float)b2;
  k.omb2 = (float)(1.0 - b2);
  k.eps = (float)eps;
  return k;
}

cudaError_t launch_adam(const PackArgs& pa, const float* grad, float* m, float* v,
                        const AdamConsts& k, const DevState* state, int update, cudaStream_t st) {
  unsigned g = nblocks(pa.count, 256);
  if (g > 152u * 8) g = 152u * 8;
  k_adam<<<g, 256, 0, st>>>(pa, grad, m, v, k, state, update);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the tensor-core copies: blocks of (layer, direction) = row tiles of 32 x K chunks of 16
  PackTcPlan plan;
  int nb = 0;
  for (int l = 0; l < kLayers; ++l)
    for (int d = 0; d < 2; ++d) {
      plan.start[2 * l + d] = nb;
      if (!pa.tcf[l]) continue;
      const int cin = l == 0 ? pa.c0 : pa.widths[l - 1], cout = pa.widths[l];
      const int R = d ? cin : cout, Kc = d ? cout : cin;
      if (R % kPackRows || Kc % 16) return cudaErrorInvalidValue;
      nb += (R / kPackRows) * (Kc / 16);
    }
  plan.start[2 * kLayers] = nb;
  if (nb == 0) return cudaSuccess;
  k_pack_tc<<<nb, 256, 0, st>>>(pa, plan, state, update);
  N2F_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------------------------
// NCHW float <-> CG layout.
template <typename T>
__global__ void k_pack_cg(const float* __restrict__ src, int C, size_t npx, T* __restrict__ dst) {
  constexpr int G = CGTraits<T>::G;
  const size_t n = (size_t)C * npx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / npx);
    const size_t p = i % npx;
    const size_t di = ((size_t)(c / G) * npx + p) * G + (c % G);
    if (N2F_IN(di, n)) dst[di] = CGTraits<T>::from_float(src[i]);
  }
}

template <typename T, typename D>
__global__ void k_unpack_cg(const T* __restrict__ src, int C, size_t npx, D* __restrict__ dst) {
  constexpr int G = CGTraits<T>::G;
  const size_t n = (size_t)C * npx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / npx);
    const size_t p = i % npx;
    const size_t si = ((size_t)(c / G) * npx + p) * G + (c % G);
    if (N2F_IN(si, n)) dst[i] = (D)CGTraits<T>::to_float(src[si]);
  }
}

cudaError_t launch_pack_cg(const float* nchw, int C, int H, int W, int bf16, void* cg,
                           cudaStream_t st) {
  const size_t npx = (size_t)H * W;
  unsigned g = nblocks((size_t)C * npx, 256);
  if (g > 152u * 16) g = 152u * 16;
  if (bf16)
    k_pack_cg<__nv_bfloat16><<<g, 256, 0, st>>>(nchw, C, npx, (__nv_bfloat16*)cg);
  else
    k_pack_cg<float><<<g, 256, 0, st>>>(nchw, C, npx, (float*)cg);
  N2F_LAUNCH_CHECK();
}

cudaError_t launch_unpack_cg(const void* cg, int C, int H, int W, int bf16, float* nchw,
                             cudaStream_t st) {
  const size_t npx = (size_t)H * W;
  unsigned g = nblocks((size_t)C * npx, 256);
  if (g > 152u * 16) g = 152u * 16;
  if (bf16)
    k_unpack_cg<__nv_bfloat16, float><<<g, 256, 0, st>>>((const __nv_bfloat16*)cg, C, npx, nchw);
  else
    k_unpack_cg<float, float><<<g, 256, 0, st>>>((const float*)cg, C, npx, nchw);
  N2F_LAUNCH_CHECK();
}

cudaError_t launch_unpack_cg_f64(const void* cg, int C, int H, int W, int bf16, double* out,
                                 cudaStream_t st) {
  const size_t npx = (size_t)H * W;
  unsigned g = nblocks((size_t)C * npx, 256);
  if (g > 152u * 16) g = 152u * 16;
  if (bf16)
    k_unpack_cg<__nv_bfloat16, double><<<g, 256, 0, st>>>((const __nv_bfloat16*)cg, C, npx, out);
  else
    k_unpack_cg<float, double><<<g, 256, 0, st>>>((const float*)cg, C, npx, out);
  N2F_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------------------------
// First layer, C_0 <= 4 input planes (Methods: the first 3x3 convolution sees the image; Fig.
// 2a caption: the input may be multi-channel). One thread per pixel: 9 C_0 taps from the
// planes (zero outside), C outputs + bias, ReLU.
template <typename T, int C0>
__device__ __forceinline__ void conv1_pixel(const float* __restrict__ img, int H, int W,
                                            const float* sw, const float* sb, int C,
                                            T* __restrict__ out, size_t p, float& mx) {
  constexpr int G = CGTraits<T>::G;
  const size_t npx = (size_t)H * W;
  const int y = (int)(p / W), x = (int)(p % W);
  float t[C0][9];
#pragma unroll
  for (int c = 0; c < C0; ++c)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int yy = y + ky - 1, xx = x + kx - 1;
        t[c][ky * 3 + kx] = (yy >= 0 && yy < H && xx >= 0 && xx < W)
                                ? img[(size_t)c * npx + (size_t)yy * W + xx]
                                : 0.f;
      }
  for (int g = 0; g < C / G; ++g) {
    float v[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int o = g * G + k;
      float s = sb[o];
#pragma unroll
      for (int c = 0; c < C0; ++c)
#pragma unroll
        for (int q = 0; q < 9; ++q) s += sw[(o * C0 + c) * 9 + q] * t[c][q];
      v[k] = s > 0.f ? s : 0.f;
      mx = fmaxf(mx, v[k]);
    }
    if (N2F_IN((size_t)g * npx + p, (size_t)(C / G) * npx)) store_group<T>(out, (size_t)g * npx + p, v);
  }
}

template <typename T, int C0>
__global__ void __launch_bounds__(256) k_conv1_fwd(const float* __restrict__ img, int H, int W,
                                                   const float* __restrict__ w,
                                                   const float* __restrict__ b, int C,
                                                   T* __restrict__ out, unsigned* amax,
                                                   const int* skip) {
  if (skip && *skip) return;
  __shared__ float sw[64 * C0 * 9], sb[64];
  for (int i = threadIdx.x; i < C * C0 * 9; i += blockDim.x) sw[i] = w[i];
  for (int i = threadIdx.x; i < C; i += blockDim.x) sb[i] = b[i];
  __syncthreads();
  const size_t npx = (size_t)H * W;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  float mx = 0.f;  // largest output of this thread (ReLU outputs are >= 0)
  if (p < npx) conv1_pixel<T, C0>(img, H, W, sw, sb, C, out, p, mx);
  if (amax) block_absmax_to(mx, amax);
}

template <typename T>
static void conv1_fwd_c0(int C0, unsigned g, const float* img, int H, int W, const float* w,
                         const float* b, int C, T* out, unsigned* amax, const int* skip,
                         cudaStream_t st) {
  switch (C0) {
    case 1: k_conv1_fwd<T, 1><<<g, 256, 0, st>>>(img, H, W, w, b, C, out, amax, skip); break;
    case 2: k_conv1_fwd<T, 2><<<g, 256, 0, st>>>(img, H, W, w, b, C, out, amax, skip); break;
    case 3: k_conv1_fwd<T, 3><<<g, 256, 0, st>>>(img, H, W, w, b, C, out, amax, skip); break;
    default: k_conv1_fwd<T, 4><<<g, 256, 0, st>>>(img, H, W, w, b, C, out, amax, skip); break;
  }
}

cudaError_t launch_conv1_fwd(const float* img, int C0, int H, int W, const float* w,
                             const float* b, int C, int bf16, void* out, unsigned* amax,
                             const int* skip, cudaStream_t st) {
  if (C > 64 || C0 < 1 || C0 > kMaxC0) return cudaErrorInvalidValue;
  const size_t npx = (size_t)H * W;
  if (bf16)
    conv1_fwd_c0<__nv_bfloat16>(C0, nblocks(npx, 256), img, H, W, w, b, C, (__nv_bfloat16*)out,
                                nullptr, skip, st);
  else
    conv1_fwd_c0<float>(C0, nblocks(npx, 256), img, H, W, w, b, C, (float*)out, amax, skip, st);
  N2F_LAUNCH_CHECK();
}

// First-layer weight gradient: dW[o][c][tap] = sum_p d(p,o) x_c(p + tap), db[o] = sum_p d(p,o).
// Block s sums pixel tiles s, s+S, ... in order; the partials are reduced in block order.
// First-layer weight and bias gradients, per block over a strided set of 64-pixel tiles: the
// tile's delta (C channels) and the K = C_0 x 9 shifted input values of each pixel are staged
// in shared memory; each thread owns a register tile of 4 output channels x 3 of the K values
// (or x the constant 1 for the biases) and runs over its share of the tile's pixels (pixel
// groups pg, pg + npg, ...), so one 16-byte load of delta feeds up to twelve FMAs. At the end
// the pixel groups' sums are added in group order and the block writes its partial row
// part[blockIdx][q], q = o K + c x 9 + tap, then the C biases.
template <typename T>
__global__ void __launch_bounds__(256) k_conv1_wgrad(const T* __restrict__ dout,
                                                     const float* __restrict__ img, int C0, int H,
                                                     int W, int C, float* __restrict__ part,
                                                     size_t part_cap, const int* skip) {
  if (skip && *skip) return;
  constexpr int G = CGTraits<T>::G;
  constexpr int TP = 64, DP = 68;  // pixels per tile; delta row pitch (16-byte aligned rows)
  __shared__ __align__(16) float sD[TP * DP];
  __shared__ float sX[TP][kMaxC0 * 9 + 1];
  const size_t npx = (size_t)H * W;
  const int K = C0 * 9;
  const int Q = C * (K + 1);  // (o, c, tap) triples then the C biases
  const int ncg = K / 3 + 1, nslot = (C / 4) * ncg, npg = 256 / nslot;
  const int t = threadIdx.x, slot = t % nslot, pg = t / nslot;
  const bool act = pg < npg;
  const int og = slot / ncg, cg = slot - og * ncg;
  const bool bias = cg == ncg - 1;
  float acc[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[i][j] = 0.f;
  const size_t ntiles = (npx + TP - 1) / TP;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t p0 = tile * TP;
    __syncthreads();
    for (int i = t; i < TP * (C / G); i += blockDim.x) {
      const int pp = i % TP, g = i / TP;
      const size_t p = p0 + pp;
      float v[G];
      if (p < npx) {
        load_group<T>(dout, (size_t)g * npx + p, v);
      } else {
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < G; k += 4)
        *reinterpret_cast<float4*>(&sD[pp * DP + g * G + k]) =
            make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    }
    for (int i = t; i < TP * K; i += blockDim.x) {
      const int pp = i / K, cq = i % K, c = cq / 9, q = cq % 9;
      const size_t p = p0 + pp;
      float v = 0.f;
      if (p < npx) {
        // 32-bit division: images hold fewer than 2^31 pixels
        const unsigned p32 = (unsigned)p, yq = p32 / (unsigned)W;
        const int y = (int)yq + q / 3 - 1, x = (int)(p32 - yq * (unsigned)W) + q % 3 - 1;
        if (y >= 0 && y < H && x >= 0 && x < W) v = img[(size_t)c * npx + (size_t)y * W + x];
      }
      sX[pp][cq] = v;
    }
    __syncthreads();
    if (act) {
      for (int pp = pg; pp < TP; pp += npg) {
        const float4 d = *reinterpret_cast<const float4*>(&sD[pp * DP + og * 4]);
        const float dv[4] = {d.x, d.y, d.z, d.w};
        float xv[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) xv[j] = bias ? (j == 0 ? 1.f : 0.f) : sX[pp][cg * 3 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) acc[i][j] += dv[i] * xv[j];
      }
    }
  }
  // the pixel groups' sums, added in group order (sD reused: npg x Q <= 2816 floats)
  __syncthreads();
  float* red = sD;
  if (act) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = og * 4 + i;
      if (bias) {
        red[pg * Q + C * K + o] = acc[i][0];
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) red[pg * Q + o * K + cg * 3 + j] = acc[i][j];
      }
    }
  }
  __syncthreads();
  for (int q = t; q < Q; q += blockDim.x) {
    float sum = 0.f;
    for (int g2 = 0; g2 < npg; ++g2) sum += red[g2 * Q + q];
    if (N2F_IN((size_t)blockIdx.x * Q + q, part_cap)) part[(size_t)blockIdx.x * Q + q] = sum;
  }
}

// out[q] = sum over s of part[s * Q + q], canonical placement of dW and db. A block owns 32
// consecutive q (the lanes); warp w sums s = w, w + 32, ... in order and the 32 warp sums are
// added in warp order, so the result is fixed for a given S (Q is a few hundred: few blocks,
// so each warp's chain of loads is kept short).
__global__ void __launch_bounds__(1024) k_reduce_conv1(const float* __restrict__ part, int S,
                                                       int C, int K, float* __restrict__ gw,
                                                       float* __restrict__ gb, const int* skip) {
  if (skip && *skip) return;
  constexpr int NW = 32;  // warps: a short chain of loads each (Q is small, few blocks)
  __shared__ float sh[NW][33];
  const int Q = C * (K + 1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (q < Q) {
    int k = w;
    for (; k + 3 * NW < S; k += 4 * NW) {  // four loads in flight, added in split order
      const float a = part[(size_t)k * Q + q], b = part[(size_t)(k + NW) * Q + q];
      const float c = part[(size_t)(k + 2 * NW) * Q + q], d = part[(size_t)(k + 3 * NW) * Q + q];
      s = (((s + a) + b) + c) + d;
    }
    for (; k < S; k += NW) s += part[(size_t)k * Q + q];
  }
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0 && q < Q) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += sh[k][lane];
    if (q < C * K)
      gw[q] = t;  // [o][c][ky][kx] == (o * C0 + c) * 9 + tap
    else
      gb[q - C * K] = t;
  }
}

cudaError_t launch_conv1_wgrad(const void* dout, const float* img, int C0, int H, int W, int C,
                               int bf16, float* part, size_t part_cap, float* gw, float* gb,
                               const int* skip, cudaStream_t st) {
  if (C > 64 || C0 < 1 || C0 > kMaxC0) return cudaErrorInvalidValue;
  const size_t npx = (size_t)H * W;
  const int K = C0 * 9, Q = C * (K + 1);
  int S = (int)((npx + 127) / 128);
  if (S > 608) S = 608;  // four blocks per SM: more loads in flight than two
  if ((size_t)S * Q > part_cap) S = (int)(part_cap / Q);
  if (S < 1) return cudaErrorInvalidValue;
  if (bf16)
    k_conv1_wgrad<__nv_bfloat16><<<S, 256, 0, st>>>((const __nv_bfloat16*)dout, img, C0, H, W,
                                                    C, part, part_cap, skip);
  else
    k_conv1_wgrad<float><<<S, 256, 0, st>>>((const float*)dout, img, C0, H, W, C, part, part_cap,
                                            skip);
  count_launch();
  k_reduce_conv1<<<nblocks(Q, 32), 1024, 0, st>>>(part, S, C, K, gw, gb, skip);
  N2F_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------------------------
// Head, training step (Methods: 1x1 convolution, sigmoid, BCE loss against the target).
// Per pixel z = b + w . a8, dL/dz = (sigmoid(z) - y) / P away from the -100 clamps of the BCE
// log terms (MSE alternative: 2 (s - y) s (1 - s) / P), delta_8 = dL/dz * w * [a8 > 0]; per
// block of 256 pixels the partial sums of dL/dz * a8 (head weight gradient), dL/dz (head bias)
// and the loss (FP64).
__device__ __forceinline__ float sigmoid_f(float z) {
  if (z >= 0.f) return 1.f / (1.f + expf(-z));
  const float e = expf(z);
  return e / (1.f + e);
}

// Unpacks a 16-byte group (G channels) held in a register.
template <typename T>
__device__ __forceinline__ void unpack_group(const uint4 q, float* v);
template <>
__device__ __forceinline__ void unpack_group<float>(const uint4 q, float* v) {
  v[0] = __uint_as_float(q.x); v[1] = __uint_as_float(q.y);
  v[2] = __uint_as_float(q.z); v[3] = __uint_as_float(q.w);
}
template <>
__device__ __forceinline__ void unpack_group<__nv_bfloat16>(const uint4 q, float* v) {
  const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// One read of the layer-8 map: a block takes 256 pixels as eight sub-tiles of 32, each staged
// in shared memory ([C/G][33] 16-byte groups, one pad group per row), from which it computes
// z (eight threads per pixel, a fixed butterfly over their partial sums), dL/dz, the
// head-gradient sums (thread c: channel c over the pixels in order) and delta_8 (stored group
// by group, coalesced). Reading the map once instead of twice (z, then delta_8) halves its
// traffic.
constexpr int kHeadTP = 32;  // pixels per sub-tile
constexpr int kHeadSub = 8;  // sub-tiles per block: 256 pixels, one row of head partials

template <typename T>
__global__ void __launch_bounds__(256, 4) k_head_train(const T* __restrict__ a8, int C, int npx,
                                                    const float* __restrict__ w9,
                                                    const float* __restrict__ b9,
                                                    const float* __restrict__ tgt, int loss_kind,
                                                    float* __restrict__ dzbuf, T* __restrict__ d8,
                                                    unsigned* dmax, double* __restrict__ loss_part,
                                                    float* __restrict__ hpart, const int* skip) {
  if (skip && *skip) return;
  constexpr int G = CGTraits<T>::G;
  constexpr int PITCH = kHeadTP + 1;
  constexpr int kTpp = 256 / kHeadTP;  // threads per pixel for z
  __shared__ uint4 tile[(256 / G) * PITCH];
  __shared__ float sw[256];
  __shared__ float sdz[kHeadTP];
  __shared__ double sl[8];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ng = C / G;
  for (int i = t; i < C; i += blockDim.x) sw[i] = w9[i];
  const float bias = b9[0];
  float acc = 0.f;     // thread c < C: sum of dL/dz * a8[c] over the block's pixels
  float dzsum = 0.f;   // thread C (or 0 when C = 256, after its channel): sum of dL/dz
  double lsum = 0.0;   // loss terms of the pixels this thread scored
  float dmx = 0.f;     // largest |delta_8| this thread stored
  // unsigned: the last block may reach past 2^31 - 1 when npx is close to it
  const unsigned pb = blockIdx.x * (unsigned)(kHeadTP * kHeadSub);
  // a thread's groups of a sub-tile (units u = t + 256 i), loaded one sub-tile ahead
  constexpr int kU = (256 / G) * kHeadTP / 256;
  uint4 nxt[kU];
  auto load_sub = [&](int sub) {
    const unsigned p0 = pb + sub * kHeadTP;
#pragma unroll
    for (int i = 0; i < kU; ++i) {
      const int u = t + 256 * i, g = u / kHeadTP, px = u % kHeadTP;
      nxt[i] = make_uint4(0u, 0u, 0u, 0u);
      if (u < ng * kHeadTP && p0 + px < (unsigned)npx)
        nxt[i] = reinterpret_cast<const uint4*>(a8)[(size_t)g * npx + p0 + px];
    }
  };
  load_sub(0);
  for (int sub = 0; sub < kHeadSub; ++sub) {
    const unsigned p0 = pb + sub * kHeadTP;
#pragma unroll
    for (int i = 0; i < kU; ++i) {
      const int u = t + 256 * i;
      if (u < ng * kHeadTP) tile[(u / kHeadTP) * PITCH + u % kHeadTP] = nxt[i];
    }
    __syncthreads();
    if (sub + 1 < kHeadSub) load_sub(sub + 1);  // in flight while this sub-tile is worked
    {  // z = b + w . a8 and dL/dz for pixel px
      const int px = t / kTpp, q = t % kTpp;
      float z = 0.f;
      for (int g = q; g < ng; g += kTpp) {
        float v[G];
        unpack_group<T>(tile[g * PITCH + px], v);
#pragma unroll
        for (int k = 0; k < G; ++k) z += sw[g * G + k] * v[k];
      }
#pragma unroll
      for (int off = 1; off < kTpp; off <<= 1) z += __shfl_xor_sync(0xffffffffu, z, off);
      z += bias;
      const unsigned p = p0 + px;
      if (q == 0) {
        float dz = 0.f;
        if (p < (unsigned)npx) {
          const float s = sigmoid_f(z), y = tgt[p];
          if (loss_kind == 0) {
            // BCE with each log term clamped at -100 (bounded for unclipped targets outside
            // [0, 1]); log s = -softplus(-z), log(1 - s) = -softplus(z)
            const float sp = log1pf(expf(-fabsf(z)));
            const float lp = -(fmaxf(-z, 0.f) + sp), lq = -(fmaxf(z, 0.f) + sp);
            const bool m1 = lp > -100.f, m2 = lq > -100.f;
            const float gr = (m1 && m2) ? s - y
                                        : (m1 ? -y * (1.f - s) : 0.f) + (m2 ? (1.f - y) * s : 0.f);
            dz = gr / (float)npx;
            lsum += -(double)y * (m1 ? lp : -100.0) - (1.0 - (double)y) * (m2 ? lq : -100.0);
          } else {
            dz = 2.f * (s - y) * s * (1.f - s) / (float)npx;
            lsum += (double)(s - y) * (double)(s - y);
          }
          dzbuf[p] = dz;
        }
        sdz[px] = dz;
      }
    }
    __syncthreads();
    if (t < C) {  // head-weight gradient: channel t, the sub-tile's pixels in order
      // the 32-bit word of the group that holds channel t (bf16: two channels a word, the
      // even one in the low half), read directly
      const int g = t / G, k = t % G;
      const uint32_t* tw =
          reinterpret_cast<const uint32_t*>(tile) + g * PITCH * 4 + (G == 4 ? k : k >> 1);
      const bool hi = G == 8 && (k & 1);
#pragma unroll 8
      for (int px = 0; px < kHeadTP; ++px) {
        const uint32_t w = tw[px * 4];
        const float v =
            G == 4 ? __uint_as_float(w) : __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
        acc += sdz[px] * v;
      }
    }
    if (t == (C < 256 ? C : 0))
      for (int px = 0; px < kHeadTP; ++px) dzsum += sdz[px];
    for (int u = t; u < ng * kHeadTP; u += 256) {  // delta_8 = dL/dz * w * [a8 > 0]
      const int g = u / kHeadTP, px = u % kHeadTP;
      const unsigned p = p0 + px;
      if (p >= (unsigned)npx) continue;
      float v[G], d[G];
      unpack_group<T>(tile[g * PITCH + px], v);
      const float dz = sdz[px];
#pragma unroll
      for (int k = 0; k < G; ++k) {
        d[k] = v[k] > 0.f ? dz * sw[g * G + k] : 0.f;
        dmx = fmaxf(dmx, fabsf(d[k]));
      }
      if (N2F_IN((size_t)g * npx + p, (size_t)ng * npx)) store_group<T>(d8, (size_t)g * npx + p, d);
    }
    __syncthreads();  // the next sub-tile overwrites the tile and sdz
  }
  float* row = hpart + (size_t)blockIdx.x * (C + 1);
  if (t < C) row[t] = acc;
  if (t == (C < 256 ? C : 0)) row[C] = dzsum;
  double l = lsum;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if (lane == 0) sl[warp] = l;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sl[k];
    loss_part[blockIdx.x] = s;
  }
  if (dmax) block_absmax_to(dmx, dmax);
}

cudaError_t launch_head_train(const void* a8, int C, int npx, const float* w9, const float* b9,
                              const float* tgt, int loss_kind, int bf16, float* dz, void* d8,
                              unsigned* dmax, double* loss_part, float* hpart, int* nblk_out,
                              const int* skip, cudaStream_t st) {
  if (C > 256) return cudaErrorInvalidValue;
  const unsigned nb = nblocks(npx, 256);
  *nblk_out = (int)nb;
  if (bf16)
    k_head_train<__nv_bfloat16><<<nb, 256, 0, st>>>((const __nv_bfloat16*)a8, C, npx, w9, b9, tgt,
                                                    loss_kind, dz, (__nv_bfloat16*)d8, nullptr,
                                                    loss_part, hpart, skip);
  else
    k_head_train<float><<<nb, 256, 0, st>>>((const float*)a8, C, npx, w9, b9, tgt, loss_kind, dz,
                                            (float*)d8, dmax, loss_part, hpart, skip);
  N2F_LAUNCH_CHECK();
}

// Loss sum (fixed tree over the per-block partials) and Adam's step counter and bias
// corrections; the head-gradient partials are summed by the column reducer.
// Blocks 0..C: head-gradient column c = sum over the R = nblk partial rows (each thread a fixed
// strided subset in order, then a fixed tree). Block C + 1: the loss (fixed tree over the
// per-block loss partials) and Adam's step counter and bias corrections.
__global__ void k_step_finish(const float* __restrict__ hpart, const double* __restrict__ lpart,
                              int nblk, int C, int npx, float* __restrict__ gw9, DevState* state,
                              double b1, double b2) {
  if (state->stopped) return;
  if ((int)blockIdx.x <= C) {
    __shared__ float shf[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < nblk; r += blockDim.x) s += hpart[(size_t)r * (C + 1) + c];
    shf[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) shf[threadIdx.x] += shf[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) gw9[c] = shf[0];
    return;
  }
  __shared__ double sh[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += lpart[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    state->loss = sh[0] / (double)npx;
    state->t += 1;
    state->b1t *= b1;
    state->b2t *= b2;
    state->bc1 = (float)(1.0 - state->b1t);
    state->bc2 = (float)(1.0 - state->b2t);
  }
}

cudaError_t launch_step_finish(const float* hpart, const double* loss_part, int nblk, int C,
                               int npx, float* gw9, float* gb9, DevState* state, double b1,
                               double b2, cudaStream_t st) {
  // gw9[0..C) and gb9 (= gw9 + C in the flat vector) are the columns of hpart
  if (gb9 != gw9 + C) return cudaErrorInvalidValue;
  k_step_finish<<<C + 2, 256, 0, st>>>(hpart, loss_part, nblk, C, npx, gw9, state, b1, b2);
  N2F_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------------------------
// Validation head (Methods: after each epoch the full noisy image goes through the network
// and the MSE against the noisy image is taken). V = sigmoid(z); (V - x)^2 summed in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_head_val(const T* __restrict__ a8, int C, int npx,
                                                  const float* __restrict__ w9,
                                                  const float* __restrict__ b9,
                                                  const float* __restrict__ x,
                                                  float* __restrict__ V,
                                                  double* __restrict__ mse_part, const int* skip) {
  if (skip && *skip) return;
  constexpr int G = CGTraits<T>::G;
  __shared__ float sw[256];
  __shared__ double sl[8];
  for (int i = threadIdx.x; i < C; i += blockDim.x) sw[i] = w9[i];
  __syncthreads();
  const unsigned p = blockIdx.x * blockDim.x + threadIdx.x;  // see k_head_train
  double e2 = 0.0;
  if (p < (unsigned)npx) {
    float z = b9[0];
    for (int g = 0; g < C / G; ++g) {
      float v[G];
      load_group<T>(a8, (size_t)g * npx + p, v);
#pragma unroll
      for (int k = 0; k < G; ++k) z += sw[g * G + k] * v[k];
    }
    const float s = sigmoid_f(z);
    V[p] = s;
    const double e = (double)s - (double)x[p];
    e2 = e * e;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
  if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sl[k];
    mse_part[blockIdx.x] = s;
  }
}

cudaError_t launch_head_val(const void* a8, int C, int npx, const float* w9, const float* b9,
                            const float* x, int bf16, float* V, double* mse_part, int* nblk_out,
                            const int* skip, cudaStream_t st) {
  if (C > 256) return cudaErrorInvalidValue;
  const unsigned nb = nblocks(npx, 256);
  *nblk_out = (int)nb;
  if (bf16)
    k_head_val<__nv_bfloat16><<<nb, 256, 0, st>>>((const __nv_bfloat16*)a8, C, npx, w9, b9, x, V,
                                                  mse_part, skip);
  else
    k_head_val<float><<<nb, 256, 0, st>>>((const float*)a8, C, npx, w9, b9, x, V, mse_part, skip);
  N2F_LAUNCH_CHECK();
}

// Stop rule (Methods: terminate once one hundred epochs pass without improving the best
// validation score). Strict improvement; the first epoch always sets the best.
__global__ void k_val_decide(const double* __restrict__ part, int nblk, double npx,
                             DevState* state, int fixed_mode, double* __restrict__ hist) {
  __shared__ double sp[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += part[k];
  sp[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (!fixed_mode && state->stopped) {
    state->decision = -1;
    return;
  }
  double tot = 0.0;
  for (int k = 0; k < (int)blockDim.x; ++k) tot += sp[k];
  const double mse = tot / npx;
  state->last_mse = mse;
  if (fixed_mode) {
    state->decision = -1;
    return;
  }
  if (!isfinite(mse)) {
    state->stopped = 3;
    state->decision = -1;
    return;
  }
  state->epoch += 1;
  if (hist) hist[(state->epoch - 1) % kHistCap] = mse;  // the job's validation history
  if (mse < state->best) {
    state->best = mse;
    state->since = 0;
    state->decision = 1;
  } else {
    state->since += 1;
    state->decision = 0;
  }
  if (state->since >= (state->incl_best ? state->patience - 1 : state->patience))
    state->stopped = 1;
  else if (state->max_epochs > 0 && state->epoch >= state->max_epochs)
    state->stopped = 2;
}

cudaError_t launch_val_decide(const double* mse_part, int nblk, size_t npx, DevState* state,
                              int fixed_mode, double* hist, cudaStream_t st) {
  k_val_decide<<<1, 256, 0, st>>>(mse_part, nblk, (double)npx, state, fixed_mode, hist);
  N2F_LAUNCH_CHECK();
}

// Output averaging (Methods: the output is the average of the last one hundred validation
// outputs). The running sum restarts at every new best, so at the stop it holds exactly the
// outputs of the epochs after the best.
__global__ void k_val_accum(const float* __restrict__ V, float* __restrict__ S,
                            float* __restrict__ Vbest, size_t n, const DevState* __restrict__ st) {
  const int d = st->decision;
  if (d < 0) return;
  const int incl = st->incl_best;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = V[i];
    if (d == 1) {
      Vbest[i] = v;
      S[i] = incl ? v : 0.f;
    } else {
      S[i] += v;
    }
  }
}

cudaError_t launch_val_accum(const float* V, float* S, float* Vbest, size_t n,
                             const DevState* state, cudaStream_t st) {
  unsigned g = nblocks(n, 256);
  if (g > 152u * 8) g = 152u * 8;
  k_val_accum<<<g, 256, 0, st>>>(V, S, Vbest, n, state);
  N2F_LAUNCH_CHECK();
}

__global__ void k_result(const float* __restrict__ V, const float* __restrict__ S,
                         const float* __restrict__ Vbest, float* __restrict__ out, size_t n,
                         const DevState* __restrict__ st, int fixed_mode) {
  int mode;  // 0: V, 1: S / cnt, 2: Vbest
  float cnt = 1.f;
  if (fixed_mode) {
    mode = 0;
  } else if (st->stopped == 1) {
    mode = 1;
    cnt = (float)st->patience;
  } else {
    const int c = st->since + (st->incl_best ? 1 : 0);
    mode = c > 0 ? 1 : 2;
    cnt = (float)c;
  }
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = mode == 0 ? V[i] : (mode == 1 ? S[i] / cnt : Vbest[i]);
}

cudaError_t launch_result(const float* V, const float* S, const float* Vbest, float* out, size_t n,
                          const DevState* state, int fixed_mode, cudaStream_t st) {
  unsigned g = nblocks(n, 256);
  if (g > 152u * 8) g = 152u * 8;
  k_result<<<g, 256, 0, st>>>(V, S, Vbest, out, n, state, fixed_mode);
  N2F_LAUNCH_CHECK();
}

// Overlapped validation: when the validation that ran beside an epoch stopped the job, that
// epoch is discarded -- the step counters return to their values at the epoch boundary (the
// weights it changed are not read again: the result comes from the validation outputs), so
// the job ends in the state it would have had with the validation in line.
__global__ void k_step_restore(DevState* __restrict__ state, const DevState* __restrict__ saved) {
  if (threadIdx.x != 0 || !state->stopped) return;
  state->t = saved->t;
  state->b1t = saved->b1t;
  state->b2t = saved->b2t;
  state->bc1 = saved->bc1;
  state->bc2 = saved->bc2;
  state->loss = saved->loss;
}

cudaError_t launch_step_restore(DevState* state, const DevState* saved, cudaStream_t st) {
  k_step_restore<<<1, 32, 0, st>>>(state, saved);
  N2F_LAUNCH_CHECK();
}

N2F_CHECK_READER(check_read_basic)

}  // namespace n2f
