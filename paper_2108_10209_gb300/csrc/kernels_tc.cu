// tcgen05 / TMEM implicit-GEMM kernels for the 3x3 layers with C_in, C_out in {32,...,256}
// (sm_103a). One warp issues TMA copies, one thread issues the MMAs into a TMEM accumulator,
// four warps read TMEM back for the fused epilogue (and, in the 3xTF32 form, split the
// activations into TF32 hi/lo parts in shared memory first).
//
// Forward / dgrad: D[px][n] = sum_{tap, c} A[px + tap][c] B[n][tap, c]: M = 128 pixels of one
//   image row, N = output channels, K = 9 C_in. The A operand of every tap is the same TMA
//   halo tile (3 rows x 130 pixels x a chunk of channels, zero outside the image = the "same"
//   padding) addressed at a shifted start: in the K-major no-swizzle layout each pixel row is
//   16 bytes, so a shift of dx pixels is a 16*dx byte offset of the descriptor.
// Weight gradient: D[o][c] = sum_px delta[px][o] x[px + tap][c] per tap: M = 128 output
//   channels, N = C_in, K = pixels; both operands are read MN-major straight from the
//   channel-grouped maps, split over pixel chunks and reduced in a fixed order.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "cg_util.cuh"
#include "n2f_internal.h"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"
#include "trainer.h"

namespace n2f {

using namespace tc;

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

// ---- forward / dgrad ----------------------------------------------------------------------
struct ConvTcParams {
  const uint8_t* w_hi;  // packed weight stage images (bf16, or the TF32 hi parts)
  const uint8_t* w_lo;  // TF32 residual images (3xTF32 form)
  const float* bias;    // forward
  const void* mask;     // dgrad: the layer's input activation (ReLU mask)
  void* out;
  int cin, cout, H, W, tiles_x;
  int stages;  // pipeline stages, 2 .. kConvMaxStages (a tuning choice; no effect on results)
  const int* skip;
  int* err;
};

// One job of a grouped launch: the same layer of several independent images (each with its
// own weights), their tiles numbered one after the other. The tensor map lives in global
// memory (written by the host before the launch, never by the device).
struct alignas(128) ConvJob {
  CUtensorMap map;
  const uint8_t* w_hi;
  const uint8_t* w_lo;
  const float* bias;
  const void* mask;
  void* out;
  const int* skip;  // the job's stop flag: its tiles are skipped once set
  int H, W, tiles_x, tile0;
};

constexpr int kTileM = 128;   // pixels per accumulator (one image row segment)
constexpr int kRowsM = 2;     // image rows per tile by default: each weight stage feeds two
                              // accumulators (1 is a tuning choice: twice the tiles, half the
                              // accumulator columns, so TMEM double-buffers at N = 256)
constexpr int kHaloX = kTileM + 2;
constexpr int kConvMaxStages = 4;

template <int BF16, int ROWS = kRowsM>
struct ConvCfg {
  static constexpr int GE = BF16 ? 8 : 4;     // channels per 16-byte group
  static constexpr int KC = BF16 ? 16 : 8;    // channels per stage (= one K step of 32 bytes)
  static constexpr int NSLAB = KC / GE;       // 16-byte K slabs per stage (2)
  static constexpr int HALO_Y = ROWS + 2;
  static constexpr uint32_t A_BYTES = NSLAB * HALO_Y * kHaloX * 16;
  static constexpr uint32_t A_SLAB = HALO_Y * kHaloX * 16;  // K distance between halo slabs
  static __host__ __device__ uint32_t b_bytes(int NT) { return 9u * NSLAB * NT * 16; }
  // stage layout: A | A_lo (tf32) | B | B_lo (tf32)
  static __host__ __device__ uint32_t a_lo_off() { return align_up(A_BYTES, 1024); }
  static __host__ __device__ uint32_t b_off() { return BF16 ? align_up(A_BYTES, 1024) : 2 * align_up(A_BYTES, 1024); }
  static __host__ __device__ uint32_t b_lo_off(int NT) { return b_off() + align_up(b_bytes(NT), 1024); }
  static __host__ __device__ uint32_t stage_bytes(int NT) {
    return BF16 ? b_off() + align_up(b_bytes(NT), 1024) : b_lo_off(NT) + align_up(b_bytes(NT), 1024);
  }
};

// Persistent: the grid holds one CTA per resident slot and each CTA takes the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... (a fixed order). The producer streams the stages of
// successive tiles without a break; the accumulators are double-buffered in TMEM when two sets
// fit (2 x kRowsM x N <= 512 columns), so a tile's epilogue overlaps the next tile's MMAs.
// Warp roles: 0 TMA producer, 1 MMA issuer; bf16: 2-9 epilogue (two warps per TMEM lane
// quarter, alternate 16-column blocks); 3xTF32: 2-5 epilogue, 6-9 operand split.
template <int BF16>
struct ConvWarps {
  static constexpr int kThreads = 320;
  static constexpr int kEpi = BF16 ? 8 : 4;  // epilogue warps
};

// What a role needs of the job a tile belongs to.
struct TileJob {
  const CUtensorMap* map;
  const uint8_t* w_hi;
  const uint8_t* w_lo;
  const float* bias;
  const void* mask;
  void* out;
  int H, W, tiles_x, local;
  bool skip;
};

// GROUPED = 0: one image, the tensor map a kernel parameter. GROUPED = 1: the tiles of
// `njobs` images of the same layer shape (p.cin, p.cout), ntiles = p.tiles_x in total; every
// role walks the same tile sequence and skips the tiles of stopped jobs.
template <int BF16, int MODE, int GROUPED, int ROWS>
__global__ void __launch_bounds__(ConvWarps<BF16>::kThreads, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tmA, ConvTcParams p,
              const ConvJob* __restrict__ jobs, int njobs) {
  using C = ConvCfg<BF16, ROWS>;
  using T = typename std::conditional<BF16, __nv_bfloat16, float>::type;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t full[kConvMaxStages], empty[kConvMaxStages], split[kConvMaxStages];
  __shared__ uint64_t accf[2], acce[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  if (!GROUPED && p.skip && *p.skip) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NT = tc_cfg(p.cin, p.cout, BF16).NT;
  const uint32_t B_BYTES = C::b_bytes(NT), SB = C::stage_bytes(NT);
  const int NS = p.stages;
  const int nk = p.cin / C::KC;
  const int ntn = p.cout / NT;
  const int ntiles = GROUPED ? p.tiles_x : p.tiles_x * ((p.H + ROWS - 1) / ROWS) * ntn;
  // tile -> its job; `cur` is the role's cursor (tiles only grow along a role's sequence)
  auto locate = [&](int tile, int& cur) {
    TileJob t;
    if constexpr (!GROUPED) {
      t.map = &tmA;
      t.w_hi = p.w_hi; t.w_lo = p.w_lo; t.bias = p.bias; t.mask = p.mask; t.out = p.out;
      t.H = p.H; t.W = p.W; t.tiles_x = p.tiles_x; t.local = tile; t.skip = false;
    } else {
      while (cur + 1 < njobs && tile >= jobs[cur + 1].tile0) ++cur;
      const ConvJob& J = jobs[cur];
      t.map = &J.map;
      t.w_hi = J.w_hi; t.w_lo = J.w_lo; t.bias = J.bias; t.mask = J.mask; t.out = J.out;
      t.H = J.H; t.W = J.W; t.tiles_x = J.tiles_x; t.local = tile - J.tile0;
      t.skip = J.skip && *J.skip;
    }
    return t;
  };
  const int acc_cols = ROWS * NT;
  const int NB = 2 * acc_cols <= 512 ? 2 : 1;  // accumulator buffers
  const uint32_t ncols = tmem_cols(NB * acc_cols);
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&split[s], 128);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 32 * ConvWarps<BF16>::kEpi);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&tslot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  // tile -> (n-tile, row pair, x segment); the n-tile varies fastest so CTAs running at the
  // same time share the activation halo in L2
  auto decode = [&](const TileJob& t, int& nt, int& ty, int& x0) {
    nt = t.local % ntn;
    const int rest = t.local / ntn;
    ty = (rest / t.tiles_x) * ROWS;
    x0 = (rest % t.tiles_x) * kTileM;
  };

  if (warp == 0) {
    if (lane == 0) {  // producer: halo tile by TMA, weight stage image by bulk copy
      uint32_t it = 0, issued_lo = 0;
      int cur = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
        const TileJob tj = locate(tile, cur);
        if (tj.skip) continue;
        int nt, ty, x0;
        decode(tj, nt, ty, x0);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = it % NS;
          if (it >= (uint32_t)NS && !mbar_wait(&empty[s], ((it / NS) - 1) & 1, abort, p.err))
            break;
          uint8_t* st = smem + s * SB;
          mbar_expect_tx(&full[s], C::A_BYTES + B_BYTES * (BF16 ? 1 : 2));
          tma_load_4d(st, tj.map, &full[s], 0, x0 - 1, ty - 1, i * C::NSLAB);
          const size_t stage = (size_t)nt * nk + i;
          bulk_load(st + C::b_off(), tj.w_hi + stage * B_BYTES, B_BYTES, &full[s]);
          if (!BF16) bulk_load(st + C::b_lo_off(NT), tj.w_lo + stage * B_BYTES, B_BYTES, &full[s]);
          issued_lo = it + 1;
        }
      }
      if (*abort)
        for (uint32_t i = issued_lo > (uint32_t)NS ? issued_lo - NS : 0; i < issued_lo; ++i)
          mbar_drain(&full[i % NS], (i / NS) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t id = idesc(BF16 ? 1 : 2, kTileM, NT, 0, 0);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      int cur = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        if (locate(tile, cur).skip) continue;
        const int buf = (int)(lt % NB);
        if (lt >= (uint32_t)NB && !mbar_wait(&acce[buf], ((lt / NB) - 1) & 1, abort, p.err)) break;
        tc_fence_after();
        const uint32_t dbase = tbase + (uint32_t)(buf * acc_cols);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(BF16 ? &full[s] : &split[s], ph, abort, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * SB);
          const uint32_t sal = sa + C::a_lo_off();
          const uint32_t sb = sa + C::b_off(), sbl = sa + C::b_lo_off(NT);
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const uint32_t bo = (uint32_t)tap * C::NSLAB * NT * 16u;
            const uint64_t db = sdesc(sb + bo, NT * 16, 128);
            const uint32_t acc = (i > 0 || tap > 0) ? 1u : 0u;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {  // output row r reads halo rows r .. r + 2
              const uint32_t ao = (uint32_t)((r + tap / 3) * kHaloX + (tap % 3)) * 16u;
              const uint64_t da = sdesc(sa + ao, C::A_SLAB, 128);
              const uint32_t d = dbase + (uint32_t)(r * NT);
              if (BF16) {
                mma_f16(d, da, db, id, acc);
              } else {
                mma_tf32(d, da, db, id, acc);
                mma_tf32(d, da, sdesc(sbl + bo, NT * 16, 128), id, 1u);
                mma_tf32(d, sdesc(sal + ao, C::A_SLAB, 128), db, id, 1u);
              }
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&accf[buf]);
        ++lt;
      }
    }
  } else if (!BF16 && warp >= 6) {
    // 3xTF32: split each fp32 halo stage into TF32 hi and lo parts, ahead of the MMAs
    const int et = threadIdx.x - 192;
    uint32_t it = 0;
    int cur = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
      if (locate(tile, cur).skip) continue;
      for (int i = 0; i < nk; ++i, ++it) {
        const int s = it % NS;
        if (!mbar_wait(&full[s], (it / NS) & 1, abort, p.err)) break;
        float4* A = reinterpret_cast<float4*>(smem + s * SB);
        float4* Al = reinterpret_cast<float4*>(smem + s * SB + C::a_lo_off());
        for (int q = et; q < (int)(C::A_BYTES / 16); q += 128) {
          float4 h, l;
          split4(A[q], h, l);
          A[q] = h;
          Al[q] = l;
        }
        fence_proxy_async();
        mbar_arrive(&split[s]);
      }
    }
  } else {
    // epilogue: TMEM -> bias + ReLU (forward) or ReLU mask (dgrad) -> global. The dgrad's
    // mask groups of the next 16-column block are loaded before this block's TMEM read.
    constexpr int EW = ConvWarps<BF16>::kEpi;
    constexpr int CSTEP = 16 * (EW / 4);
    constexpr int GE = C::GE;
    constexpr int NG = 16 / GE;  // 16-byte groups per 16 columns
    const int wq = warp & 3;  // the TMEM lane quarter this warp may read
    const int cfirst = 16 * ((warp - 2) >> 2);
    const int row = wq * 32 + lane;
    // dgrad: the mask (the layer's forward activation, long evicted from L2) of a CTA's next
    // tile is requested into L2 one tile ahead, while that tile's MMAs run
    int pcur = 0;
    auto prefetch_mask = [&](int tile) {
      if (MODE != 1 || tile >= ntiles || warp != 2 || lane != 0) return;
      const TileJob tj = locate(tile, pcur);
      if (tj.skip) return;
      int nt, ty, x0;
      decode(tj, nt, ty, x0);
      const size_t npx = (size_t)tj.H * tj.W;
      const int npx_row = min(kTileM, tj.W - x0);
      const char* m = static_cast<const char*>(tj.mask);
      for (int r = 0; r < ROWS && ty + r < tj.H; ++r)
        for (int g = nt * NT / GE; g < (nt + 1) * NT / GE; ++g)
          bulk_prefetch_l2(m + ((size_t)g * npx + (size_t)(ty + r) * tj.W + x0) * 16,
                           (uint32_t)npx_row * 16u);
    };
    prefetch_mask(blockIdx.x);
    uint32_t lt = 0;
    int cur = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      prefetch_mask(tile + gridDim.x);
      const TileJob tj = locate(tile, cur);
      if (tj.skip) continue;
      const int buf = (int)(lt % NB);
      if (!mbar_wait(&accf[buf], (lt / NB) & 1, abort, p.err)) {
        mbar_drain(&accf[buf], (lt / NB) & 1);
        break;
      }
      tc_fence_after();
      int nt, ty, x0;
      decode(tj, nt, ty, x0);
      const int x = x0 + row;
      const size_t npx = (size_t)tj.H * tj.W;
      const uint4* mask = reinterpret_cast<const uint4*>(tj.mask);
      const uint32_t cbase = tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(buf * acc_cols);
      // group index of (16-column block c0, group q) and whether its pixel exists
      auto gidx = [&](int c0, int q) {
        const size_t pix = (size_t)(ty + c0 / NT) * tj.W + x;
        return (size_t)((nt * NT + (c0 % NT) + q * GE) / GE) * npx + pix;
      };
      auto live = [&](int c0) { return x < tj.W && ty + c0 / NT < tj.H; };
      uint4 mnext[NG];
      if (MODE == 1 && live(cfirst))
#pragma unroll
        for (int q = 0; q < NG; ++q) mnext[q] = __ldg(mask + gidx(cfirst, q));
      for (int c0 = cfirst; c0 < acc_cols; c0 += CSTEP) {
        uint4 mcur[NG];
#pragma unroll
        for (int q = 0; q < NG; ++q) mcur[q] = mnext[q];
        const int c1 = c0 + CSTEP;
        if (MODE == 1 && c1 < acc_cols && live(c1))
#pragma unroll
          for (int q = 0; q < NG; ++q) mnext[q] = __ldg(mask + gidx(c1, q));
        uint32_t r[16];
        tmem_ld16(cbase + c0, r);
        tmem_ld_wait();
        if (!live(c0)) continue;
        const int o0 = nt * NT + (c0 % NT);
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
#pragma unroll
        for (int q = 0; q < NG; ++q) {
          float* vv = v + q * GE;
          if (MODE == 0) {
#pragma unroll
            for (int j = 0; j < GE; ++j) {
              const float t = vv[j] + __ldg(tj.bias + o0 + q * GE + j);
              vv[j] = t > 0.f ? t : 0.f;
            }
          } else {
            float mk[GE];
            group_from_raw<T>(mcur[q], mk);
#pragma unroll
            for (int j = 0; j < GE; ++j) vv[j] = mk[j] > 0.f ? vv[j] : 0.f;
          }
          store_group<T>((T*)tj.out, gidx(c0, q), vv);
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      ++lt;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// ---- bf16 weight gradient, several taps per CTA -----------------------------------------
// A CTA covers a group of taps that share image rows, for a slice of cn input channels: the x
// halo tile (R rows x (KP + 2 pu) pixels x cn channels, MN-major) is loaded once per pixel
// chunk and each tap's B operand is the same tile at a descriptor offset of (row, dx) pixels
// (16 bytes per pixel). The group's accumulators sit side by side in TMEM (taps x cn <= 512
// columns). Every group has the same number of taps, so all CTAs carry equal work.
struct TapGroups {
  int n;                                  // groups
  int first[9], count[9], row0[9], c0[9];  // taps first..first+count-1, rows row0..row0+R-1,
                                          // input channels c0..c0+cn-1
  int R;                                  // halo rows (same for every group)
  int cn;                                 // input channels per group
};

TapGroups tap_groups(int cin) {
  TapGroups g{};
  if (cin <= 32) {  // 9 x 32 = 288 columns: all taps, 3-row halo
    g.n = 1; g.first[0] = 0; g.count[0] = 9; g.row0[0] = 0; g.c0[0] = 0; g.R = 3; g.cn = cin;
  } else if (cin <= 128) {  // one row of 3 taps per group
    g.n = 3; g.R = 1; g.cn = cin;
    for (int r = 0; r < 3; ++r) { g.first[r] = 3 * r; g.count[r] = 3; g.row0[r] = r; g.c0[r] = 0; }
  } else {  // C_in = 256: one row of 3 taps for one half of the input channels
    g.n = 6; g.R = 1; g.cn = 128;
    for (int r = 0; r < 3; ++r)
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * r + h;
        g.first[k] = 3 * r; g.count[k] = 3; g.row0[k] = r; g.c0[k] = 128 * h;
      }
  }
  return g;
}

// The bias gradient db[o] = sum_px delta[px][o] comes out of the same GEMM: in the CTAs of tap
// group 0 the B operand of the group's last tap carries two more 8-channel groups, constant bf16
// ones (zeros in the float32 form's second and third parts), so that tap's MMAs (N = C + 16)
// also accumulate sum_px delta into 16 more TMEM columns, at no extra instruction.
__device__ __forceinline__ void fill_ext(uint8_t* ext, uint32_t bytes, uint32_t value) {
  for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(ext)[i] = value;
}
constexpr uint32_t kBf16PairOne = 0x3F803F80u;  // two bf16 1.0

struct WgBf16Params {
  float* part;  // [S][9][C_in][C_out]
  int cin, cout, H, W, chunks_x, total_chunks, per_split;
  int stages;  // pipeline stages
  int pu;      // pixels per TMA unit of both maps
  float* bpart;  // [S][C_out] bias-gradient partials, written by the tap group 0 CTAs
  TapGroups tg;
  const int* skip;
  int* err;
};

constexpr int kWbKP = 64;       // pixels per stage
constexpr int kWbMaxStages = 6;
constexpr uint32_t kWbA = 128u * kWbKP * 2;  // delta tile, 128 channels (zero-filled past C_out)

// x halo pitch: the chunk's KP pixels plus one TMA unit of pu pixels on each side
__host__ __device__ inline int wb_pitch(int pu) { return kWbKP + 2 * pu; }
__host__ __device__ inline uint32_t wb_b_bytes(int cin, int R, int pu) {
  return (uint32_t)(cin / 8) * R * wb_pitch(pu) * 16;
}
// the two extra 8-channel groups (ones) after the x tile
__host__ __device__ inline uint32_t wb_ext_bytes(int R, int pu) { return 2u * R * wb_pitch(pu) * 16; }
__host__ __device__ inline uint32_t wb_stage(int cin, int R, int pu) {
  return align_up(kWbA, 1024) + align_up(wb_b_bytes(cin, R, pu) + wb_ext_bytes(R, pu), 1024);
}
// tap-expanded stage (small C_in): after the raw x tile, [taps x C/8 + 2][KP px][16 B] with the
// two bias groups (ones) last, so one MMA spans every tap of the group
__host__ __device__ inline uint32_t wb_exp_off(int cin, int R, int pu) {
  return align_up(kWbA, 1024) + align_up(wb_b_bytes(cin, R, pu), 1024);
}
__host__ __device__ inline uint32_t wb_stage_exp(int cin, int R, int pu, int taps) {
  return wb_exp_off(cin, R, pu) + align_up(((uint32_t)taps * cin / 8 + 2) * kWbKP * 16, 1024);
}

// EXP = 1 (small C_in): warps 2-5 first copy each stage's x tile into the tap-expanded layout
// (pure 16-byte copies), then serve as the epilogue.
template <int EXP>
__global__ void __launch_bounds__(192, 1) k_wgrad_tc_bf16(const __grid_constant__ CUtensorMap tmD,
                                                         const __grid_constant__ CUtensorMap tmX,
                                                         WgBf16Params p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t full[kWbMaxStages], empty[kWbMaxStages], split[kWbMaxStages], accf;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  if (p.skip && *p.skip) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o0 = blockIdx.x * 128, grp = blockIdx.y, s_idx = blockIdx.z;
  const int t0 = p.tg.first[grp], nt = p.tg.count[grp], r0 = p.tg.row0[grp], R = p.tg.R;
  const int cn = p.tg.cn, c0g = p.tg.c0[grp];
  const int ns = p.stages;
  const int cbeg = s_idx * p.per_split;
  const int cend = min(p.total_chunks, cbeg + p.per_split);
  const int nk = cend > cbeg ? cend - cbeg : 0;
  const int pu = p.pu, HX = wb_pitch(pu);
  const uint32_t BB = wb_b_bytes(cn, R, pu);
  const uint32_t SB = EXP ? wb_stage_exp(cn, R, pu, nt) : wb_stage(cn, R, pu);
  const uint32_t e_off = wb_exp_off(cn, R, pu);
  const uint32_t b_off = align_up(kWbA, 1024);
  const bool bias = grp == 0;
  const uint32_t ncols = tmem_cols(nt * cn + (bias ? 16 : 0));
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&split[s], 4);
    }
    mbar_init(&accf, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&tslot, ncols);
  if (bias) {
    for (int s = 0; s < ns; ++s)
      if (EXP)
        fill_ext(smem + s * SB + e_off + (uint32_t)nt * cn / 8 * kWbKP * 16, 2u * kWbKP * 16,
                 kBf16PairOne);
      else
        fill_ext(smem + s * SB + b_off + BB, wb_ext_bytes(R, pu), kBf16PairOne);
    fence_proxy_async();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % ns;
        if (i >= ns && !mbar_wait(&empty[s], ((i / ns) - 1) & 1, abort, p.err))
          break;
        const int ch = cbeg + i;
        const int y = ch / p.chunks_x, x0 = (ch % p.chunks_x) * kWbKP;
        uint8_t* st = smem + s * SB;
        mbar_expect_tx(&full[s], kWbA + BB);
        tma_load_4d(st, &tmD, &full[s], 0, x0 / pu, y, o0 / 8);
        tma_load_4d(st + b_off, &tmX, &full[s], 0, x0 / pu - 1, y + r0 - 1, c0g / 8);
        issued = i + 1;
      }
      if (*abort)
        for (int i = issued > ns ? issued - ns : 0; i < issued; ++i)
          mbar_drain(&full[i % ns], (i / ns) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc(1, 128, cn, 1, 1), idx = idesc(1, 128, cn + 16, 1, 1);
      const uint32_t a_sbo = kWbKP * 16;                    // next 8-channel group of delta
      const uint32_t b_sbo = (uint32_t)R * HX * 16;  // next 8-channel group of x
      for (int i = 0; i < nk; ++i) {
        const int s = i % ns;
        if (!mbar_wait(EXP ? &split[s] : &full[s], (i / ns) & 1, abort, p.err)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + s * SB), sb = sa + b_off;
        if constexpr (EXP) {
          // taps side by side along N, in chunks of at most 256 columns (multiples of 16)
          const int ntot = nt * cn, nch = (ntot + 255) / 256;
          const int csz = (ntot / nch + 15) / 16 * 16;
          for (int c0 = 0; c0 < ntot; c0 += csz) {
            const int n = min(csz, ntot - c0) + ((bias && c0 + csz >= ntot) ? 16 : 0);
            const uint32_t idc = idesc(1, 128, n, 1, 1);
            const uint32_t eb = sa + e_off + (uint32_t)(c0 / 8) * kWbKP * 16u;
#pragma unroll
            for (int k = 0; k < kWbKP / 16; ++k)
              mma_f16(tbase + (uint32_t)c0, sdesc(sa + (uint32_t)k * 256u, 128, a_sbo),
                      sdesc(eb + (uint32_t)k * 256u, 128, kWbKP * 16), idc,
                      (i > 0 || k > 0) ? 1u : 0u);
          }
        } else {
          for (int j = 0; j < nt; ++j) {
            const int tap = t0 + j;
            // pixel p of the chunk, tap column dx, sits at halo column p + dx - 1 + pu
            const uint32_t boff = (uint32_t)(((tap / 3) - r0) * HX + (tap % 3) + pu - 1) * 16u;
#pragma unroll
            for (int k = 0; k < kWbKP / 16; ++k) {
              const uint32_t ko = (uint32_t)k * 16u * 16u;
              mma_f16(tbase + (uint32_t)(j * cn), sdesc(sa + ko, 128, a_sbo),
                      sdesc(sb + boff + ko, 128, b_sbo), (bias && j == nt - 1) ? idx : id,
                      (i > 0 || k > 0) ? 1u : 0u);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&accf);
    }
  } else {
    if constexpr (EXP) {
      // group gq = j * g8n + g8 holds tap j's view of channel group g8: pixel px of the chunk
      // at raw row (tap / 3 - r0), raw column pu - 1 + px + tap % 3
      const int g8n = cn / 8, et = threadIdx.x - 64;
      for (int i = 0; i < nk; ++i) {
        const int s = i % ns;
        if (!mbar_wait(&full[s], (i / ns) & 1, abort, p.err)) break;
        const uint4* raw = reinterpret_cast<const uint4*>(smem + s * SB + b_off);
        uint4* ex = reinterpret_cast<uint4*>(smem + s * SB + e_off);
        for (int u = et; u < nt * g8n * kWbKP; u += 128) {
          const int gq = u / kWbKP, px = u % kWbKP;
          const int j = gq / g8n, g8 = gq - j * g8n, tap = t0 + j;
          ex[u] = raw[(g8 * R + (tap / 3 - r0)) * HX + pu - 1 + px + tap % 3];
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&split[s]);
      }
    }
    if (!mbar_wait(&accf, 0, abort, p.err)) mbar_drain(&accf, 0);
    tc_fence_after();
    const int wq = warp & 3;
    const int o = o0 + wq * 32 + lane;
    const bool live = o < p.cout && !*abort;
    for (int j = 0; j < nt; ++j) {
      const int tap = t0 + j;
      // part[s][tap][c][o]: the warp's 32 lanes are 32 consecutive o, one 128-byte row per c
      float* dst = p.part + ((size_t)s_idx * 9 + tap) * p.cin * p.cout + (size_t)c0g * p.cout + o;
      for (int c0 = 0; c0 < cn; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(j * cn + c0), r);
        tmem_ld_wait();
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[(size_t)(c0 + q) * p.cout] = nk ? __uint_as_float(r[q]) : 0.f;
      }
    }
    if (bias) {
      uint32_t r[16];
      tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(nt * cn), r);
      tmem_ld_wait();
      if (live) p.bpart[(size_t)s_idx * p.cout + o] = nk ? __uint_as_float(r[0]) : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// ---- float32 weight gradient as three bf16 parts per operand --------------------------------
// Each fp32 value x is split into x = b0 + b1 + b2 (bf16, each the rounded remainder of the
// previous) and D = sum of the six products b_i c_j with i + j <= 2; the three dropped products
// are below 2^-25 of the true one. bf16 operands can be read MN-major, so the tap-grouped halo
// scheme of the bf16 kernel applies unchanged: TMA brings the fp32 tiles, eight split warps
// write the three bf16 images of each, one MMA warp issues six MMAs per tap and K step.
constexpr int kW3KP = 16;  // pixels per stage (one bf16 K step)
constexpr int kW3MaxStages = 4;
constexpr int kW3SplitWarps = 8;
constexpr int kW3Threads = 64 + 32 * kW3SplitWarps;

struct W3Layout {
  uint32_t rawA, rawB, a[3], b[3], stage;
};

// raw x tile pitch: the 16 chunk pixels plus one TMA unit of pu pixels on each side
__host__ __device__ inline int w3_raw_pitch(int pu) { return kW3KP + 2 * pu; }

// exp: the x parts are written tap-expanded, [taps x C/8][16 px][16 B] + 2 bias groups, so one
// MMA covers several taps (N = taps x C): used when C is small (N = C alone would leave the
// tensor pipe idle between MMAs, each of which costs at least ~48 cycles)
__host__ __device__ inline W3Layout w3_layout(int cin, int R, int pu, bool exp = false,
                                              int taps = 0) {
  W3Layout L;
  const uint32_t ra = 128u * kW3KP * 4;                         // [32 g4][16 px][16 B]
  const uint32_t rb = (uint32_t)cin * R * w3_raw_pitch(pu) * 4;  // [C/4][R][16 + 2 pu][16 B]
  const uint32_t pa = 128u * kW3KP * 2;                         // [16 g8][16 px][16 B]
  const uint32_t pb = exp ? ((uint32_t)taps * cin / 8 + 2) * kW3KP * 16
                          : (uint32_t)cin * R * (kW3KP + 2) * 2  // [C/8][R][18 px][16 B]
                                + 2u * R * (kW3KP + 2) * 16;     // + 2 bias groups
  uint32_t o = 0;
  L.rawA = o; o += align_up(ra, 1024);
  L.rawB = o; o += align_up(rb, 1024);
  for (int k = 0; k < 3; ++k) { L.a[k] = o; o += align_up(pa, 1024); }
  for (int k = 0; k < 3; ++k) { L.b[k] = o; o += align_up(pb, 1024); }
  L.stage = o;
  return L;
}

// Two fp32 values -> their three bf16 parts, packed in pairs (value a in the low half). The
// remainders v - b0 and (v - b0) - b1 are exact in fp32.
__device__ __forceinline__ void split3_pair(float a, float b, uint32_t& w0, uint32_t& w1,
                                            uint32_t& w2) {
  const __nv_bfloat162 p0 = __floats2bfloat162_rn(a, b);
  const float2 f0 = __bfloat1622float2(p0);
  const float ra = a - f0.x, rb = b - f0.y;
  const __nv_bfloat162 p1 = __floats2bfloat162_rn(ra, rb);
  const float2 f1 = __bfloat1622float2(p1);
  const __nv_bfloat162 p2 = __floats2bfloat162_rn(ra - f1.x, rb - f1.y);
  w0 = *reinterpret_cast<const uint32_t*>(&p0);
  w1 = *reinterpret_cast<const uint32_t*>(&p1);
  w2 = *reinterpret_cast<const uint32_t*>(&p2);
}

// One 16-byte group of 8 channels: the fp32 groups lo (channels 0-3) and hi (4-7) -> the three
// bf16 images at element index u.
__device__ __forceinline__ void split3_group(const float4 lo, const float4 hi, uint4* b0, uint4* b1,
                                             uint4* b2, int u) {
  uint4 o0, o1, o2;
  split3_pair(lo.x, lo.y, o0.x, o1.x, o2.x);
  split3_pair(lo.z, lo.w, o0.y, o1.y, o2.y);
  split3_pair(hi.x, hi.y, o0.z, o1.z, o2.z);
  split3_pair(hi.z, hi.w, o0.w, o1.w, o2.w);
  b0[u] = o0;
  b1[u] = o1;
  b2[u] = o2;
}

// Splits one stage. Delta tile: raw [32 g4][16 px], parts [16 g8][16 px]. x tile: raw
// [C/4][R][16 + 2 pu px], parts [C/8][R][18 px] (raw column pu - 1 + i -> part column i). Each
// quarter-warp takes 8 consecutive pixels of one row, so its eight 16-byte reads fall in
// distinct bank groups; the 2 halo pixels of each row follow in a short second pass.
template <int R, int EXP>
__device__ __forceinline__ void split3_stage(const uint8_t* st, uint8_t* stw, const W3Layout& L,
                                             int g8n, int pu, int et, int nt, int t0, int r0) {
  constexpr int kThr = 32 * kW3SplitWarps;
  constexpr int PP = kW3KP + 2;  // part pitch
  const int PR = w3_raw_pitch(pu);
  {
    const float4* raw = reinterpret_cast<const float4*>(st + L.rawA);
    for (int u = et; u < 16 * kW3KP; u += kThr) {
      const int g8 = u / kW3KP, px = u % kW3KP;
      split3_group(raw[(2 * g8) * kW3KP + px], raw[(2 * g8 + 1) * kW3KP + px],
                   reinterpret_cast<uint4*>(stw + L.a[0]), reinterpret_cast<uint4*>(stw + L.a[1]),
                   reinterpret_cast<uint4*>(stw + L.a[2]), u);
    }
  }
  const float4* raw = reinterpret_cast<const float4*>(st + L.rawB);
  uint4* b0 = reinterpret_cast<uint4*>(stw + L.b[0]);
  uint4* b1 = reinterpret_cast<uint4*>(stw + L.b[1]);
  uint4* b2 = reinterpret_cast<uint4*>(stw + L.b[2]);
  if constexpr (EXP) {
    // group gq = j * g8n + g8 holds tap j's view of channel group g8: pixel px of the chunk at
    // raw row (tap / 3 - r0), raw column pu - 1 + px + tap % 3
    for (int u = et; u < nt * g8n * kW3KP; u += kThr) {
      const int gq = u / kW3KP, px = u % kW3KP;
      const int j = gq / g8n, g8 = gq - j * g8n, tap = t0 + j;
      const int r = tap / 3 - r0, col = pu - 1 + px + tap % 3;
      split3_group(raw[((2 * g8) * R + r) * PR + col], raw[((2 * g8 + 1) * R + r) * PR + col], b0,
                   b1, b2, u);
    }
    return;
  }
  const int nmain = g8n * R * kW3KP;
  for (int u = et; u < nmain; u += kThr) {
    const int q = u / kW3KP, i = 1 + u % kW3KP;  // q = g8 * R + r, part column i
    const int g8 = q / R, r = q - g8 * R, px = pu - 1 + i;
    split3_group(raw[((2 * g8) * R + r) * PR + px], raw[((2 * g8 + 1) * R + r) * PR + px], b0, b1,
                 b2, q * PP + i);
  }
  for (int u = et; u < g8n * R * 2; u += kThr) {
    const int q = u >> 1, i = (u & 1) ? PP - 1 : 0;
    const int g8 = q / R, r = q - g8 * R, px = pu - 1 + i;
    split3_group(raw[((2 * g8) * R + r) * PR + px], raw[((2 * g8 + 1) * R + r) * PR + px], b0, b1,
                 b2, q * PP + i);
  }
}

template <int R, int EXP>
__global__ void __launch_bounds__(kW3Threads, 2) k_wgrad_tc_f32(const __grid_constant__ CUtensorMap tmD,
                                                               const __grid_constant__ CUtensorMap tmX,
                                                               WgBf16Params p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t full[kW3MaxStages], empty[kW3MaxStages], split[kW3MaxStages], accf;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  if (p.skip && *p.skip) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o0 = blockIdx.x * 128, grp = blockIdx.y, s_idx = blockIdx.z;
  const int t0 = p.tg.first[grp], nt = p.tg.count[grp], r0 = p.tg.row0[grp];
  const int cn = p.tg.cn, c0g = p.tg.c0[grp];
  const int ns = p.stages;
  const int cbeg = s_idx * p.per_split;
  const int cend = min(p.total_chunks, cbeg + p.per_split);
  const int nk = cend > cbeg ? cend - cbeg : 0;
  const int pu = p.pu;
  const W3Layout L = w3_layout(cn, R, pu, EXP, nt);
  const uint32_t RB = (uint32_t)cn * R * w3_raw_pitch(pu) * 4;
  const bool bias = grp == 0;
  const uint32_t ncols = tmem_cols(nt * cn + (bias ? 16 : 0));
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&split[s], kW3SplitWarps);
    }
    mbar_init(&accf, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&tslot, ncols);
  if (bias) {  // part 0: ones, parts 1 and 2: zeros, so the bias columns sum a0 + a1 + a2
    const uint32_t eo = EXP ? (uint32_t)nt * cn / 8 * kW3KP * 16 : (uint32_t)cn * R * (kW3KP + 2) * 2;
    const uint32_t eb = EXP ? 2u * kW3KP * 16 : 2u * R * (kW3KP + 2) * 16;
    for (int s = 0; s < ns; ++s)
      for (int q = 0; q < 3; ++q)
        fill_ext(smem + s * L.stage + L.b[q] + eo, eb, q == 0 ? kBf16PairOne : 0u);
    fence_proxy_async();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % ns;
        if (i >= ns && !mbar_wait(&empty[s], ((i / ns) - 1) & 1, abort, p.err)) break;
        const int ch = cbeg + i;
        const int y = ch / p.chunks_x, x0 = (ch % p.chunks_x) * kW3KP;
        uint8_t* st = smem + s * L.stage;
        mbar_expect_tx(&full[s], 128u * kW3KP * 4 + RB);
        tma_load_4d(st + L.rawA, &tmD, &full[s], 0, x0 / pu, y, o0 / 4);
        tma_load_4d(st + L.rawB, &tmX, &full[s], 0, x0 / pu - 1, y + r0 - 1, c0g / 4);
        issued = i + 1;
      }
      if (*abort)
        for (int i = issued > ns ? issued - ns : 0; i < issued; ++i)
          mbar_drain(&full[i % ns], (i / ns) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idn = idesc(1, 128, cn, 1, 1), idx = idesc(1, 128, cn + 16, 1, 1);
      const uint32_t a_sbo = kW3KP * 16;                     // next 8-channel group of delta
      const uint32_t b_sbo = (uint32_t)R * (kW3KP + 2) * 16;  // next 8-channel group of x
      for (int i = 0; i < nk; ++i) {
        const int s = i % ns;
        if (!mbar_wait(&split[s], (i / ns) & 1, abort, p.err)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * L.stage);
        uint64_t da[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) da[k] = sdesc(st + L.a[k], 128, a_sbo);
        if constexpr (EXP) {
          // the taps side by side along N, in chunks of at most 256 columns (multiples of 16)
          const int ntot = nt * cn, nch = (ntot + 255) / 256;
          const int csz = (ntot / nch + 15) / 16 * 16;
          for (int c0 = 0; c0 < ntot; c0 += csz) {
            const int n = min(csz, ntot - c0) + ((bias && c0 + csz >= ntot) ? 16 : 0);
            const uint32_t id = idesc(1, 128, n, 1, 1);
            uint64_t db[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) db[q] = sdesc(st + L.b[q] + (uint32_t)(c0 / 8) * kW3KP * 16u, 128, kW3KP * 16);
            const uint32_t d = tbase + (uint32_t)c0;
            mma_f16(d, da[0], db[0], id, i > 0 ? 1u : 0u);
            mma_f16(d, da[0], db[1], id, 1u);
            mma_f16(d, da[1], db[0], id, 1u);
            mma_f16(d, da[0], db[2], id, 1u);
            mma_f16(d, da[1], db[1], id, 1u);
            mma_f16(d, da[2], db[0], id, 1u);
          }
        } else {
        for (int j = 0; j < nt; ++j) {
            const int tap = t0 + j;
            const uint32_t boff = (uint32_t)(((tap / 3) - r0) * (kW3KP + 2) + (tap % 3)) * 16u;
            uint64_t db[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) db[k] = sdesc(st + L.b[k] + boff, 128, b_sbo);
            const uint32_t d = tbase + (uint32_t)(j * cn);
            const uint32_t id = (bias && j == nt - 1) ? idx : idn;
            mma_f16(d, da[0], db[0], id, i > 0 ? 1u : 0u);
            mma_f16(d, da[0], db[1], id, 1u);
            mma_f16(d, da[1], db[0], id, 1u);
            mma_f16(d, da[0], db[2], id, 1u);
            mma_f16(d, da[1], db[1], id, 1u);
            mma_f16(d, da[2], db[0], id, 1u);
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&accf);
    }
  } else {
    const int et = threadIdx.x - 64;
    for (int i = 0; i < nk; ++i) {
      const int s = i % ns;
      if (!mbar_wait(&full[s], (i / ns) & 1, abort, p.err)) break;
      uint8_t* st = smem + s * L.stage;
      split3_stage<R, EXP>(st, st, L, cn / 8, pu, et, nt, t0, r0);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&split[s]);
    }
    if (!mbar_wait(&accf, 0, abort, p.err)) mbar_drain(&accf, 0);
    tc_fence_after();
    // warps 2..9: TMEM lane quarter warp % 4, column half (warp - 2) / 4 (16-column blocks
    // alternate between the two halves)
    const int wq = warp & 3, half = (warp - 2) >> 2;
    const int o = o0 + wq * 32 + lane;
    const bool live = o < p.cout && !*abort;
    for (int j = 0; j < nt; ++j) {
      const int tap = t0 + j;
      // part[s][tap][c][o]: the warp's 32 lanes are 32 consecutive o, one 128-byte row per c
      float* dst = p.part + ((size_t)s_idx * 9 + tap) * p.cin * p.cout + (size_t)c0g * p.cout + o;
      for (int c0 = 16 * half; c0 < cn; c0 += 32) {
        uint32_t r[16];
        tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(j * cn + c0), r);
        tmem_ld_wait();
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[(size_t)(c0 + q) * p.cout] = nk ? __uint_as_float(r[q]) : 0.f;
      }
    }
    if (bias && half == 0) {
      uint32_t r[16];
      tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(nt * cn), r);
      tmem_ld_wait();
      if (live) p.bpart[(size_t)s_idx * p.cout + o] = nk ? __uint_as_float(r[0]) : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// gw[(o*C_in + c)*9 + tap] = sum over s of part[s][tap][c][o]. A block owns 32 consecutive o
// (the lanes, so every read is one 128-byte row) of one input channel c and all 9 taps; warp w
// sums the splits s = w, w + 8, ... in order and the eight warp sums are added in warp order,
// so the result is fixed for a given number of splits.
constexpr int kRwO = 32;
__global__ void __launch_bounds__(256) k_reduce_wgrad_tc(const float* __restrict__ part, int S,
                                                         int cin, int cout,
                                                         float* __restrict__ gw, const int* skip) {
  if (skip && *skip) return;
  __shared__ float sh[8][9][kRwO + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int otiles = (cout + kRwO - 1) / kRwO;
  const int o0 = (blockIdx.x % otiles) * kRwO, c = blockIdx.x / otiles;
  const int o = o0 + lane;
  const size_t per = (size_t)9 * cout * cin, tstride = (size_t)cin * cout;
  float acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = 0.f;
  if (o < cout) {
    // splits w, w + 8, ... in order, four loads of each tap in flight (a, b, c, d hold the
    // splits w + 32 i, w + 32 i + 8, ... and are added in that order)
    const float* src = part + (size_t)c * cout + o;
    int k = w;
    for (; k + 24 < S; k += 32)
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const float* q = src + (size_t)t * tstride;
        const float a = q[k * per], b = q[(k + 8) * per], cc = q[(k + 16) * per],
                    d = q[(k + 24) * per];
        acc[t] = (((acc[t] + a) + b) + cc) + d;
      }
    for (; k < S; k += 8)
#pragma unroll
      for (int t = 0; t < 9; ++t) acc[t] += src[k * per + t * tstride];
  }
#pragma unroll
  for (int t = 0; t < 9; ++t) sh[w][t][lane] = acc[t];
  __syncthreads();
  for (int i = threadIdx.x; i < kRwO * 9; i += 256) {
    const int oo = i / 9, t = i % 9;
    if (o0 + oo >= cout) continue;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) v += sh[k][t][oo];
    gw[((size_t)(o0 + oo) * cin + c) * 9 + t] = v;
  }
}

}  // namespace

// out[c] = sum_{r < R} part[r * C + c]: one block per column, each thread sums a fixed strided
// subset of rows in order, then a fixed tree: deterministic for a given R.
__global__ void k_reduce_cols(const float* __restrict__ part, int R, int C, float* __restrict__ out,
                              const int* skip) {
  if (skip && *skip) return;
  __shared__ float sh[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < R; r += blockDim.x) s += part[(size_t)r * C + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

cudaError_t launch_reduce_cols(const float* part, int R, int C, float* out, const int* skip,
                               cudaStream_t st) {
  k_reduce_cols<<<C, 256, 0, st>>>(part, R, C, out, skip);
  count_launch();
  return cudaGetLastError();
}

namespace {

template <int BF16, int MODE, int GROUPED, int ROWS>
cudaError_t conv_tc_launch(const CUtensorMap& m, const ConvTcParams& p, const ConvJob* jobs,
                           int njobs, dim3 grid, uint32_t smem, cudaStream_t st) {
  k_conv_tc<BF16, MODE, GROUPED, ROWS><<<grid, ConvWarps<BF16>::kThreads, smem, st>>>(m, p, jobs,
                                                                                    njobs);
  return cudaGetLastError();
}

}  // namespace

// Sets the dynamic shared-memory limits of every tensor-core kernel and resolves the tensor-map
// encoder, so that later launches (possibly inside a stream capture) do neither.
cudaError_t tc_prepare() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    if (!encode_fn()) {
      result = cudaErrorNotSupported;
      return;
    }
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // dynamic limit = the per-block opt-in total minus the kernel's static shared memory
    auto set = [&](const void* f) {
      if (e != cudaSuccess) return;
      cudaFuncAttributes fa;
      e = cudaFuncGetAttributes(&fa, f);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    };
    set((const void*)k_conv_tc<1, 0, 0, 2>);
    set((const void*)k_conv_tc<1, 0, 0, 1>);
    set((const void*)k_conv_tc<1, 1, 0, 2>);
    set((const void*)k_conv_tc<1, 1, 0, 1>);
    set((const void*)k_conv_tc<0, 0, 0, 2>);
    set((const void*)k_conv_tc<0, 0, 0, 1>);
    set((const void*)k_conv_tc<0, 1, 0, 2>);
    set((const void*)k_conv_tc<0, 1, 0, 1>);
    set((const void*)k_conv_tc<1, 0, 1, 2>);
    set((const void*)k_conv_tc<1, 1, 1, 2>);
    set((const void*)k_conv_tc<0, 0, 1, 2>);
    set((const void*)k_conv_tc<0, 1, 1, 2>);
    set((const void*)k_wgrad_tc_bf16<0>);
    set((const void*)k_wgrad_tc_bf16<1>);
    set((const void*)k_wgrad_tc_f32<1, 0>);
    set((const void*)k_wgrad_tc_f32<1, 1>);
    set((const void*)k_wgrad_tc_f32<3, 1>);
    result = e;
  });
  return result;
}

bool tc_supported(int cin, int cout) {
  auto ok = [](int c) { return c == 32 || c == 64 || c == 128 || c == 256; };
  return ok(cin) && ok(cout) && encode_fn() != nullptr;
}

bool tc_wgrad_supported(int cin, int cout, int bf16) {
  (void)bf16;
  return tc_supported(cin, cout);
}

size_t tc_weight_elems(int cin, int cout) { return (size_t)cin * cout * 9; }

// ---- launch configuration and its tuner ---------------------------------------------------
// A conv launch is persistent: grid = 152 x (CTAs per SM). Two choices change only the speed,
// never a result (every tile is computed the same way by whichever CTA takes it): the number of
// pipeline stages and the CTAs resident per SM (capped by TMEM, 512 columns, and by shared
// memory; shared memory is padded so that exactly the chosen number fit).
struct ConvTune {
  int stages = 2, per_sm = 0, rows = kRowsM;  // per_sm 0: as many as fit
};

static uint32_t conv_stage_bytes(int bf16, int NT, int rows) {
  if (rows == 1) return bf16 ? ConvCfg<1, 1>::stage_bytes(NT) : ConvCfg<0, 1>::stage_bytes(NT);
  return bf16 ? ConvCfg<1, 2>::stage_bytes(NT) : ConvCfg<0, 2>::stage_bytes(NT);
}

static int conv_max_res(int NT, int rows) {
  const int acc_cols = rows * NT;
  return 512 / (int)tmem_cols((2 * acc_cols <= 512 ? 2 : 1) * acc_cols);
}

struct ConvKey {
  int mode, bf16, cin, cout, H, W;
  bool operator<(const ConvKey& o) const {
    return std::tie(mode, bf16, cin, cout, H, W) < std::tie(o.mode, o.bf16, o.cin, o.cout, o.H, o.W);
  }
};
static std::mutex g_tune_mu;
static std::map<ConvKey, ConvTune> g_tune;

static ConvTune conv_tune_for(const ConvKey& k) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  return it == g_tune.end() ? ConvTune() : it->second;
}

static cudaError_t conv_tc_dispatch(int mode, int bf16, const CUtensorMap& m, ConvTcParams p,
                                    const ConvJob* jobs, int njobs, long ntiles, ConvTune tune,
                                    cudaStream_t st) {
  const TcCfg f = tc_cfg(p.cin, p.cout, bf16);
  const int rows = jobs ? kRowsM : tune.rows;  // grouped launches keep the default tiles
  const uint32_t sb = conv_stage_bytes(bf16, f.NT, rows);
  const int max_res = conv_max_res(f.NT, rows);
  int stages = tune.stages;
  while (stages > 2 && (uint32_t)stages * sb > 227u * 1024u - 2048u) --stages;
  uint32_t smem = (uint32_t)stages * sb;
  int per_sm = (int)((227u * 1024u) / (smem + 2048u));
  if (per_sm > max_res) per_sm = max_res;
  if (tune.per_sm > 0 && tune.per_sm < per_sm) per_sm = tune.per_sm;
  if (per_sm < 1) per_sm = 1;
  const uint32_t min_smem = (228u * 1024u) / (uint32_t)(per_sm + 1) + 1024u;
  if (smem < min_smem) smem = min_smem;
  p.stages = stages;
  const long slots = 152L * per_sm;
  dim3 grid((unsigned)(ntiles < slots ? ntiles : slots), 1);
  if (grid.x == 0) return cudaSuccess;
  if (jobs) {
    if (bf16)
      return mode == 0 ? conv_tc_launch<1, 0, 1, 2>(m, p, jobs, njobs, grid, smem, st)
                       : conv_tc_launch<1, 1, 1, 2>(m, p, jobs, njobs, grid, smem, st);
    return mode == 0 ? conv_tc_launch<0, 0, 1, 2>(m, p, jobs, njobs, grid, smem, st)
                     : conv_tc_launch<0, 1, 1, 2>(m, p, jobs, njobs, grid, smem, st);
  }
  if (rows == 1) {
    if (bf16)
      return mode == 0 ? conv_tc_launch<1, 0, 0, 1>(m, p, jobs, njobs, grid, smem, st)
                       : conv_tc_launch<1, 1, 0, 1>(m, p, jobs, njobs, grid, smem, st);
    return mode == 0 ? conv_tc_launch<0, 0, 0, 1>(m, p, jobs, njobs, grid, smem, st)
                     : conv_tc_launch<0, 1, 0, 1>(m, p, jobs, njobs, grid, smem, st);
  }
  if (bf16)
    return mode == 0 ? conv_tc_launch<1, 0, 0, 2>(m, p, jobs, njobs, grid, smem, st)
                     : conv_tc_launch<1, 1, 0, 2>(m, p, jobs, njobs, grid, smem, st);
  return mode == 0 ? conv_tc_launch<0, 0, 0, 2>(m, p, jobs, njobs, grid, smem, st)
                   : conv_tc_launch<0, 1, 0, 2>(m, p, jobs, njobs, grid, smem, st);
}

static cudaError_t conv_params(int bf16, const void* in, int cin, int cout, int H, int W,
                               const void* w_hi, const void* w_lo, const float* b,
                               const void* mask, void* out, const int* skip, int* err, int rows,
                               CUtensorMap* m, ConvTcParams* p) {
  const int KC = bf16 ? ConvCfg<1>::KC : ConvCfg<0>::KC;
  const int GE = bf16 ? 8 : 4;
  cudaError_t e = make_map(m, in, bf16, cin, H, W, kHaloX, rows + 2, KC / GE);
  if (e != cudaSuccess) return e;
  p->w_hi = (const uint8_t*)w_hi;
  p->w_lo = (const uint8_t*)w_lo;
  p->bias = b;
  p->mask = mask;
  p->out = out;
  p->cin = cin;
  p->cout = cout;
  p->H = H;
  p->W = W;
  p->tiles_x = (W + kTileM - 1) / kTileM;
  p->stages = 2;
  p->skip = skip;
  p->err = err;
  return cudaSuccess;
}

cudaError_t conv_tc_autotune(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                             const void* w_hi, const void* w_lo, const float* b, const void* mask,
                             void* out, int* err, cudaStream_t st) {
  if (!tc_supported(cin, cout)) return cudaErrorNotSupported;
  if (const cudaError_t pe = tc_prepare()) return pe;
  const ConvKey key{mode, bf16, cin, cout, H, W};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.count(key)) return cudaSuccess;
  }
  const TcCfg f = tc_cfg(cin, cout, bf16);
  cudaEvent_t a = nullptr, z = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  ConvTune best;
  float best_ms = 1e30f;
  for (int rows = 1; rows <= 2 && e == cudaSuccess; ++rows) {
    CUtensorMap m;
    ConvTcParams p;
    e = conv_params(bf16, in, cin, cout, H, W, w_hi, w_lo, b, mask, out, nullptr, err, rows, &m, &p);
    if (e != cudaSuccess) break;
    const long ntiles = (long)p.tiles_x * ((H + rows - 1) / rows) * (cout / f.NT);
    const uint32_t sb = conv_stage_bytes(bf16, f.NT, rows);
    for (int stages = 2; stages <= kConvMaxStages && e == cudaSuccess; ++stages) {
      if ((uint32_t)stages * sb > 227u * 1024u - 2048u) break;
      for (int per_sm = 1; per_sm <= conv_max_res(f.NT, rows) && e == cudaSuccess; ++per_sm) {
        if (per_sm * ((uint32_t)stages * sb + 2048u) > 227u * 1024u) break;
        const ConvTune t{stages, per_sm, rows};
        float ms = 0.f;
        e = conv_tc_dispatch(mode, bf16, m, p, nullptr, 0, ntiles, t, st);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r)
          e = conv_tc_dispatch(mode, bf16, m, p, nullptr, 0, ntiles, t, st);
        if (e == cudaSuccess) e = cudaEventRecord(z, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(z);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return cudaSuccess;
}

cudaError_t launch_conv_tc(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                           const void* w_hi, const void* w_lo, const float* b, const void* mask,
                           void* out, const int* skip, int* err, cudaStream_t st) {
  if (!tc_supported(cin, cout)) return cudaErrorNotSupported;
  if (const cudaError_t pe = tc_prepare()) return pe;
  const TcCfg f = tc_cfg(cin, cout, bf16);
  const ConvTune t = conv_tune_for(ConvKey{mode, bf16, cin, cout, H, W});
  CUtensorMap m;
  ConvTcParams p;
  cudaError_t e = conv_params(bf16, in, cin, cout, H, W, w_hi, w_lo, b, mask, out, skip, err,
                              t.rows, &m, &p);
  if (e != cudaSuccess) return e;
  const long ntiles = (long)p.tiles_x * ((H + t.rows - 1) / t.rows) * (cout / f.NT);
  e = conv_tc_dispatch(mode, bf16, m, p, nullptr, 0, ntiles, t, st);
  count_launch();
  return e;
}

size_t conv_job_size() { return sizeof(ConvJob); }

cudaError_t conv_group_table(int mode, int bf16, int cin, int cout, const ConvGroupEntry* e,
                             int n, void* table, long* ntiles) {
  (void)mode;
  if (!tc_supported(cin, cout)) return cudaErrorNotSupported;
  const TcCfg f = tc_cfg(cin, cout, bf16);
  const int KC = bf16 ? ConvCfg<1>::KC : ConvCfg<0>::KC;
  const int GE = bf16 ? 8 : 4;
  ConvJob* t = static_cast<ConvJob*>(table);
  long tiles = 0;
  for (int k = 0; k < n; ++k) {
    memset(&t[k], 0, sizeof(ConvJob));
    cudaError_t r = make_map(&t[k].map, e[k].in, bf16, cin, e[k].H, e[k].W, kHaloX, kRowsM + 2,
                             KC / GE);
    if (r != cudaSuccess) return r;
    t[k].w_hi = (const uint8_t*)e[k].w_hi;
    t[k].w_lo = (const uint8_t*)e[k].w_lo;
    t[k].bias = e[k].bias;
    t[k].mask = e[k].mask;
    t[k].out = e[k].out;
    t[k].skip = e[k].skip;
    t[k].H = e[k].H;
    t[k].W = e[k].W;
    t[k].tiles_x = (e[k].W + kTileM - 1) / kTileM;
    t[k].tile0 = (int)tiles;
    tiles += (long)t[k].tiles_x * ((e[k].H + kRowsM - 1) / kRowsM) * (cout / f.NT);
  }
  *ntiles = tiles;
  return cudaSuccess;
}

cudaError_t launch_conv_tc_grouped(int mode, int bf16, int cin, int cout, const void* dtable,
                                   int n, long ntiles, int* err, cudaStream_t st) {
  if (!tc_supported(cin, cout)) return cudaErrorNotSupported;
  if (const cudaError_t pe = tc_prepare()) return pe;
  if (ntiles > 0x7fffffffL) return cudaErrorInvalidValue;
  ConvTcParams p;
  memset(&p, 0, sizeof(p));
  p.cin = cin;
  p.cout = cout;
  p.tiles_x = (int)ntiles;  // the grouped kernel's total tile count
  p.stages = 2;
  p.err = err;
  CUtensorMap unused;
  memset(&unused, 0, sizeof(unused));
  const cudaError_t e =
      conv_tc_dispatch(mode, bf16, unused, p, (const ConvJob*)dtable, n, ntiles, ConvTune(), st);
  count_launch();
  return e;
}


// bf16 = 1: bf16 maps, k_wgrad_tc_bf16; bf16 = 0: float32 maps, k_wgrad_tc_f32 (three bf16 parts)
static cudaError_t launch_wgrad_grouped(int bf16, const void* dout, const void* in, int cin,
                                        int cout, int H, int W, float* part, size_t part_cap,
                                        float* gw, float* gb, const int* skip, int* err,
                                        cudaStream_t st) {
  const TapGroups tg = tap_groups(cin);
  const int KP = bf16 ? kWbKP : kW3KP, GE = bf16 ? 8 : 4;
  // pixels per TMA unit: 128-byte box rows for bf16 (the halo grows by 14 pixels of 66),
  // 64-byte rows for float32 (the raw tile of 16 pixels would grow too much with 8)
  const int pu_max = bf16 ? 8 : 4;
  int pu = 1;
  while (pu < pu_max && W % (2 * pu) == 0) pu *= 2;
  CUtensorMap md, mx;
  cudaError_t e = make_map(&md, dout, bf16, cout, H, W, KP / pu, 1, 128 / GE, pu);
  if (e == cudaSuccess) e = make_map(&mx, in, bf16, cin, H, W, KP / pu + 2, tg.R, tg.cn / GE, pu);
  if (e != cudaSuccess) return e;
  const int otiles = (cout + 127) / 128;
  WgBf16Params p;
  p.cin = cin;
  p.cout = cout;
  p.H = H;
  p.W = W;
  p.chunks_x = (W + KP - 1) / KP;
  p.total_chunks = p.chunks_x * H;
  p.tg = tg;
  p.pu = pu;
  const size_t per_split_elems = (size_t)9 * cout * cin;
  int maxcols = 0;  // group 0 also holds the 16 bias columns
  for (int g = 0; g < tg.n; ++g) {
    const int cols = tg.count[g] * tg.cn + (g == 0 ? 16 : 0);
    maxcols = cols > maxcols ? cols : maxcols;
  }
  const int max_res = 512 / (int)tmem_cols(maxcols);  // CTAs per SM that TMEM allows
  // as many stages as fit beside the CTAs that TMEM allows on one SM
  // tap-expanded x operand when a tap alone would give MMAs of small N: float32 form for
  // C_in <= 64, bf16 form for C_in = 32 (its expansion is a copy pass)
  const bool exp = bf16 ? tg.cn <= 32 : tg.cn <= 64;
  const uint32_t sb = bf16 ? (exp ? wb_stage_exp(tg.cn, tg.R, pu, tg.count[0]) : wb_stage(tg.cn, tg.R, pu))
                           : w3_layout(tg.cn, tg.R, pu, exp, tg.count[0]).stage;
  const int max_stages = bf16 ? kWbMaxStages : kW3MaxStages;
  p.stages = (int)((227u * 1024u / (uint32_t)max_res - 2048u) / sb);
  if (p.stages > max_stages) p.stages = max_stages;
  if (p.stages < 2) p.stages = 2;
  uint32_t smem = (uint32_t)p.stages * sb;
  // a CTA holding more than half of TMEM keeps the SM to itself
  if (max_res == 1 && smem < 116u * 1024u) smem = 116u * 1024u;
  const int per_sm = (int)((227u * 1024u) / (smem + 2048u));
  const int ctas = otiles * tg.n;
  // one wave of equal CTAs (every group carries the same work), unless it leaves more than a
  // tenth of the slots idle; each extra wave costs a pipeline fill and a partial-sum epilogue
  const int slots = 152 * (per_sm > 0 ? per_sm : 1);
  int S = slots / ctas;
  if (S * ctas * 10 < slots * 9) S = 2 * slots / ctas;
  if (S > p.total_chunks / 16) S = p.total_chunks / 16;  // at least 16 pixel chunks per split
  if (S < 1) S = 1;
  while (S > 1 && (size_t)S * (per_split_elems + cout) + 64 > part_cap) --S;
  if ((size_t)S * (per_split_elems + cout) + 64 > part_cap) return cudaErrorInvalidValue;
  p.per_split = (p.total_chunks + S - 1) / S;
  S = (p.total_chunks + p.per_split - 1) / p.per_split;
  p.part = part;
  p.bpart = part + ((size_t)S * per_split_elems + 63) / 64 * 64;
  p.skip = skip;
  p.err = err;
  const dim3 grid((unsigned)otiles, (unsigned)tg.n, (unsigned)S);
  if (bf16 && exp)
    k_wgrad_tc_bf16<1><<<grid, 192, smem, st>>>(md, mx, p);
  else if (bf16)
    k_wgrad_tc_bf16<0><<<grid, 192, smem, st>>>(md, mx, p);
  else if (tg.R == 3)
    k_wgrad_tc_f32<3, 1><<<grid, kW3Threads, smem, st>>>(md, mx, p);
  else if (exp)
    k_wgrad_tc_f32<1, 1><<<grid, kW3Threads, smem, st>>>(md, mx, p);
  else
    k_wgrad_tc_f32<1, 0><<<grid, kW3Threads, smem, st>>>(md, mx, p);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_reduce_wgrad_tc<<<(unsigned)(((cout + kRwO - 1) / kRwO) * cin), 256, 0, st>>>(part, S, cin,
                                                                                 cout, gw, skip);
  count_launch();
  // bias: the S per-split sums of tap group 0, added in split order
  return launch_reduce_cols(p.bpart, S, cout, gb, skip, st);
}

cudaError_t launch_wgrad_tc(int bf16, const void* dout, const void* in, int cin, int cout, int H,
                            int W, float* part, size_t part_cap, float* gw, float* gb,
                            const int* skip, int* err, cudaStream_t st) {
  if (!tc_wgrad_supported(cin, cout, bf16)) return cudaErrorNotSupported;
  if (const cudaError_t pe = tc_prepare()) return pe;
  return launch_wgrad_grouped(bf16, dout, in, cin, cout, H, W, part, part_cap, gw, gb, skip, err,
                              st);
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
