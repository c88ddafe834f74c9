// tcgen05 / TMEM implicit-GEMM forward and dgrad kernels for the 3x3 layers with C_in, C_out in
// {32, ..., 256} (sm_103a), their launch tuner and the grouped (many-image) launch.
//
// D[px][n] = sum_{tap, c} A[px + tap][c] B[n][tap, c]: M = 128 pixels of one image row, N =
// output channels, K = 9 C_in. The A operand of every tap is the same TMA halo tile (rows + 2
// rows x 132 pixels from two left of the tile x a chunk of channels, zero outside the image =
// the "same" padding) addressed at a shifted start: in the K-major no-swizzle layout each pixel
// row is 16 bytes, so a shift of dx pixels is a 16*dx byte offset of the descriptor. Starting
// two pixels left lets TMA move the tile in two-pixel (32-byte) box rows when W is even: with
// 16-byte rows it fetches every 32-byte L2 sector twice. One warp issues TMA copies,
// one thread issues the MMAs into TMEM accumulators, the epilogue warps read TMEM back for the
// fused bias + ReLU (forward) or ReLU mask (dgrad), and in the float32 form a warpgroup splits
// the activations into scaled fp16 hi/lo parts in shared memory first (f16_split.cuh; the
// weights arrive as packed fp16 parts), so each K step is three f16-kind MMAs.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "cg_util.cuh"
#include "checked.cuh"
#include "n2f_internal.h"
#include "tc_common.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"
#include "trainer.h"

namespace n2f {

using namespace tc;

namespace {

// ---- forward / dgrad ----------------------------------------------------------------------
struct ConvTcParams {
  const uint8_t* w_hi;  // packed weight stage images (bf16, or the fp16 hi parts)
  const uint8_t* w_lo;  // fp16 residual images (float32 form)
  const float* bias;    // forward
  const void* mask;     // dgrad: the layer's input activation (ReLU mask)
  void* out;
  ConvScales sc;        // float32 form: largest magnitudes of A, of the weights, of the output
  int cin, cout, H, W, tiles_x;
  int pu;      // pixels per TMA box row of the halo map (2 when W is even, else 1)
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
  ConvScales sc;
  int H, W, tiles_x, tile0, pu;
};

constexpr int kTileM = 128;   // pixels per accumulator (one image row segment)
constexpr int kRowsM = 2;     // image rows per tile by default: each weight stage feeds two
                              // accumulators (1 is a tuning choice: twice the tiles, half the
                              // accumulator columns, so TMEM double-buffers at N = 256)
constexpr int kHaloX = kTileM + 4;  // halo tile pixels: x0 - 2 .. x0 + 129
constexpr int kConvMaxStages = 4;

template <int BF16, int ROWS = kRowsM>
struct ConvCfg {
  static constexpr int GE = BF16 ? 8 : 4;  // channels per 16-byte group of the activation map
  static constexpr int KC = 16;            // channels per stage (one 16-element K step)
  static constexpr int NSLAB = 2;          // 16-byte K slabs of a 16-bit operand per stage
  static constexpr int NRAW = KC / GE;     // map groups per pixel and stage (2 bf16, 4 fp32)
  static constexpr int HALO_Y = ROWS + 2;
  static constexpr uint32_t A_SLAB = HALO_Y * kHaloX * 16;  // K distance between halo slabs
  static constexpr uint32_t A_BYTES = NRAW * A_SLAB;         // the TMA halo tile
  // float32 form: the split leaves the hi parts in slabs 0-1 and the lo parts in slabs 2-3
  static constexpr uint32_t A_LO = 2 * A_SLAB;
  static __host__ __device__ uint32_t b_bytes(int NT) { return 9u * NSLAB * NT * 16; }
  // stage layout: A (raw, split in place) | B | B_lo (float32 form)
  static __host__ __device__ uint32_t b_off() { return align_up(A_BYTES, 1024); }
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
// quarter, alternate 16-column blocks); float32: 2-5 epilogue, 6-9 operand split.
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
  ConvScales sc;
  int H, W, tiles_x, local, pu;
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
      t.sc = p.sc;
      t.H = p.H; t.W = p.W; t.tiles_x = p.tiles_x; t.local = tile; t.skip = false; t.pu = p.pu;
    } else {
      while (cur + 1 < njobs && tile >= jobs[cur + 1].tile0) ++cur;
      const ConvJob& J = jobs[cur];
      t.map = &J.map;
      t.w_hi = J.w_hi; t.w_lo = J.w_lo; t.bias = J.bias; t.mask = J.mask; t.out = J.out;
      t.sc = J.sc;
      t.H = J.H; t.W = J.W; t.tiles_x = J.tiles_x; t.local = tile - J.tile0; t.pu = J.pu;
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
          tma_load_4d(st, tj.map, &full[s], 0, (x0 - 2) / tj.pu, ty - 1, i * C::NRAW);
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
      const uint32_t id = idesc(BF16 ? 1 : 0, kTileM, NT, 0, 0);  // bf16 / fp16 operands
      // descriptors of stage 0; a stage, a tap and a row only add their byte offset / 16 to the
      // start-address field (every address is below 2^18, so the 14-bit field never carries)
      const uint32_t s0 = smem_u32(smem);
      const uint64_t dA0 = sdesc(s0, C::A_SLAB, 128), dAl0 = sdesc(s0 + C::A_LO, C::A_SLAB, 128);
      const uint64_t dB0 = sdesc(s0 + C::b_off(), NT * 16, 128);
      const uint64_t dBl0 = sdesc(s0 + C::b_lo_off(NT), NT * 16, 128);
      const uint64_t btap = (uint64_t)(C::NSLAB * NT);  // one tap of B, in 16-byte units
      uint32_t lt = 0;
      int s = 0;  // stage and phase of the next K step (the producer's sequence)
      uint32_t ph = 0;
      bool ok = true;
      int cur = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        if (locate(tile, cur).skip) continue;
        const int buf = (int)(lt % NB);
        if (lt >= (uint32_t)NB && !mbar_wait(&acce[buf], ((lt / NB) - 1) & 1, abort, p.err)) break;
        tc_fence_after();
        const uint32_t dbase = tbase + (uint32_t)(buf * acc_cols);
        for (int i = 0; i < nk; ++i) {
          if (!mbar_wait(BF16 ? &full[s] : &split[s], ph, abort, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t so = (uint64_t)((uint32_t)s * SB >> 4);
          const uint64_t dA = dA0 + so, dAl = dAl0 + so;
          uint64_t db = dB0 + so, dbl = dBl0 + so;
#pragma unroll
          for (int tap = 0; tap < 9; ++tap, db += btap, dbl += btap) {
            const uint32_t acc = (i > 0 || tap > 0) ? 1u : 0u;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {  // output row r reads halo rows r .. r + 2
              // output pixel m, tap column dx in 0..2 reads halo column m + dx + 1
              const uint64_t ao = (uint64_t)((r + tap / 3) * kHaloX + (tap % 3) + 1);  // 16 B units
              const uint32_t d = dbase + (uint32_t)(r * NT);
              mma_f16(d, dA + ao, db, id, acc);
              if (!BF16) {  // hi*lo and lo*hi
                mma_f16(d, dA + ao, dbl, id, 1u);
                mma_f16(d, dAl + ao, db, id, 1u);
              }
            }
          }
          mma_commit(&empty[s]);
          if (++s == NS) { s = 0; ph ^= 1u; }
        }
        mma_commit(&accf[buf]);
        ++lt;
      }
    }
  } else if (!BF16 && warp >= 6) {
    // float32 form: each halo pixel's 16 fp32 channels (four map groups) -> the scaled fp16 hi
    // parts (slabs 0-1) and lo parts (slabs 2-3), in place: a thread owns one pixel in all four
    // slabs. The scale comes from the A tensor's largest magnitude.
    const int et = threadIdx.x - 192;
    constexpr int QS = (int)(C::A_SLAB / 16);  // halo pixels
    uint32_t it = 0;
    int cur = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
      const TileJob tj = locate(tile, cur);
      if (tj.skip) continue;
      const float sc = f16_scale(tj.sc.in);
      for (int i = 0; i < nk; ++i, ++it) {
        const int s = it % NS;
        if (!mbar_wait(&full[s], (it / NS) & 1, abort, p.err)) break;
        float4* A = reinterpret_cast<float4*>(smem + s * SB);
        uint4* U = reinterpret_cast<uint4*>(smem + s * SB);
        for (int q = et; q < QS; q += 128) {
          const float4 r0 = A[q], r1 = A[QS + q], r2 = A[2 * QS + q], r3 = A[3 * QS + q];
          uint4 h0, l0, h1, l1;
          split_f16_group(r0, r1, sc, h0, l0);
          split_f16_group(r2, r3, sc, h1, l1);
          U[q] = h0;
          U[QS + q] = h1;
          U[2 * QS + q] = l0;
          U[3 * QS + q] = l1;
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
      // float32 form: undo the operand scales (exact powers of two, applied one at a time)
      const float ua = BF16 ? 1.f : f16_unscale(tj.sc.in), uw = BF16 ? 1.f : f16_unscale(tj.sc.w);
      float mx = 0.f;  // largest |output| of this thread's tile part
      const size_t npx = (size_t)tj.H * tj.W;
      const uint4* mask = reinterpret_cast<const uint4*>(tj.mask);
      const uint32_t cbase = tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(buf * acc_cols);
      // group index of (16-column block c0, group q) and whether its pixel exists
      auto gidx = [&](int c0, int q) {
        const size_t pix = (size_t)(ty + c0 / NT) * tj.W + x;
        return (size_t)((nt * NT + (c0 % NT) + q * GE) / GE) * npx + pix;
      };
      auto live = [&](int c0) { return x < tj.W && ty + c0 / NT < tj.H; };
      const size_t ngroups = (size_t)(ntn * NT / GE) * npx;  // groups of the output (and mask)
      uint4 mnext[NG];
      if (MODE == 1 && live(cfirst))
#pragma unroll
        for (int q = 0; q < NG; ++q)
          if (N2F_IN(gidx(cfirst, q), ngroups)) mnext[q] = __ldg(mask + gidx(cfirst, q));
      for (int c0 = cfirst; c0 < acc_cols; c0 += CSTEP) {
        uint4 mcur[NG];
#pragma unroll
        for (int q = 0; q < NG; ++q) mcur[q] = mnext[q];
        const int c1 = c0 + CSTEP;
        if (MODE == 1 && c1 < acc_cols && live(c1))
#pragma unroll
          for (int q = 0; q < NG; ++q)
            if (N2F_IN(gidx(c1, q), ngroups)) mnext[q] = __ldg(mask + gidx(c1, q));
        uint32_t r[16];
        tmem_ld16(cbase + c0, r);
        tmem_ld_wait();
        if (!live(c0)) continue;
        const int o0 = nt * NT + (c0 % NT);
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = BF16 ? __uint_as_float(r[j]) : __uint_as_float(r[j]) * ua * uw;
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
          if (!BF16)
#pragma unroll
            for (int j = 0; j < GE; ++j) mx = fmaxf(mx, fabsf(vv[j]));
          if (N2F_IN(gidx(c0, q), ngroups)) store_group<T>((T*)tj.out, gidx(c0, q), vv);
        }
      }
      if (!BF16 && tj.sc.out) warp_absmax_to(mx, tj.sc.out);
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

template <int BF16, int MODE, int GROUPED, int ROWS>
cudaError_t conv_tc_launch(const CUtensorMap& m, const ConvTcParams& p, const ConvJob* jobs,
                           int njobs, dim3 grid, uint32_t smem, cudaStream_t st) {
  k_conv_tc<BF16, MODE, GROUPED, ROWS><<<grid, ConvWarps<BF16>::kThreads, smem, st>>>(m, p, jobs,
                                                                                    njobs);
  return cudaGetLastError();
}

}  // namespace

// Sets the dynamic shared-memory limit of every forward / dgrad kernel (the per-block opt-in total
// minus its static shared memory), so that later launches (possibly inside a stream capture)
// need no attribute calls.
cudaError_t conv_tc_prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
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
  return e;
}

bool tc_supported(int cin, int cout) {
  auto ok = [](int c) { return c == 32 || c == 64 || c == 128 || c == 256; };
  return ok(cin) && ok(cout) && encode_fn() != nullptr;
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
                               const void* mask, void* out, ConvScales sc, const int* skip,
                               int* err, int rows, CUtensorMap* m, ConvTcParams* p) {
  if (!bf16 && (!sc.in || !sc.w || !w_lo)) return cudaErrorInvalidValue;
  const int NRAW = bf16 ? ConvCfg<1>::NRAW : ConvCfg<0>::NRAW;
  const int pu = W % 2 == 0 ? 2 : 1;
  cudaError_t e = make_map(m, in, bf16, cin, H, W, kHaloX / pu, rows + 2, NRAW, pu);
  if (e != cudaSuccess) return e;
  p->w_hi = (const uint8_t*)w_hi;
  p->w_lo = (const uint8_t*)w_lo;
  p->bias = b;
  p->mask = mask;
  p->out = out;
  p->sc = sc;
  p->cin = cin;
  p->cout = cout;
  p->H = H;
  p->W = W;
  p->tiles_x = (W + kTileM - 1) / kTileM;
  p->pu = pu;
  p->stages = 2;
  p->skip = skip;
  p->err = err;
  return cudaSuccess;
}

cudaError_t conv_tc_autotune(int mode, int bf16, const void* in, int cin, int cout, int H, int W,
                             const void* w_hi, const void* w_lo, const float* b, const void* mask,
                             void* out, ConvScales sc, int* err, cudaStream_t st) {
  sc.out = nullptr;  // trial launches leave the tensors' magnitude words alone
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
    e = conv_params(bf16, in, cin, cout, H, W, w_hi, w_lo, b, mask, out, sc, nullptr, err, rows,
                    &m, &p);
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
                           void* out, ConvScales sc, const int* skip, int* err, cudaStream_t st) {
  if (!tc_supported(cin, cout)) return cudaErrorNotSupported;
  if (const cudaError_t pe = tc_prepare()) return pe;
  const TcCfg f = tc_cfg(cin, cout, bf16);
  const ConvTune t = conv_tune_for(ConvKey{mode, bf16, cin, cout, H, W});
  CUtensorMap m;
  ConvTcParams p;
  cudaError_t e = conv_params(bf16, in, cin, cout, H, W, w_hi, w_lo, b, mask, out, sc, skip, err,
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
  const int NRAW = bf16 ? ConvCfg<1>::NRAW : ConvCfg<0>::NRAW;
  ConvJob* t = static_cast<ConvJob*>(table);
  long tiles = 0;
  for (int k = 0; k < n; ++k) {
    memset(static_cast<void*>(&t[k]), 0, sizeof(ConvJob));  // the table is host bytes
    if (!bf16 && (!e[k].sc.in || !e[k].sc.w || !e[k].w_lo)) return cudaErrorInvalidValue;
    const int pu = e[k].W % 2 == 0 ? 2 : 1;
    cudaError_t r = make_map(&t[k].map, e[k].in, bf16, cin, e[k].H, e[k].W, kHaloX / pu,
                             kRowsM + 2, NRAW, pu);
    if (r != cudaSuccess) return r;
    t[k].pu = pu;
    t[k].sc = e[k].sc;
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
  memset(static_cast<void*>(&p), 0, sizeof(p));
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

N2F_CHECK_READER(check_read_conv)

}  // namespace n2f
