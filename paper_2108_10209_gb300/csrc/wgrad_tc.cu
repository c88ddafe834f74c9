// tcgen05 / TMEM weight-gradient kernels for the 3x3 layers (sm_103a) and their fixed-order
// reductions.
//
// D[o][c] = sum_px delta[px][o] x[px + tap][c] per tap: M = 128 output channels, N = C_in (per
// tap, or several taps side by side), K = pixels; the operands are read MN-major from the
// channel-grouped maps, the pixel sum is split over pixel chunks and the partial sums are
// reduced in a fixed order. The bias gradient comes out of the same GEMM (a B operand extended
// by 16 columns of ones).
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
// group 0 the B operand of the group's last tap carries two more 8-channel groups, constant
// ones (bf16, or fp16 in the float32 form's hi part and zeros in its lo part), so that tap's
// MMAs (N = C + 16) also accumulate sum_px delta into 16 more TMEM columns, at no extra
// instruction.
__device__ __forceinline__ void fill_ext(uint8_t* ext, uint32_t bytes, uint32_t value) {
  for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(ext)[i] = value;
}
constexpr uint32_t kBf16PairOne = 0x3F803F80u;  // two bf16 1.0
constexpr uint32_t kF16PairOne = 0x3C003C00u;   // two fp16 1.0

struct WgBf16Params {
  float* part;  // [S][9][C_in][C_out]
  size_t part_cap;  // floats of the workspace at part (partials, then the bias partials)
  int cin, cout, H, W, chunks_x, total_chunks, per_split;
  int stages;  // pipeline stages
  int pu;      // bf16 kernel: pixels per TMA unit of both maps
  float* bpart;  // [S][C_out] bias-gradient partials, written by the tap group 0 CTAs
  TapGroups tg;
  const unsigned* dmax;  // float32 form: largest |delta| and |x| (operand scales)
  const unsigned* xmax;
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

// Warps after the producer and the MMA warp: the epilogue, and for EXP = 1 (small C_in) first
// the copy of each stage's x tile into the tap-expanded layout (pure 16-byte copies). The copy
// of a 64-pixel chunk is 2304 groups for the nine taps of C_in = 32; four warps took ~3600
// cycles a chunk for ~600 tensor cycles, so the tap-expanded kernel has sixteen.
template <int EXP>
struct WbWarps {
  static constexpr int kCopy = EXP ? 16 : 4;  // copy / epilogue warps
  static constexpr int kThreads = 64 + 32 * kCopy;
  // each copy thread's groups of one chunk (at most 36 8-channel groups x 64 pixels)
  static constexpr int kMaxCopy = (36 * kWbKP + 32 * kCopy - 1) / (32 * kCopy);
};

template <int EXP>
__global__ void __launch_bounds__(WbWarps<EXP>::kThreads, 1) k_wgrad_tc_bf16(const __grid_constant__ CUtensorMap tmD,
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
  // delta's 8-channel groups that hold output channels (the rest of the M = 128 rows is zero)
  const int dgroups = min(16, (p.cout - o0 + 7) / 8);
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&split[s], WbWarps<EXP>::kCopy);
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
      int issued = 0, s = 0, y = cbeg / p.chunks_x, cx = cbeg - y * p.chunks_x;
      uint32_t ph = 0;
      for (int i = 0; i < nk; ++i) {
        if (i >= ns && !mbar_wait(&empty[s], ph ^ 1u, abort, p.err)) break;
        const int x0 = cx * kWbKP;
        uint8_t* st = smem + s * SB;
        mbar_expect_tx(&full[s], kWbA + BB);
        tma_load_4d(st, &tmD, &full[s], 0, x0 / pu, y, o0 / 8);
        tma_load_4d(st + b_off, &tmX, &full[s], 0, x0 / pu - 1, y + r0 - 1, c0g / 8);
        issued = i + 1;
        if (++cx == p.chunks_x) { cx = 0; ++y; }
        if (++s == ns) { s = 0; ph ^= 1u; }
      }
      if (*abort)
        for (int i = issued > ns ? issued - ns : 0; i < issued; ++i)
          mbar_drain(&full[i % ns], (i / ns) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // descriptors and instruction words fixed up front for stage 0 (stage s adds
      // s x SB / 16 to the start-address field): per chunk, the MMA groups (taps of the group, or
      // tap-expanded column chunks of at most 256) x the four 16-pixel K steps
      constexpr int kWbMma = EXP ? 2 : 3, kKs = kWbKP / 16;
      const uint32_t a_sbo = kWbKP * 16;             // next 8-channel group of delta
      const uint32_t b_sbo = (uint32_t)R * HX * 16;  // next 8-channel group of x
      const uint32_t s0 = smem_u32(smem);
      uint64_t da[kKs], db[kWbMma];
      uint32_t dcol[kWbMma], idw[kWbMma];
      int ngrp = 0;
#pragma unroll
      for (int k = 0; k < kKs; ++k) da[k] = sdesc(s0 + (uint32_t)k * 256u, 128, a_sbo);
      if constexpr (EXP) {
        const int ntot = nt * cn, nch = (ntot + 255) / 256;
        const int csz = (ntot / nch + 15) / 16 * 16;
        for (int c0 = 0; c0 < ntot && ngrp < kWbMma; c0 += csz, ++ngrp) {
          const int n = min(csz, ntot - c0) + ((bias && c0 + csz >= ntot) ? 16 : 0);
          idw[ngrp] = idesc(1, 128, n, 1, 1);
          dcol[ngrp] = tbase + (uint32_t)c0;
          db[ngrp] = sdesc(s0 + e_off + (uint32_t)(c0 / 8) * kWbKP * 16u, 128, kWbKP * 16);
        }
      } else {
        for (int j = 0; j < nt && j < kWbMma; ++j, ++ngrp) {
          const int tap = t0 + j;
          // pixel p of the chunk, tap column dx, sits at halo column p + dx - 1 + pu
          const uint32_t boff = (uint32_t)(((tap / 3) - r0) * HX + (tap % 3) + pu - 1) * 16u;
          db[j] = sdesc(s0 + b_off + boff, 128, b_sbo);
          dcol[j] = tbase + (uint32_t)(j * cn);
          idw[j] = idesc(1, 128, cn + ((bias && j == nt - 1) ? 16 : 0), 1, 1);
        }
      }
      int s = 0;
      uint32_t ph = 0;
      for (int i = 0; i < nk; ++i) {
        if (!mbar_wait(EXP ? &split[s] : &full[s], ph, abort, p.err)) break;
        tc_fence_after();
        const uint64_t so = (uint64_t)((uint32_t)s * SB >> 4);
#pragma unroll
        for (int g = 0; g < kWbMma; ++g) {
          if (g >= ngrp) break;
#pragma unroll
          for (int k = 0; k < kKs; ++k)  // K step k: 16 pixels = 256 bytes further
            mma_f16(dcol[g], da[k] + so, db[g] + so + (uint64_t)(16 * k), idw[g],
                    (i > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
        if (++s == ns) { s = 0; ph ^= 1u; }
      }
      mma_commit(&accf);
    }
  } else {
    if constexpr (EXP) {
      // group gq = j * g8n + g8 holds tap j's view of channel group g8: pixel px of the chunk
      // at raw row (tap / 3 - r0), raw column pu - 1 + px + tap % 3. A thread's groups are the
      // same for every chunk: their raw offsets are worked out once.
      constexpr int kThr = 32 * WbWarps<EXP>::kCopy, kMax = WbWarps<EXP>::kMaxCopy;
      const int g8n = cn / 8, et = threadIdx.x - 64, n = nt * g8n * kWbKP;
      int src[kMax];
#pragma unroll
      for (int k = 0; k < kMax; ++k) {
        const int u = et + k * kThr, gq = u / kWbKP, px = u % kWbKP;
        const int j = gq / g8n, g8 = gq - j * g8n, tap = t0 + j;
        src[k] = (g8 * R + (tap / 3 - r0)) * HX + pu - 1 + px + tap % 3;
      }
      for (int i = 0; i < nk; ++i) {
        const int s = i % ns;
        if (!mbar_wait(&full[s], (i / ns) & 1, abort, p.err)) break;
        const uint4* raw = reinterpret_cast<const uint4*>(smem + s * SB + b_off);
        uint4* ex = reinterpret_cast<uint4*>(smem + s * SB + e_off);
#pragma unroll
        for (int k = 0; k < kMax; ++k)
          if (et + k * kThr < n) ex[et + k * kThr] = raw[src[k]];
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&split[s]);
      }
    }
    if (!mbar_wait(&accf, 0, abort, p.err)) mbar_drain(&accf, 0);
    tc_fence_after();
    // warps 2..: TMEM lane quarter warp % 4, column set (warp - 2) / 4 (16-column blocks dealt
    // round the sets)
    constexpr int kSets = WbWarps<EXP>::kCopy / 4;
    const int wq = warp & 3, set = (warp - 2) >> 2;
    const int o = o0 + wq * 32 + lane;
    const bool live = o < p.cout && !*abort;
    for (int j = 0; j < nt; ++j) {
      const int tap = t0 + j;
      // part[s][tap][c][o]: the warp's 32 lanes are 32 consecutive o, one 128-byte row per c
      float* dst = p.part + ((size_t)s_idx * 9 + tap) * p.cin * p.cout + (size_t)c0g * p.cout + o;
      for (int c0 = 16 * set; c0 < cn; c0 += 16 * kSets) {
        uint32_t r[16];
        tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(j * cn + c0), r);
        tmem_ld_wait();
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (N2F_IN(dst + (size_t)(c0 + q) * p.cout - p.part, p.part_cap))
            dst[(size_t)(c0 + q) * p.cout] = nk ? __uint_as_float(r[q]) : 0.f;
      }
    }
    if (bias && set == 0) {
      uint32_t r[16];
      tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(nt * cn), r);
      tmem_ld_wait();
      if (live && N2F_IN(p.bpart + (size_t)s_idx * p.cout + o - p.part, p.part_cap))
        p.bpart[(size_t)s_idx * p.cout + o] = nk ? __uint_as_float(r[0]) : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// ---- float32 weight gradient as two scaled fp16 parts per operand ---------------------------
// Float32 form: delta and x are split into scaled fp16 hi and lo parts (f16_split.cuh) and
// D = hi*hi + hi*lo + lo*hi. fp16 operands can be read MN-major, so the tap-grouped halo scheme
// of the bf16 kernel applies unchanged: TMA brings the fp32 tiles, eight split warps write the
// two fp16 images of each, one MMA warp issues three MMAs per tap and K step.
constexpr int kW3KP = 16;  // pixels per stage (one 16-element K step)
constexpr int kW3MaxStages = 12;
// split warps (then epilogue warps): 16 where the CTA holds its SM alone (TMEM: the one-row
// layers and the nine-tap C_in = 32 layers), as two teams of eight that split alternate
// chunks, so two chunks are split at once (a chunk gives each thread one to three groups: its
// latency, not its instructions, bounds it); 8, one team, for the three-tap C_in = 64 layers,
// which run two CTAs per SM
template <int R, int EXP>
struct W3Warps {
  static constexpr bool kPair = EXP && R == 1;  // two CTAs per SM
  static constexpr int kSplit = kPair ? 8 : 16;
  static constexpr int kTeams = kPair ? 1 : 2;
  static constexpr int kTeamWarps = kSplit / kTeams;
  static constexpr int kThreads = 64 + 32 * kSplit;
  static constexpr int kPerSm = kPair ? 2 : 1;
};
static_assert(kW3MaxStages % W3Warps<1, 0>::kTeams == 0 && 2 % W3Warps<1, 0>::kTeams == 0 &&
                  kW3MaxStages % W3Warps<3, 1>::kTeams == 0 && 2 % W3Warps<3, 1>::kTeams == 0,
              "float32 stage counts must stay multiples of the split team count");

// One-row layers (not tap-expanded) split in place: the fp16 hi and lo images of each pair of
// fp32 4-channel groups take that pair's two slots (hi in the first, lo in the second), so a
// stage is its raw tiles alone (about half the bytes) and twice as many stages fit; the MMA
// descriptors step two slots per 8-channel group. Tap-expanded layers write separate images.
struct W3Layout {
  uint32_t rawA, rawB, a[2], b[2], stage;
  uint32_t a_sbo, b_sbo;  // bytes between the operand images' 8-channel groups
  uint32_t ext;           // offset of the two bias groups' images (B operand, tap group 0)
};

// raw x tile pitch: the 16 chunk pixels plus pu halo pixels on each side (the kernel loads whole
// pixels, pu = 1)
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
  L.rawB = o;
  if (!exp) {  // in place: a[k] / b[k] are the first hi / lo slots
    const uint32_t slot = (uint32_t)R * w3_raw_pitch(pu) * 16;  // one 4-channel group of x
    o += align_up(rb + 4u * slot, 1024);  // + the two bias groups' hi and lo slots
    L.a[0] = L.rawA;
    L.a[1] = L.rawA + kW3KP * 16;
    L.b[0] = L.rawB;
    L.b[1] = L.rawB + slot;
    L.a_sbo = 2u * kW3KP * 16;
    L.b_sbo = 2u * slot;
    L.ext = L.rawB + (uint32_t)cin / 4 * slot;
    L.stage = o;
    return L;
  }
  o += align_up(rb, 1024);
  for (int k = 0; k < 2; ++k) { L.a[k] = o; o += align_up(pa, 1024); }
  for (int k = 0; k < 2; ++k) { L.b[k] = o; o += align_up(pb, 1024); }
  L.a_sbo = kW3KP * 16;
  L.b_sbo = (uint32_t)R * (kW3KP + 2) * 16;
  L.ext = 0;
  L.stage = o;
  return L;
}

// One 16-byte group of 8 channels: the fp32 groups lo (channels 0-3) and hi (4-7) -> the hi and
// lo fp16 images at element index u.
__device__ __forceinline__ void split2_group(const float4 c03, const float4 c47, float s,
                                             uint4* p0, uint4* p1, int u) {
  uint4 h, l;
  split_f16_group(c03, c47, s, h, l);
  p0[u] = h;
  p1[u] = l;
}

// The split of one stage, planned once per thread. Delta tile: raw [32 g4][16 px], parts
// [16 g8][16 px]; only the 8-channel groups below C_out are split (the others stay zero). x
// tile: raw [C/4][R][16 + 2 pu px], parts [C/8][R][18 px] (raw column pu - 1 + i -> part column
// i), or tap-expanded [taps x C/8][16 px]. The parts' 8-channel groups lie L.a_sbo / L.b_sbo
// bytes apart: in the in-place layout (pu = 1, one-row layers) group g8's hi and lo images take
// raw slots 2 g8 and 2 g8 + 1, the very slots the thread read them from. The layout and the
// chunk's taps are the same for every chunk, so each thread's groups -- the raw float4 index
// of their channels 0-3 (channels 4-7 lie a fixed stride on) and the part index -- are worked
// out once; a chunk's split is then loads, conversions and stores only. Consecutive threads
// take consecutive pixels of one row, so a quarter-warp's eight 16-byte reads fall in distinct
// bank groups.
template <int R, int EXP>
struct SplitPlan {
  static constexpr int kThr = 32 * W3Warps<R, EXP>::kTeamWarps;
  static constexpr int kMaxA = (16 * kW3KP + kThr - 1) / kThr;
  // x groups: tap-expanded at most 9 taps x 4 or 3 taps x 8 groups of 16 pixels; one-row at
  // most 16 groups x (16 + 2 halo) pixels
  static constexpr int kMaxB =
      EXP ? (36 * kW3KP + kThr - 1) / kThr : (16 * (kW3KP + 2) + kThr - 1) / kThr;
  int na = 0, nb = 0;
  int as[kMaxA], ad[kMaxA];
  int bs[kMaxB], bd[kMaxB];
  int bstep;  // float4 units from a group's channels 0-3 to its channels 4-7 in the raw x tile

  __device__ __forceinline__ SplitPlan(const W3Layout& L, int dgroups, int g8n, int pu, int et,
                                       int nt, int t0, int r0) {
    constexpr int PP = kW3KP + 2;  // part pitch
    const int PR = w3_raw_pitch(pu);
    bstep = R * PR;
    const int ga = (int)(L.a_sbo / 16);  // 16-byte units between the parts' groups
#pragma unroll
    for (int k = 0; k < kMaxA; ++k) {
      const int u = et + k * kThr;
      if (u < dgroups * kW3KP) {
        const int g8 = u / kW3KP, px = u % kW3KP;
        as[k] = (2 * g8) * kW3KP + px;
        ad[k] = g8 * ga + px;
        na = k + 1;  // u grows with k: the valid entries are a prefix
      }
    }
    if constexpr (EXP) {
      // group gq = j * g8n + g8 holds tap j's view of channel group g8: pixel px of the chunk
      // at raw row (tap / 3 - r0), raw column pu - 1 + px + tap % 3
      const int n = nt * g8n * kW3KP;
#pragma unroll
      for (int k = 0; k < kMaxB; ++k) {
        const int u = et + k * kThr;
        if (u < n) {
          const int gq = u / kW3KP, px = u % kW3KP;
          const int j = gq / g8n, g8 = gq - j * g8n, tap = t0 + j;
          const int r = tap / 3 - r0, col = pu - 1 + px + tap % 3;
          bs[k] = ((2 * g8) * R + r) * PR + col;
          bd[k] = u;
          nb = k + 1;
        }
      }
    } else {
      const int gb = (int)(L.b_sbo / 16);
      const int nmain = g8n * R * kW3KP, n = nmain + g8n * R * 2;
#pragma unroll
      for (int k = 0; k < kMaxB; ++k) {
        const int u = et + k * kThr;
        if (u < n) {
          int q, i;
          if (u < nmain) {
            q = u / kW3KP;
            i = 1 + u % kW3KP;
          } else {  // the 2 halo pixels of each row
            q = (u - nmain) >> 1;
            i = ((u - nmain) & 1) ? PP - 1 : 0;
          }
          const int g8 = q / R, r = q - g8 * R, px = pu - 1 + i;
          bs[k] = ((2 * g8) * R + r) * PR + px;
          bd[k] = g8 * gb + r * PP + i;
          nb = k + 1;
        }
      }
    }
  }
};

template <int R, int EXP>
__device__ __forceinline__ void split2_stage(uint8_t* st, const W3Layout& L,
                                             const SplitPlan<R, EXP>& pl, float sd, float sx) {
  const float4* rawA = reinterpret_cast<const float4*>(st + L.rawA);
  uint4* a0 = reinterpret_cast<uint4*>(st + L.a[0]);
  uint4* a1 = reinterpret_cast<uint4*>(st + L.a[1]);
#pragma unroll
  for (int k = 0; k < SplitPlan<R, EXP>::kMaxA; ++k)
    if (k < pl.na) split2_group(rawA[pl.as[k]], rawA[pl.as[k] + kW3KP], sd, a0, a1, pl.ad[k]);
  const float4* rawB = reinterpret_cast<const float4*>(st + L.rawB);
  uint4* b0 = reinterpret_cast<uint4*>(st + L.b[0]);
  uint4* b1 = reinterpret_cast<uint4*>(st + L.b[1]);
#pragma unroll
  for (int k = 0; k < SplitPlan<R, EXP>::kMaxB; ++k)
    if (k < pl.nb) split2_group(rawB[pl.bs[k]], rawB[pl.bs[k] + pl.bstep], sx, b0, b1, pl.bd[k]);
}

template <int R, int EXP>
__global__ void __launch_bounds__(W3Warps<R, EXP>::kThreads, W3Warps<R, EXP>::kPerSm) k_wgrad_tc_f32(const __grid_constant__ CUtensorMap tmD,
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
  // both tiles come by whole-pixel box rows (make_map_rows): x with one halo pixel each side
  const W3Layout L = w3_layout(cn, R, 1, EXP, nt);
  const uint32_t RB = (uint32_t)cn * R * w3_raw_pitch(1) * 4;
  const bool bias = grp == 0;
  const uint32_t ncols = tmem_cols(nt * cn + (bias ? 16 : 0));
  // delta's 8-channel groups that hold output channels (the rest of the M = 128 rows is zero)
  const int dgroups = min(16, (p.cout - o0 + 7) / 8);
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&split[s], W3Warps<R, EXP>::kTeamWarps);
    }
    mbar_init(&accf, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&tslot, ncols);
  if (EXP && dgroups < 16) {
    // separate delta part images: the groups never split are zeroed once (in place, the TMA
    // box's zero fill beyond C_out leaves zero parts in those slots every chunk)
    const uint32_t gbytes = kW3KP * 16, ga = L.a_sbo;
    for (int s = 0; s < ns; ++s)
      for (int q = 0; q < 2; ++q)
        for (int g8 = dgroups; g8 < 16; ++g8)
          fill_ext(smem + s * L.stage + L.a[q] + g8 * ga, gbytes, 0u);
  }
  if (bias) {  // hi part: ones, lo part: zeros, so the bias columns sum a_hi + a_lo
    if (EXP) {
      const uint32_t eo = (uint32_t)nt * cn / 8 * kW3KP * 16, eb = 2u * kW3KP * 16;
      for (int s = 0; s < ns; ++s)
        for (int q = 0; q < 2; ++q)
          fill_ext(smem + s * L.stage + L.b[q] + eo, eb, q == 0 ? kF16PairOne : 0u);
    } else {  // in place: the two bias groups' hi, lo, hi, lo slots after the raw x tile
      const uint32_t slot = L.b_sbo / 2;
      for (int s = 0; s < ns; ++s)
        for (int k = 0; k < 4; ++k)
          fill_ext(smem + s * L.stage + L.ext + k * slot, slot, (k & 1) ? 0u : kF16PairOne);
    }
  }
  fence_proxy_async();  // the fills above are read by the MMAs (async proxy)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0, s = 0, y = cbeg / p.chunks_x, cx = cbeg - y * p.chunks_x;
      uint32_t ph = 0;
      for (int i = 0; i < nk; ++i) {
        if (i >= ns && !mbar_wait(&empty[s], ph ^ 1u, abort, p.err)) break;
        const int x0 = cx * kW3KP;
        uint8_t* st = smem + s * L.stage;
        mbar_expect_tx(&full[s], 128u * kW3KP * 4 + RB);
        tma_load_3d(st + L.rawA, &tmD, &full[s], 4 * x0, y, o0 / 4);
        tma_load_3d(st + L.rawB, &tmX, &full[s], 4 * (x0 - 1), y + r0 - 1, c0g / 4);
        issued = i + 1;
        if (++cx == p.chunks_x) { cx = 0; ++y; }
        if (++s == ns) { s = 0; ph ^= 1u; }
      }
      if (*abort)
        for (int i = issued > ns ? issued - ns : 0; i < issued; ++i)
          mbar_drain(&full[i % ns], (i / ns) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // Every MMA's descriptors and instruction word are fixed up front for stage 0; stage s
      // adds (s x stage bytes) / 16 to the start-address field (addresses stay below 2^18, so
      // the 14-bit field never carries). Up to kW3Mma MMA groups per chunk: the taps of the
      // group (one row) or, tap-expanded, the column chunks of at most 256.
      constexpr int kW3Mma = EXP ? 2 : 3;
      const uint32_t a_sbo = L.a_sbo;  // next 8-channel group of delta
      const uint32_t b_sbo = L.b_sbo;  // next 8-channel group of x
      const uint32_t s0 = smem_u32(smem);
      uint64_t da[2], db[kW3Mma][2];
      uint32_t dcol[kW3Mma], idw[kW3Mma];
      int ngrp = 0;
#pragma unroll
      for (int k = 0; k < 2; ++k) da[k] = sdesc(s0 + L.a[k], 128, a_sbo);
      if constexpr (EXP) {
        const int ntot = nt * cn, nch = (ntot + 255) / 256;
        const int csz = (ntot / nch + 15) / 16 * 16;
        for (int c0 = 0; c0 < ntot && ngrp < kW3Mma; c0 += csz, ++ngrp) {
          const int n = min(csz, ntot - c0) + ((bias && c0 + csz >= ntot) ? 16 : 0);
          idw[ngrp] = idesc(0, 128, n, 1, 1);
          dcol[ngrp] = tbase + (uint32_t)c0;
          for (int q = 0; q < 2; ++q)
            db[ngrp][q] = sdesc(s0 + L.b[q] + (uint32_t)(c0 / 8) * kW3KP * 16u, 128, kW3KP * 16);
        }
      } else {
        for (int j = 0; j < nt && j < kW3Mma; ++j, ++ngrp) {
          const int tap = t0 + j;
          const uint32_t boff = (uint32_t)(((tap / 3) - r0) * (kW3KP + 2) + (tap % 3)) * 16u;
          for (int k = 0; k < 2; ++k) db[j][k] = sdesc(s0 + L.b[k] + boff, 128, b_sbo);
          dcol[j] = tbase + (uint32_t)(j * cn);
          idw[j] = idesc(0, 128, cn + ((bias && j == nt - 1) ? 16 : 0), 1, 1);
        }
      }
      int s = 0;
      uint32_t ph = 0;
      for (int i = 0; i < nk; ++i) {
        if (!mbar_wait(&split[s], ph, abort, p.err)) break;
        tc_fence_after();
        const uint64_t so = (uint64_t)((uint32_t)s * L.stage >> 4);
        const uint32_t acc0 = i > 0 ? 1u : 0u;
#pragma unroll
        for (int g = 0; g < kW3Mma; ++g) {
          if (g >= ngrp) break;
          mma_f16(dcol[g], da[0] + so, db[g][0] + so, idw[g], acc0);
          mma_f16(dcol[g], da[0] + so, db[g][1] + so, idw[g], 1u);
          mma_f16(dcol[g], da[1] + so, db[g][0] + so, idw[g], 1u);
        }
        mma_commit(&empty[s]);
        if (++s == ns) { s = 0; ph ^= 1u; }
      }
      mma_commit(&accf);
    }
  } else {
    constexpr int kTT = 32 * W3Warps<R, EXP>::kTeamWarps;  // threads per team
    const int team = (threadIdx.x - 64) / kTT, et = (threadIdx.x - 64) % kTT;
    const float sd = f16_scale(p.dmax), sx = f16_scale(p.xmax);
    const SplitPlan<R, EXP> plan(L, dgroups, cn / 8, 1, et, nt, t0, r0);
    int s = 0;
    uint32_t ph = 0;
    for (int i = 0; i < nk; ++i) {
      if (i % W3Warps<R, EXP>::kTeams == team) {  // this team's chunk
        if (!mbar_wait(&full[s], ph, abort, p.err)) break;
        uint8_t* st = smem + s * L.stage;
        split2_stage<R, EXP>(st, L, plan, sd, sx);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&split[s]);
      }
      if (++s == ns) { s = 0; ph ^= 1u; }
    }
    if (!mbar_wait(&accf, 0, abort, p.err)) mbar_drain(&accf, 0);
    tc_fence_after();
    // warps 2..: TMEM lane quarter warp % 4, column set (warp - 2) / 4 (16-column blocks are
    // dealt round the sets)
    constexpr int kSets = W3Warps<R, EXP>::kSplit / 4;
    const int wq = warp & 3, half = (warp - 2) >> 2;
    const int o = o0 + wq * 32 + lane;
    const bool live = o < p.cout && !*abort;
    // undo the operand scales (exact powers of two, applied one at a time)
    const float ud = f16_unscale(p.dmax), ux = f16_unscale(p.xmax);
    for (int j = 0; j < nt; ++j) {
      const int tap = t0 + j;
      // part[s][tap][c][o]: the warp's 32 lanes are 32 consecutive o, one 128-byte row per c
      float* dst = p.part + ((size_t)s_idx * 9 + tap) * p.cin * p.cout + (size_t)c0g * p.cout + o;
      for (int c0 = 16 * half; c0 < cn; c0 += 16 * kSets) {
        uint32_t r[16];
        tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(j * cn + c0), r);
        tmem_ld_wait();
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (N2F_IN(dst + (size_t)(c0 + q) * p.cout - p.part, p.part_cap))
            dst[(size_t)(c0 + q) * p.cout] = nk ? __uint_as_float(r[q]) * ud * ux : 0.f;
      }
    }
    if (bias && half == 0) {
      uint32_t r[16];
      tmem_ld16(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(nt * cn), r);
      tmem_ld_wait();
      if (live && N2F_IN(p.bpart + (size_t)s_idx * p.cout + o - p.part, p.part_cap))
        p.bpart[(size_t)s_idx * p.cout + o] = nk ? __uint_as_float(r[0]) * ud : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// gw[(o*C_in + c)*9 + tap] = sum over s of part[s][tap][c][o], and gb[o] = sum over s of
// bpart[s][o]. Work unit: four consecutive o of one (tap, c) row (a float4 of every split's
// slab). A block's eight warps form kRwGroups(S) split ranges x (8 / that) unit groups of 32
// units; each thread sums its unit over its contiguous range of splits in split order (four
// loads in flight), and the ranges' sums are then added in range order, so the result is fixed
// for a given number of splits. The S loads of a unit are spread over up to eight warps so that
// the many-split layers (small C) do not wait on one long chain of loads. The last blocks do the
// bias partials the same way.
__host__ __device__ inline int kRwGroups(int S) { return S >= 32 ? 8 : S >= 16 ? 4 : S >= 8 ? 2 : 1; }

__global__ void __launch_bounds__(256) k_reduce_wgrad_tc(const float* __restrict__ part, int S,
                                                         int cin, int cout,
                                                         float* __restrict__ gw,
                                                         const float* __restrict__ bpart,
                                                         float* __restrict__ gb, int wblocks,
                                                         size_t part_cap, const int* skip) {
  if (skip && *skip) return;
  __shared__ float4 red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int R = kRwGroups(S), UG = 8 / R;  // split ranges, unit groups per block
  const int r = w % R, ug = w / R;
  const bool bias = (int)blockIdx.x >= wblocks;
  const int blk = bias ? (int)blockIdx.x - wblocks : (int)blockIdx.x;
  const size_t per4 = bias ? (size_t)cout / 4 : (size_t)9 * cin * cout / 4;  // units per split
  const float4* src = reinterpret_cast<const float4*>(bias ? bpart : part);
  const size_t u = ((size_t)blk * UG + ug) * 32 + lane;
  const int s0 = (int)((long)S * r / R), s1 = (int)((long)S * (r + 1) / R);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  // float4 units of the workspace from src on
  const size_t cap4 = (part_cap - (size_t)((bias ? bpart : part) - part)) / 4;
  if (u < per4 && N2F_IN((size_t)(s1 > 0 ? s1 - 1 : 0) * per4 + u, cap4)) {
    const float4* q = src + u;
    int k = s0;
    for (; k + 4 <= s1; k += 4) {
      const float4 a = q[(size_t)k * per4], b = q[(size_t)(k + 1) * per4],
                   c = q[(size_t)(k + 2) * per4], d = q[(size_t)(k + 3) * per4];
      acc.x = (((acc.x + a.x) + b.x) + c.x) + d.x;
      acc.y = (((acc.y + a.y) + b.y) + c.y) + d.y;
      acc.z = (((acc.z + a.z) + b.z) + c.z) + d.z;
      acc.w = (((acc.w + a.w) + b.w) + c.w) + d.w;
    }
    for (; k < s1; ++k) {
      const float4 a = q[(size_t)k * per4];
      acc.x += a.x;
      acc.y += a.y;
      acc.z += a.z;
      acc.w += a.w;
    }
  }
  red[w][lane] = acc;
  __syncthreads();
  if (r != 0 || u >= per4) return;
  float4 v = red[ug * R][lane];
  for (int k = 1; k < R; ++k) {
    const float4 a = red[ug * R + k][lane];
    v.x += a.x;
    v.y += a.y;
    v.z += a.z;
    v.w += a.w;
  }
  if (bias) {  // gb comes from the caller at the op-level entry points: align before a float4 store
    if ((reinterpret_cast<uintptr_t>(gb) & 15u) == 0) {
      reinterpret_cast<float4*>(gb)[u] = v;
    } else {
      gb[4 * u] = v.x;
      gb[4 * u + 1] = v.y;
      gb[4 * u + 2] = v.z;
      gb[4 * u + 3] = v.w;
    }
    return;
  }
  // unit u = (tap * C_in + c) * (C_out / 4) + o / 4
  const size_t row = u / ((size_t)cout / 4);
  const int o = (int)(u - row * ((size_t)cout / 4)) * 4;
  const int tap = (int)(row / cin), c = (int)(row - (size_t)tap * cin);
  const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (N2F_IN(((size_t)(o + j) * cin + c) * 9 + tap, (size_t)9 * cin * cout))
      gw[((size_t)(o + j) * cin + c) * 9 + tap] = vv[j];
}

// Grid of k_reduce_wgrad_tc: weight blocks, then bias blocks.
inline void reduce_grid(int S, int cin, int cout, int* wblocks, int* total) {
  const int per_block = 32 * (8 / kRwGroups(S));  // units per block
  const size_t uw = (size_t)9 * cin * cout / 4, ub = (size_t)cout / 4;
  *wblocks = (int)((uw + per_block - 1) / per_block);
  *total = *wblocks + (int)((ub + per_block - 1) / per_block);
}

}  // namespace


// Sets the dynamic shared-memory limit of every weight-gradient kernel (the per-block opt-in total
// minus its static shared memory), so that later launches (possibly inside a stream capture)
// need no attribute calls.
cudaError_t wgrad_tc_prepare() {
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
    set((const void*)k_wgrad_tc_bf16<0>);
    set((const void*)k_wgrad_tc_bf16<1>);
    set((const void*)k_wgrad_tc_f32<1, 0>);
    set((const void*)k_wgrad_tc_f32<1, 1>);
    set((const void*)k_wgrad_tc_f32<3, 1>);
  return e;
}

bool tc_wgrad_supported(int cin, int cout, int bf16) {
  (void)bf16;
  return tc_supported(cin, cout);
}

// bf16 = 1: bf16 maps, k_wgrad_tc_bf16; bf16 = 0: float32 maps, k_wgrad_tc_f32 (two fp16 parts)
static cudaError_t launch_wgrad_grouped(int bf16, const void* dout, const void* in, int cin,
                                        int cout, int H, int W, const unsigned* dmax,
                                        const unsigned* xmax, float* part, size_t part_cap,
                                        float* gw, float* gb, const int* skip, int* err,
                                        cudaStream_t st) {
  if (!bf16 && (!dmax || !xmax)) return cudaErrorInvalidValue;
  const TapGroups tg = tap_groups(cin);
  const int KP = bf16 ? kWbKP : kW3KP, GE = bf16 ? 8 : 4;
  // bf16: pixels per TMA unit, up to 8 (128-byte box rows; the halo grows by 14 pixels of 66)
  int pu = 1;
  while (bf16 && pu < 8 && W % (2 * pu) == 0) pu *= 2;
  CUtensorMap md, mx;
  // bf16 tiles by pu-pixel units (128-byte box rows); float32 tiles by whole-pixel box rows (one
  // row of 16 or 18 pixels per channel group and image row, no halo units)
  cudaError_t e = bf16 ? make_map(&md, dout, bf16, cout, H, W, KP / pu, 1, 128 / GE, pu)
                       : make_map_rows(&md, dout, cout, H, W, KP, 1, 128 / 4);
  if (e == cudaSuccess)
    e = bf16 ? make_map(&mx, in, bf16, cin, H, W, KP / pu + 2, tg.R, tg.cn / GE, pu)
             : make_map_rows(&mx, in, cin, H, W, KP + 2, tg.R, tg.cn / 4);
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
  p.dmax = dmax;
  p.xmax = xmax;
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
  // a float32 split thread's x groups must fit its plan (SplitPlan::kMaxB): at most 36
  // tap-expanded 8-channel groups, or 16 groups of one row
  if (!bf16 && (exp ? tg.count[0] * tg.cn / 8 > 36 : tg.cn / 8 * tg.R > 16))
    return cudaErrorInvalidValue;
  const uint32_t sb = bf16 ? (exp ? wb_stage_exp(tg.cn, tg.R, pu, tg.count[0]) : wb_stage(tg.cn, tg.R, pu))
                           : w3_layout(tg.cn, tg.R, 1, exp, tg.count[0]).stage;
  const int max_stages = bf16 ? kWbMaxStages : kW3MaxStages;
  p.stages = (int)((227u * 1024u / (uint32_t)max_res - 2048u) / sb);
  if (p.stages > max_stages) p.stages = max_stages;
  // float32 layers with two split teams: team k takes chunks i = k (mod teams); a team's next
  // chunk reuses the stage of chunk (next - stages), which must be one of its own (already
  // waited for) or its parity wait could see that older load's phase: stages a multiple of the
  // team count
  const int teams = bf16 ? 1 : tg.R == 3 ? W3Warps<3, 1>::kTeams
                                         : exp ? W3Warps<1, 1>::kTeams : W3Warps<1, 0>::kTeams;
  p.stages -= p.stages % teams;
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
  p.part_cap = part_cap;
  p.bpart = part + ((size_t)S * per_split_elems + 63) / 64 * 64;
  p.skip = skip;
  p.err = err;
  const dim3 grid((unsigned)otiles, (unsigned)tg.n, (unsigned)S);
  if (bf16 && exp)
    k_wgrad_tc_bf16<1><<<grid, WbWarps<1>::kThreads, smem, st>>>(md, mx, p);
  else if (bf16)
    k_wgrad_tc_bf16<0><<<grid, WbWarps<0>::kThreads, smem, st>>>(md, mx, p);
  else if (tg.R == 3)
    k_wgrad_tc_f32<3, 1><<<grid, W3Warps<3, 1>::kThreads, smem, st>>>(md, mx, p);
  else if (exp)
    k_wgrad_tc_f32<1, 1><<<grid, W3Warps<1, 1>::kThreads, smem, st>>>(md, mx, p);
  else
    k_wgrad_tc_f32<1, 0><<<grid, W3Warps<1, 0>::kThreads, smem, st>>>(md, mx, p);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // weights, and (last blocks) the bias from the S per-split sums of tap group 0
  int wblocks = 0, rblocks = 0;
  reduce_grid(S, cin, cout, &wblocks, &rblocks);
  k_reduce_wgrad_tc<<<(unsigned)rblocks, 256, 0, st>>>(part, S, cin, cout, gw, p.bpart, gb,
                                                       wblocks, part_cap, skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_wgrad_tc(int bf16, const void* dout, const void* in, int cin, int cout, int H,
                            int W, const unsigned* dmax, const unsigned* xmax, float* part,
                            size_t part_cap, float* gw, float* gb, const int* skip, int* err,
                            cudaStream_t st) {
  if (!tc_wgrad_supported(cin, cout, bf16)) return cudaErrorNotSupported;
  if (const cudaError_t pe = tc_prepare()) return pe;
  return launch_wgrad_grouped(bf16, dout, in, cin, cout, H, W, dmax, xmax, part, part_cap, gw, gb,
                              skip, err, st);
}

N2F_CHECK_READER(check_read_wgrad)

}  // namespace n2f
