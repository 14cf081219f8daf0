// a11 (training of the learned proposal; not in the paper): weight gradient of a 128 -> 128
// convolution layer on the fifth-generation tensor cores,
//   dw[t][ci][co] += sum over sequences n and positions p of in[n][p + t - 3][ci] * g[n][p][co],
// for the seven taps t, as a GEMM per tap with M = 128 input channels, N = 128 output channels
// and K = positions.
//
// Layout: activations and gradients are BF16 rows [sequence][position + 3][128 channels] (three
// zero halo rows on either side), so a tile of positions is already "MN-major" for the MMA:
// channels contiguous, positions strided.  A CTA owns a run of 128-position tiles and a group of
// taps (0-3 or 4-6) whose FP32 accumulators (128 columns each) fill the tensor memory.  One
// thread stages each tile with TMA tensor copies into a three-stage ring, two tiles ahead of
// the MMAs: 16 boxes of 8 channels x 131 input rows (the tile's positions shifted by the
// group's first tap, plus the group's other tap shifts) and 16 boxes of 8 channels x 128
// gradient rows; box c lands at c * stride, so that each 16-byte chunk (8 channels of one
// row) sits at channel-group * stride + row * 16, rows are 16 bytes apart throughout, and a
// tap's shift is a start-address offset of 16 bytes per row.  The same thread issues, per
// tap, eight tcgen05.mma (K = 16 positions each) and commits them on the stage's mbarrier,
// which the next copy into that stage waits for.  The CTAs of the three-tap group also
// accumulate the bias gradient db[co] = sum over positions of g[p][co] in their free fourth
// accumulator, as one more MMA per K-step with an operand of ones (every row of that
// accumulator is the column sum).  At the end the four warps read their 32 accumulator lanes
// (input channels) back and add them to dw with 16-byte FP32 atomics along the output
// channels.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"
#include "prop.h"
#include "tc.cuh"

namespace mss {

namespace {

constexpr int kWgThreads = 128;
constexpr int kWgTile = 128;                              // positions per tile (MMA K total)
constexpr int kWgTapsPerCta = 4;                          // 4 x 128 FP32 columns = all of TMEM
constexpr int kWgARows = 136;                             // 128 + 3 tap shifts, padded to 8
constexpr int kWgABox = 131;                              // rows copied: 128 + 3 tap shifts
constexpr uint32_t kWgAStride = kWgARows * 16;            // bytes between 8-channel groups of A
constexpr uint32_t kWgBStride = kWgTile * 16;             // the same for B
constexpr uint32_t kWgABytes = 16 * kWgAStride;           // 34,816
constexpr uint32_t kWgBBytes = 16 * kWgBStride;           // 32,768
constexpr uint32_t kWgStage = kWgABytes + kWgBBytes;
constexpr uint32_t kWgTx = 16 * (kWgABox + kWgTile) * 16; // bytes landing per tile
constexpr int kWgStages = 3;                              // copies two tiles ahead
constexpr uint32_t kWgOnes = kWgStages * kWgStage;         // 4 KB of BF16 ones (bias operand)
constexpr uint32_t kWgOnesBytes = 4096;
constexpr uint32_t kWgSmem = kWgOnes + kWgOnesBytes + 64;  // stages, ones, mbarriers, TMEM slot
constexpr uint64_t kWgWaitNs = 2000000000ull;
static_assert(kWgAStride % 128 == 0 && kWgBStride % 128 == 0 && kWgStage % 128 == 0, "TMA destinations");
// MN-major operands without swizzling: core matrices of 8 rows (K) x 16 bytes (8 MN
// elements); the descriptor's leading offset is the distance between core matrices adjacent
// in K (8 rows = 128 B here), its stride offset the distance between core matrices adjacent in
// MN (checked on GB300 with a single MMA of known integers against both assignments, and with a
// start address inside a core matrix, which the tap shift uses).
constexpr uint32_t kWgCoreK = 128;
// instruction descriptor: BF16 x BF16 -> FP32, M = N = 128, A and B MN-major (bits 15, 16)
constexpr uint32_t kWgIdesc = idesc_bf16_f32(128, 128) | (1u << 15) | (1u << 16);

// 2-D tiled TMA load (channel x, row y) completing on bar
__device__ __forceinline__ void tma_tile_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(kWgThreads, 1)
    k_conv_wgrad_tc(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tg,
                    const int32_t* __restrict__ lens, float* __restrict__ dw, float* __restrict__ db,
                    int32_t n_seq, int32_t rows,
                    int32_t tiles_per_cta, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kWgOnes + kWgOnesBytes);      // [kWgStages]
  uint64_t* done = full + kWgStages;                                              // [kWgStages]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(done + kWgStages);
  uint32_t* s_issued = s_tmem + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t0 = blockIdx.y * kWgTapsPerCta;
  const int ntaps = min(kWgTapsPerCta, kPropTaps - t0);
  const int tiles_per_seq = (rows - 6) / kWgTile;
  const int64_t total = (int64_t)n_seq * tiles_per_seq;
  const int64_t first = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t last = min(total, first + tiles_per_cta);
  // the three-tap group's free accumulator (columns 384 ..) takes the bias gradient
  const bool with_bias = db != nullptr && ntaps < kWgTapsPerCta;
  for (int e = tid; e < (int)(kWgOnesBytes / 4); e += kWgThreads)
    reinterpret_cast<uint32_t*>(sm + kWgOnes)[e] = 0x3F803F80u;  // BF16 1.0, 1.0
  fence_proxy_async_smem();

  if (tid == 0) {
    for (int k = 0; k < kWgStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&done[k], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(s_tmem, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (tid == 0) {
    // tiles past a sequence's length carry zero gradients: skip them
    auto next_live = [&](int64_t tile) {
      while (tile < last) {
        const int n = (int)(tile / tiles_per_seq);
        if ((int)(tile - (int64_t)n * tiles_per_seq) * kWgTile < lens[n]) break;
        ++tile;
      }
      return tile;
    };
    // live tile k goes to stage k mod kWgStages: input rows p0 + t0 .. + 130 (buffer rows; the
    // rows past what this group's taps read are never multiplied) and gradient rows p0 + 3 ..
    auto stage_copy = [&](int64_t tile, int s) {
      const int n = (int)(tile / tiles_per_seq);
      const int p0 = (int)(tile - (int64_t)n * tiles_per_seq) * kWgTile;
      const uint32_t sA = smem_u32(sm + s * kWgStage), sB = sA + kWgABytes;
      mbar_arrive_expect_tx(&full[s], kWgTx);
      const int32_t ya = n * rows + p0 + t0, yb = n * rows + p0 + 3;
      for (int c = 0; c < 16; ++c) {
        tma_tile_2d(sA + c * kWgAStride, &tin, 8 * c, ya, &full[s]);
        tma_tile_2d(sB + c * kWgBStride, &tg, 8 * c, yb, &full[s]);
      }
    };
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tin)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tg)) : "memory");
    bool ok = true;
    int64_t fetch = next_live(first);
    int copied = 0, issued = 0;
    for (int k = 0; k < kWgStages - 1 && fetch < last; ++k) {
      stage_copy(fetch, k);
      fetch = next_live(fetch + 1);
      ++copied;
    }
    while (issued < copied) {
      const int s = issued % kWgStages;
      if (fetch < last) {
        // copied == issued + kWgStages - 1: the stage to refill was last read by tile issued - 1
        if (issued >= 1)
          ok = mbar_wait(&done[(issued - 1) % kWgStages], (uint32_t)(((issued - 1) / kWgStages) & 1), kWgWaitNs);
        if (!ok) break;
        stage_copy(fetch, copied % kWgStages);
        fetch = next_live(fetch + 1);
        ++copied;
      }
      ok = mbar_wait(&full[s], (uint32_t)((issued / kWgStages) & 1), kWgWaitNs);
      if (!ok) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sm + s * kWgStage), b0 = a0 + kWgABytes;
      for (int j = 0; j < ntaps; ++j) {
#pragma unroll
        for (int kk = 0; kk < kWgTile / 16; ++kk)
          tc_mma_bf16(tmem + (uint32_t)(j * 128), smem_desc(a0 + (uint32_t)(j + 16 * kk) * 16, kWgCoreK, kWgAStride),
                      smem_desc(b0 + (uint32_t)(16 * kk) * 16, kWgCoreK, kWgBStride), kWgIdesc,
                      (issued > 0 || kk > 0) ? 1u : 0u);
      }
      if (with_bias) {
        // ones [K = 16 positions][M = 128]: any layout of the 4 KB of ones; leading offset
        // 128 B, stride offset 256 B keep the 2 x 16 core matrices inside it
        const uint64_t ones = smem_desc(smem_u32(sm + kWgOnes), kWgCoreK, 256);
#pragma unroll
        for (int kk = 0; kk < kWgTile / 16; ++kk)
          tc_mma_bf16(tmem + (uint32_t)(kWgTapsPerCta - 1) * 128, ones,
                      smem_desc(b0 + (uint32_t)(16 * kk) * 16, kWgCoreK, kWgBStride), kWgIdesc,
                      (issued > 0 || kk > 0) ? 1u : 0u);
      }
      tc_commit(&done[s]);
      ++issued;
    }
    // wait (bounded) for the last committed tile of each stage and for every copy armed
    bool drained = true;
    for (int k = issued - 1; k >= 0 && k >= issued - kWgStages; --k)
      if (!mbar_wait(&done[k % kWgStages], (uint32_t)((k / kWgStages) & 1), kWgWaitNs)) drained = false;
    for (int k = issued; k < copied; ++k)
      if (!mbar_wait(&full[k % kWgStages], (uint32_t)((k / kWgStages) & 1), kWgWaitNs)) drained = false;
    if (!ok || !drained) {
      atomicOr(err, ERR_TIMEOUT);
      issued = -1;
    }
    *s_issued = (uint32_t)issued;
  }
  __syncthreads();
  const int issued = (int)*s_issued;
  if (issued > 0) {
    // every MMA has completed and no copy is in flight: the stage buffers are free.  Each
    // warp turns its 32 x 32 blocks (thread = input channel) around in shared memory (rows
    // padded to 33 floats) so that its atomic adds are 16-byte vectors along the output
    // channels: a warp instruction covers 4 rows x 128 contiguous bytes.
    tc_fence_after();
    float* st = reinterpret_cast<float*>(sm) + warp * 32 * 33;
    for (int j = 0; j < ntaps; ++j) {
      float* dwt = dw + (int64_t)(t0 + j) * kPropC * kPropC + (int64_t)(warp * 32) * kPropC;
      for (int c = 0; c < 128; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 128 + c), r);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 32; ++q) st[lane * 33 + q] = __uint_as_float(r[q]);
        __syncwarp();
        const int c4 = 4 * (lane & 7);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = (lane >> 3) + 4 * k;
          const float* row = st + i * 33 + c4;
          atomicAdd(reinterpret_cast<float4*>(dwt + (int64_t)i * kPropC + c + c4),
                    make_float4(row[0], row[1], row[2], row[3]));
        }
        __syncwarp();
      }
    }
  }
  if (issued > 0 && with_bias && warp == 0) {  // row 0 of the ones accumulator: lane 0 of warp 0
    for (int c = 0; c < 128; c += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + (uint32_t)(kWgTapsPerCta - 1) * 128 + (uint32_t)c, r);
      tmem_wait_ld();
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 32; ++q) atomicAdd(db + c + q, __uint_as_float(r[q]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// First-layer gradients on the tensor cores: dw1[4t + b][co] += sum over positions p of
// [x[p + t - 3] = b] * g[p][co] and db1[co] += sum of g[p][co], as the GEMM
// D[f][co] = sum_p F[p][f] g[p][co] with the one-hot features F (f = 4t + b < 28, f = 28 all
// ones, the rest zero) as an MN-major A operand built from the codes (M = 128, rows 29.. zero)
// and the gradient tiles as B, staged by TMA exactly as for the other layers.  Warps 1-3 build
// A; thread 0 stages B and issues the 8 MMAs per tile into one 128-column accumulator.
constexpr int kL1gStages = 3;
constexpr uint32_t kL1gSmem = kL1gStages * kWgStage + 128;

__global__ void __launch_bounds__(kWgThreads, 1)
    k_l1_wgrad_tc(const __grid_constant__ CUtensorMap tg, const uint8_t* __restrict__ codes, int32_t ld,
                  const int32_t* __restrict__ lens, float* __restrict__ dw1, float* __restrict__ db1, int32_t n_seq,
                  int32_t rows, int32_t tiles_per_cta, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kL1gStages * kWgStage);  // [3] B landed
  uint64_t* built = full + kL1gStages;                                       // [3] A built (3 warps)
  uint64_t* done = built + kL1gStages;                                       // [3] MMAs completed
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(done + kL1gStages);
  uint32_t* s_issued = s_tmem + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_per_seq = (rows - 6) / kWgTile;
  const int64_t total = (int64_t)n_seq * tiles_per_seq;
  const int64_t first = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t last = min(total, first + tiles_per_cta);
  if (tid == 0) {
    for (int k = 0; k < kL1gStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&built[k], 3);
      mbar_init(&done[k], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(s_tmem, 128);
    tmem_relinquish();
  }
  // the feature rows 32 .. 127 of every stage's A stay zero
  for (int e = tid; e < kL1gStages * 12 * (int)kWgAStride / 16; e += kWgThreads) {
    const int st = e / (12 * (int)kWgAStride / 16), rem = e - st * (12 * (int)kWgAStride / 16);
    *reinterpret_cast<uint4*>(sm + st * kWgStage + 4 * kWgAStride + rem * 16) = make_uint4(0, 0, 0, 0);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  auto next_live = [&](int64_t tile) {
    while (tile < last) {
      const int n = (int)(tile / tiles_per_seq);
      if ((int)(tile - (int64_t)n * tiles_per_seq) * kWgTile < lens[n]) break;
      ++tile;
    }
    return tile;
  };

  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tg)) : "memory");
    bool ok = true;
    int issued = 0, copied = 0;
    int64_t fetch = next_live(first);
    auto stage_copy = [&](int64_t tile, int s) {
      const int n = (int)(tile / tiles_per_seq);
      const int p0 = (int)(tile - (int64_t)n * tiles_per_seq) * kWgTile;
      const uint32_t sB = smem_u32(sm + s * kWgStage) + kWgABytes;
      mbar_arrive_expect_tx(&full[s], 16 * kWgTile * 16);
      for (int c = 0; c < 16; ++c) tma_tile_2d(sB + c * kWgBStride, &tg, 8 * c, n * rows + p0 + 3, &full[s]);
    };
    for (int k = 0; k < kL1gStages - 1 && fetch < last; ++k) {
      stage_copy(fetch, k);
      fetch = next_live(fetch + 1);
      ++copied;
    }
    while (issued < copied) {
      const int s = issued % kL1gStages;
      if (fetch < last) {
        if (issued >= 1)
          ok = mbar_wait(&done[(issued - 1) % kL1gStages], (uint32_t)(((issued - 1) / kL1gStages) & 1), kWgWaitNs);
        if (!ok) break;
        stage_copy(fetch, copied % kL1gStages);
        fetch = next_live(fetch + 1);
        ++copied;
      }
      const uint32_t par = (uint32_t)((issued / kL1gStages) & 1);
      ok = mbar_wait(&full[s], par, kWgWaitNs) && mbar_wait(&built[s], par, kWgWaitNs);
      if (!ok) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sm + s * kWgStage), b0 = a0 + kWgABytes;
#pragma unroll
      for (int kk = 0; kk < kWgTile / 16; ++kk)
        tc_mma_bf16(tmem, smem_desc(a0 + (uint32_t)(16 * kk) * 16, kWgCoreK, kWgAStride),
                    smem_desc(b0 + (uint32_t)(16 * kk) * 16, kWgCoreK, kWgBStride), kWgIdesc,
                    (issued > 0 || kk > 0) ? 1u : 0u);
      tc_commit(&done[s]);
      ++issued;
    }
    bool drained = true;
    for (int k = issued - 1; k >= 0 && k >= issued - kL1gStages; --k)
      if (!mbar_wait(&done[k % kL1gStages], (uint32_t)((k / kL1gStages) & 1), kWgWaitNs)) drained = false;
    for (int k = issued; k < copied; ++k)
      if (!mbar_wait(&full[k % kL1gStages], (uint32_t)((k / kL1gStages) & 1), kWgWaitNs)) drained = false;
    if (!ok || !drained) {
      atomicOr(err, ERR_TIMEOUT);
      issued = -1;
    }
    *s_issued = (uint32_t)issued;
  } else if (warp >= 1) {
    // A builders: live tile k in stage k mod 3; chunk (row r = position p0 + r, feature group
    // c < 4) holds features 8c .. 8c + 7 (taps 2c and 2c + 1; group 3: tap 6 and the ones)
    bool ok = true;
    int k = 0;
    for (int64_t tile = next_live(first); tile < last; tile = next_live(tile + 1), ++k) {
      const int s = k % kL1gStages;
      if (k >= kL1gStages && ok)
        ok = __all_sync(0xffffffffu,
                        mbar_wait(&done[s], (uint32_t)(((k - kL1gStages) / kL1gStages) & 1), kWgWaitNs));
      if (ok) {
        const int n = (int)(tile / tiles_per_seq);
        const int p0 = (int)(tile - (int64_t)n * tiles_per_seq) * kWgTile;
        const int len = lens[n];
        const uint8_t* cn = codes + (int64_t)n * ld;
        uint8_t* a = sm + s * kWgStage;
        for (int e = tid - 32; e < kWgTile * 4; e += kWgThreads - 32) {
          const int r = e >> 2, c = e & 3;
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int t = 2 * c + h, q = p0 + r + t - 3;
            uint32_t cd = (t < kPropTaps && q >= 0 && q < len) ? (uint32_t)cn[q] : 4u;
            w[2 * h] = (cd == 0u ? 0x3F80u : 0u) | (cd == 1u ? 0x3F800000u : 0u);
            w[2 * h + 1] = (cd == 2u ? 0x3F80u : 0u) | (cd == 3u ? 0x3F800000u : 0u);
          }
          if (c == 3) w[2] = 0x3F80u, w[3] = 0u;  // feature 28: ones; 29-31: zero
          *reinterpret_cast<uint4*>(a + c * kWgAStride + r * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_proxy_async_smem();
      } else if (lane == 0) {
        atomicOr(err, ERR_TIMEOUT);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&built[s]);
    }
  }
  __syncthreads();
  const int issued = (int)*s_issued;
  if (issued > 0) {
    // rows 0..28 of the accumulator (warp 0's lanes) through shared memory, then coalesced
    // atomic adds along the output channels
    tc_fence_after();
    float* st = reinterpret_cast<float*>(sm);  // [29][129]
    if (warp == 0)
      for (int c = 0; c < 128; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (uint32_t)c, r);
        tmem_wait_ld();
        if (lane < 29)
#pragma unroll
          for (int q = 0; q < 32; ++q) st[lane * 129 + c + q] = __uint_as_float(r[q]);
      }
    __syncthreads();
    for (int f = 0; f < 29; ++f) {
      const float v = st[f * 129 + tid];
      if (v != 0.f) atomicAdd(f < 28 ? dw1 + f * kPropC + tid : db1 + tid, v);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

}  // namespace

cudaError_t prop_conv_wgrad_tc(const __nv_bfloat16* in, const __nv_bfloat16* g, const int32_t* lens, float* dw,
                               float* db, int32_t n, int32_t rows, int32_t* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)n * ((rows - 6) / kWgTile);
  if (total <= 0) return cudaSuccess;
  CUtensorMap tin, tg;
  e = prop_tensor_map_rows(&tin, in, (int64_t)n * rows, 8, (uint32_t)kWgABox, false);
  if (e == cudaSuccess) e = prop_tensor_map_rows(&tg, g, (int64_t)n * rows, 8, (uint32_t)kWgTile, false);
  if (e != cudaSuccess) return e;
  const int groups = (kPropTaps + kWgTapsPerCta - 1) / kWgTapsPerCta;
  // about one CTA per SM: runs of tiles per tap group
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(total, (num_sms + groups - 1) / groups));
  const int32_t per = (int32_t)((total + ctas - 1) / ctas);
  dim3 grid((unsigned)((total + per - 1) / per), (unsigned)groups);
  k_conv_wgrad_tc<<<grid, kWgThreads, kWgSmem, s>>>(tin, tg, lens, dw, db, n, rows, per, err);
  return cudaGetLastError();
}

}  // namespace mss

namespace mss {

cudaError_t prop_l1_wgrad(const uint8_t* codes, const int32_t* lens, int32_t ld, const __nv_bfloat16* g, float* dw1,
                          float* db1, int32_t n, int32_t rows, int32_t* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_l1_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kL1gSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)n * ((rows - 6) / kWgTile);
  if (total <= 0) return cudaSuccess;
  CUtensorMap tg;
  e = prop_tensor_map_rows(&tg, g, (int64_t)n * rows, 8, (uint32_t)kWgTile, false);
  if (e != cudaSuccess) return e;
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(total, num_sms));
  const int32_t per = (int32_t)((total + ctas - 1) / ctas);
  k_l1_wgrad_tc<<<(unsigned)((total + per - 1) / per), kWgThreads, kL1gSmem, s>>>(tg, codes, ld, lens, dw1, db1, n, rows,
                                                                                 per, err);
  return cudaGetLastError();
}

}  // namespace mss
