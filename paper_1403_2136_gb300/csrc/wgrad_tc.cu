// a11 (training of the learned proposal; not in the paper): weight gradient of a 128 -> 128
// convolution layer on the fifth-generation tensor cores,
//   dw[t][ci][co] += sum over sequences n and positions p of in[n][p + t - 3][ci] * g[n][p][co],
// for the seven taps t, as a GEMM per tap with M = 128 input channels, N = 128 output channels
// and K = positions.
//
// Layout: activations and gradients are BF16 rows [sequence][position + 3][128 channels] (three
// zero halo rows on either side), so a tile of positions is already "MN-major" for the MMA:
// channels contiguous, positions strided.  A CTA owns a run of 128-position tiles and a group of
// taps (0-3 or 4-6) whose FP32 accumulators (128 columns each) fill the tensor memory.  Per
// tile its 128 threads copy, with 16-byte cp.async, the input rows of the tile's positions
// shifted by the group's first tap (131 rows, padded to 136) and the 128 gradient rows into a
// three-stage ring, two tiles ahead of the MMAs; each 16-byte chunk (8 channels of one row) lands at
// channel-group * stride + row * 16, so that rows are 16 bytes apart throughout and a tap's
// shift is a start-address offset of 16 bytes per row.  One thread issues, per tap, eight
// tcgen05.mma (K = 16 positions each) and commits them on the stage's mbarrier; the next copy
// into that stage waits for it.  At the end the four warps read their 32 accumulator
// lanes (input channels) back and add them to dw with FP32 atomics.  Every wait is bounded.
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
constexpr uint32_t kWgAStride = kWgARows * 16;            // bytes between 8-channel groups of A
constexpr uint32_t kWgBStride = kWgTile * 16;             // the same for B
constexpr uint32_t kWgABytes = 16 * kWgAStride;           // 34,816
constexpr uint32_t kWgBBytes = 16 * kWgBStride;           // 32,768
constexpr uint32_t kWgStage = kWgABytes + kWgBBytes;
constexpr int kWgStages = 3;                              // copies two tiles ahead
constexpr uint32_t kWgSmem = kWgStages * kWgStage + 64;   // stages, mbarriers, TMEM slot
constexpr uint64_t kWgWaitNs = 2000000000ull;
// MN-major operands without swizzling: core matrices of 8 rows (K) x 16 bytes (8 MN
// elements); the descriptor's leading offset is the distance between core matrices adjacent
// in K (8 rows = 128 B here), its stride offset the distance between core matrices adjacent in
// MN (checked on GB300 with a single MMA of known integers against both assignments, and with a
// start address inside a core matrix, which the tap shift uses).
constexpr uint32_t kWgCoreK = 128;
// instruction descriptor: BF16 x BF16 -> FP32, M = N = 128, A and B MN-major (bits 15, 16)
constexpr uint32_t kWgIdesc = idesc_bf16_f32(128, 128) | (1u << 15) | (1u << 16);

__device__ __forceinline__ void cp_async16_wg(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__global__ void __launch_bounds__(kWgThreads, 1)
    k_conv_wgrad_tc(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ g,
                    const int32_t* __restrict__ lens, float* __restrict__ dw, int32_t n_seq, int32_t rows,
                    int32_t tiles_per_cta, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* done = reinterpret_cast<uint64_t*>(sm + kWgStages * kWgStage);   // [kWgStages]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kWgStages * kWgStage + 8 * kWgStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t0 = blockIdx.y * kWgTapsPerCta;
  const int ntaps = min(kWgTapsPerCta, kPropTaps - t0);
  const int tiles_per_seq = (rows - 6) / kWgTile;
  const int64_t total = (int64_t)n_seq * tiles_per_seq;
  const int64_t first = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t last = min(total, first + tiles_per_cta);

  if (tid == 0) {
    for (int k = 0; k < kWgStages; ++k) mbar_init(&done[k], 1);
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

  // tiles past a sequence's length carry zero gradients: skip them (the same for every thread)
  auto next_live = [&](int64_t tile) {
    while (tile < last) {
      const int n = (int)(tile / tiles_per_seq);
      if ((int)(tile - (int64_t)n * tiles_per_seq) * kWgTile < lens[n]) break;
      ++tile;
    }
    return tile;
  };
  // copy tile `tile` into stage s: the input rows p0 + t0 + r (buffer rows: position
  // p0 + t0 + r - 3), r < ntaps - 1 + 128 (the last tile's last row is the sequence's last buffer
  // row; the pad rows up to 135 are never read by an MMA of a tap of this group), and the
  // gradient rows of positions p0 .. p0 + 127 (buffer rows p0 + 3 ...)
  auto stage_copy = [&](int64_t tile, int s) {
    const int n = (int)(tile / tiles_per_seq);
    const int p0 = (int)(tile - (int64_t)n * tiles_per_seq) * kWgTile;
    const uint32_t sA = smem_u32(sm + s * kWgStage), sB = sA + kWgABytes;
    const __nv_bfloat16* ia = in + ((int64_t)n * rows + p0 + t0) * kPropC;
    const int arows = ntaps - 1 + kWgTile;
    for (int e = tid; e < arows * 16; e += kWgThreads) {
      const int r = e >> 4, c = e & 15;
      cp_async16_wg(sA + c * kWgAStride + r * 16, ia + (int64_t)r * kPropC + c * 8);
    }
    const __nv_bfloat16* gb = g + ((int64_t)n * rows + p0 + 3) * kPropC;
    for (int e = tid; e < kWgTile * 16; e += kWgThreads) {
      const int r = e >> 4, c = e & 15;
      cp_async16_wg(sB + c * kWgBStride + r * 16, gb + (int64_t)r * kPropC + c * 8);
    }
  };

  // Live tile k goes to stage k mod kWgStages and its MMAs commit on done[k mod kWgStages].
  // Every thread commits one cp.async group per prologue slot and per loop iteration (empty
  // once the tiles run out), so that group k holds live tile k's copies.
  bool ok = true;
  int64_t fetch = next_live(first);  // the next live tile to copy
  int copied = 0, issued = 0;         // live tiles copied / whose MMAs were issued
  for (int k = 0; k < kWgStages - 1; ++k) {
    if (fetch < last) {
      stage_copy(fetch, k);
      fetch = next_live(fetch + 1);
      ++copied;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  while (issued < copied) {
    const int s = issued % kWgStages;
    if (fetch < last) {
      // copied == issued + kWgStages - 1: the stage to refill was last read by tile issued - 1
      if (issued >= 1)
        ok = mbar_wait(&done[(issued - 1) % kWgStages], (uint32_t)(((issued - 1) / kWgStages) & 1), kWgWaitNs);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      stage_copy(fetch, copied % kWgStages);
      fetch = next_live(fetch + 1);
      ++copied;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(kWgStages - 1) : "memory");  // group `issued` landed
    fence_proxy_async_smem();  // the copies are visible to the tensor cores
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sm + s * kWgStage), b0 = a0 + kWgABytes;
      for (int j = 0; j < ntaps; ++j) {
#pragma unroll
        for (int kk = 0; kk < kWgTile / 16; ++kk)
          tc_mma_bf16(tmem + (uint32_t)(j * 128), smem_desc(a0 + (uint32_t)(j + 16 * kk) * 16, kWgCoreK, kWgAStride),
                      smem_desc(b0 + (uint32_t)(16 * kk) * 16, kWgCoreK, kWgBStride), kWgIdesc,
                      (issued > 0 || kk > 0) ? 1u : 0u);
      }
      tc_commit(&done[s]);
    }
    ++issued;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy in flight past this point
  // wait for the last committed tile of each stage (bounded), then read the accumulators
  bool drained = true;
  for (int k = issued - 1; k >= 0 && k >= issued - kWgStages; --k)
    if (!mbar_wait(&done[k % kWgStages], (uint32_t)((k / kWgStages) & 1), kWgWaitNs)) drained = false;
  if (!ok || !drained) {
    if (tid == 0) atomicOr(err, ERR_TIMEOUT);
  } else if (issued > 0) {
    tc_fence_after();
    for (int j = 0; j < ntaps; ++j) {
      float* dwt = dw + (int64_t)(t0 + j) * kPropC * kPropC + (int64_t)(warp * 32 + lane) * kPropC;
      for (int c = 0; c < 128; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 128 + c), r);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 32; ++q) atomicAdd(dwt + c + q, __uint_as_float(r[q]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace

cudaError_t prop_conv_wgrad_tc(const __nv_bfloat16* in, const __nv_bfloat16* g, const int32_t* lens, float* dw,
                               int32_t n, int32_t rows, int32_t* err, cudaStream_t s) {
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
  const int groups = (kPropTaps + kWgTapsPerCta - 1) / kWgTapsPerCta;
  // about one CTA per SM: runs of tiles per tap group
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(total, (num_sms + groups - 1) / groups));
  const int32_t per = (int32_t)((total + ctas - 1) / ctas);
  dim3 grid((unsigned)((total + per - 1) / per), (unsigned)groups);
  k_conv_wgrad_tc<<<grid, kWgThreads, kWgSmem, s>>>(in, g, lens, dw, n, rows, per, err);
  return cudaGetLastError();
}

}  // namespace mss
