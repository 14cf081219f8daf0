// First layer of the proposal network (a8, 4 one-hot bases -> 128 channels, kernel 7) on the
// fifth-generation tensor cores:
//   out[p][co] = relu(b[co] + sum over taps t of w1[t][x[p + t - 3]][co])  for p < len, else 0,
// where a position outside the sequence or an N contributes nothing.
//
// As a GEMM per item (128 positions of one sequence): D[co][p] = sum_k A[co][k] * B[p][k] with
// B the one-hot features, B[p][4t + b] = 1 if x[p + t - 3] = b (K = 28, padded to 32), and A
// the FP32 weights written exactly as the sum of three BF16 parts (hi = bf16(w),
// mid = bf16(w - hi), lo = bf16(w - hi - mid): 3 x 8 significant bits), one 32-wide K block
// per part, so K = 96 and every product is exact; the tensor cores accumulate in FP32.
//
// Persistent, two CTAs (192 threads each) per SM, items strided over the CTAs.  The CTA builds A
// (24 KB, canonical K-major) once.  Roles, linked only by mbarriers:
//   warp 0  builds each item's B tile (128 positions x 32 BF16, canonical K-major, 8 KB) from
//           the codes into a two-stage ring;
//   warp 1  one thread issues the item's 6 MMAs (M = 128 channels, N = 128 positions, three
//           parts x two K-steps of 16) into one of two 128-column accumulators;
//   warps 2-5  epilogue: thread = output channel (the warp's tensor-memory lane quarter); it
//           reads the accumulator, releases it, adds the bias, applies ReLU and the length
//           mask and stores BF16.
// Every wait is time-bounded and reports through the error word.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"
#include "prop.h"
#include "tc.cuh"

namespace mss {

namespace {

constexpr int kL1M = 128;                   // positions per item (the MMA's N)
constexpr int kL1KPart = 32;                // one-hot features per weight part (28 used)
constexpr int kL1Parts = 3;
constexpr uint32_t kL1Lbo = 128;            // core matrices adjacent in K
constexpr uint32_t kL1SboB = (kL1KPart / 8) * 128;            // 512: 8-row groups of B
constexpr uint32_t kL1SboA = (kL1Parts * kL1KPart / 8) * 128;  // 1536: 8-row groups of A
constexpr uint32_t kL1BytesA = kPropC * kL1Parts * kL1KPart * 2;  // 24,576
constexpr uint32_t kL1BytesB = kL1M * kL1KPart * 2;               // 8,192
constexpr int kL1Stages = 2;
constexpr uint32_t kL1OffB = kL1BytesA;
constexpr int kL1Codes = 160;                        // codes of positions p0 - 3 .. p0 + 132 (136 used)
constexpr uint32_t kL1OffCodes = kL1OffB + kL1Stages * kL1BytesB;
constexpr uint32_t kL1OffBar = kL1OffCodes + kL1Stages * kL1Codes;
// at most two CTAs per SM, whose accumulators (256 columns each) fill the tensor memory
constexpr uint32_t kL1Smem = 80 * 1024;
static_assert(kL1OffBar + 128 <= kL1Smem, "shared memory of the first-layer CTA");
constexpr int kL1Threads = 192;
constexpr uint32_t kL1TmemCols = kL1Stages * kL1M;  // 256
constexpr uint32_t kL1Idesc = idesc_bf16_f32(kPropC, kL1M);
constexpr uint64_t kL1WaitNs = 2000000000ull;

// byte offset of element (row, k) in a canonical K-major tile whose 8-row groups are sbo apart
__device__ __forceinline__ uint32_t canon_at(uint32_t row, uint32_t k, uint32_t sbo) {
  return (row >> 3) * sbo + (k >> 3) * kL1Lbo + (row & 7u) * 16u + (k & 7u) * 2u;
}

__global__ void __launch_bounds__(kL1Threads, 1)
    k_embed_l1_tc(const uint8_t* __restrict__ codes, const int32_t* __restrict__ lens, int32_t ld,
                  const float* __restrict__ w1, const float* __restrict__ b1, __nv_bfloat16* __restrict__ out,
                  int32_t rows, int32_t ntile, int32_t items, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int first = blockIdx.x, stride = gridDim.x;
  const int count = first < items ? (items - 1 - first) / stride + 1 : 0;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kL1OffBar);
  uint64_t* bfull = bar;                    // [2] the stage's B tile is built
  uint64_t* bfree = bar + 2;                // [2] the MMAs reading it completed
  uint64_t* dfull = bar + 4;                // [2] the accumulator of the stage is complete
  uint64_t* dfree = bar + 6;                // [2] the epilogue has read it
  if (tid == 0) {
    for (int s = 0; s < kL1Stages; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bfree[s], 1);
      mbar_init(&dfull[s], 1);
      mbar_init(&dfree[s], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, kL1TmemCols);
    tmem_relinquish();
  }
  // A: the three BF16 parts of every weight, [channel][part * 32 + 4 t + b]
  for (int e = tid; e < kPropC * kL1Parts * kL1KPart; e += kL1Threads) {
    const int co = e / (kL1Parts * kL1KPart), k = e - co * (kL1Parts * kL1KPart);
    const int part = k / kL1KPart, kk = k - part * kL1KPart, t = kk >> 2, b = kk & 3;
    float v = 0.f;
    if (t < kPropTaps) {
      const float w = w1[(t * 4 + b) * kPropC + co];
      const float hi = __bfloat162float(__float2bfloat16_rn(w));
      const float r1 = w - hi;
      const float mid = __bfloat162float(__float2bfloat16_rn(r1));
      v = part == 0 ? hi : (part == 1 ? mid : r1 - mid);
    }
    *reinterpret_cast<__nv_bfloat16*>(sm + canon_at((uint32_t)co, (uint32_t)k, kL1SboA)) = __float2bfloat16_rn(v);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sA = smem_u32(sm), sB = sA + kL1OffB;

  if (warp == 0) {  // B builder: the item's codes into shared memory, then 16 chunks per lane
    bool ok = true;
    for (int k = 0; k < count && count > 0; ++k) {
      const int s = k % kL1Stages, u = k / kL1Stages;
      if (k >= kL1Stages && ok)
        ok = __all_sync(0xffffffffu, mbar_wait(&bfree[s], (uint32_t)((u - 1) & 1), kL1WaitNs));
      if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
      const int j = first + k * stride;
      const int n = j / ntile, p0 = (j - n * ntile) * kL1M;
      const int len = lens[n];
      if (ok && p0 < len) {
        // cb[e] = code of position p0 - 3 + e (4 outside the sequence): one batch of loads
        const uint8_t* cn = codes + (int64_t)n * ld;
        uint8_t* cb = sm + kL1OffCodes + s * kL1Codes;
#pragma unroll
        for (int e = lane; e < kL1Codes; e += 32) {
          const int q = p0 - 3 + e;
          cb[e] = (e < kL1M + 8 && q >= 0 && q < len) ? cn[q] : (uint8_t)4;
        }
        __syncwarp();
        uint8_t* dst = sm + kL1OffB + s * kL1BytesB;
#pragma unroll 4
        for (int e = lane; e < kL1M * (kL1KPart / 8); e += 32) {
          const int p = e >> 2, g = e & 3;  // chunk g: taps 2g and 2g + 1 (tap 7 is padding)
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int t = 2 * g + h;
            const uint32_t c = t < kPropTaps ? (uint32_t)cb[p + t] : 4u;
            // four BF16 indicators of bases 0..3: 1.0 = 0x3F80
            w[2 * h] = (c == 0u ? 0x3F80u : 0u) | (c == 1u ? 0x3F800000u : 0u);
            w[2 * h + 1] = (c == 2u ? 0x3F80u : 0u) | (c == 3u ? 0x3F800000u : 0u);
          }
          *reinterpret_cast<uint4*>(dst + canon_at((uint32_t)p, (uint32_t)(8 * g), kL1SboB)) =
              make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_proxy_async_smem();  // visible to the tensor cores
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bfull[s]);
    }
  } else if (warp == 1) {
    if (lane == 0 && count > 0) {  // MMA issuer
      for (int k = 0; k < count; ++k) {
        const int s = k % kL1Stages, u = k / kL1Stages;
        bool go = mbar_wait(&bfull[s], (uint32_t)(u & 1), kL1WaitNs);
        if (go && k >= kL1Stages) go = mbar_wait(&dfree[s], (uint32_t)((u - 1) & 1), kL1WaitNs);
        if (!go) atomicOr(err, ERR_TIMEOUT);
        tc_fence_after();
        const int j = first + k * stride;
        const int n = j / ntile, p0 = (j - n * ntile) * kL1M;
        if (go && p0 < lens[n]) {
          const uint32_t d = tmem + (uint32_t)(s * kL1M), b0 = sB + s * kL1BytesB;
#pragma unroll
          for (int part = 0; part < kL1Parts; ++part)
#pragma unroll
            for (int ks = 0; ks < kL1KPart / 16; ++ks)
              tc_mma_bf16(d, smem_desc(sA + (uint32_t)(part * 2 + ks) * 256, kL1Lbo, kL1SboA),
                          smem_desc(b0 + (uint32_t)ks * 256, kL1Lbo, kL1SboB), kL1Idesc,
                          (part > 0 || ks > 0) ? 1u : 0u);
          tc_commit(&bfree[s]);
          tc_commit(&dfull[s]);
        } else {
          mbar_arrive(&bfree[s]);
          mbar_arrive(&dfull[s]);
        }
      }
    }
  } else {  // epilogue: thread = output channel 32 (warp mod 4) + lane, the item's 128 positions
    const int q = warp & 3, co = 32 * q + lane;
    const float bco = b1[co];
    for (int k = 0; k < count; ++k) {
      const int s = k % kL1Stages, u = k / kL1Stages;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&dfull[s], (uint32_t)(u & 1), kL1WaitNs));
      if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
      tc_fence_after();
      uint32_t x[4][32];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * kL1M);
#pragma unroll
      for (int c = 0; c < 4; ++c) tmem_ld32(ta + 32 * c, x[c]);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dfree[s]);
      const int j = first + k * stride;
      const int n = j / ntile, p0 = (j - n * ntile) * kL1M;
      const int len = lens[n];
      const int64_t base = ((int64_t)n * rows + p0 + 3) * kPropC + co;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int p = p0 + 32 * c + i;
          const float v = (ok && p < len) ? fmaxf(__uint_as_float(x[c][i]) + bco, 0.f) : 0.f;
          out[base + (int64_t)(32 * c + i) * kPropC] = __float2bfloat16_rn(v);
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kL1TmemCols);
  }
}

}  // namespace

cudaError_t prop_embed_l1(const uint8_t* codes, const int32_t* lens, int32_t ld, int32_t n, const float* w1,
                          const float* b1, __nv_bfloat16* out, int32_t rows, int32_t* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_embed_l1_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kL1Smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int32_t ntile = (rows - 6) / kL1M;
  const int64_t items = (int64_t)n * ntile;
  if (items <= 0) return cudaSuccess;
  if (items > INT32_MAX) return cudaErrorInvalidValue;
  const int64_t grid = std::min<int64_t>(std::max(1, 2 * sms), items);
  k_embed_l1_tc<<<(unsigned)grid, kL1Threads, kL1Smem, s>>>(codes, lens, ld, w1, b1, out, rows, ntile,
                                                            (int32_t)items, err);
  return cudaGetLastError();
}

}  // namespace mss
