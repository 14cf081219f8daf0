// 128 -> 128 convolution of the proposal network on the fifth-generation tensor cores (a8
// forward, a11 backward-data): out[p][co] = sum over taps t and input channels ci of
// in[p + t - 3][ci] * w[t][ci][co], then bias + ReLU + length mask (forward) or the previous
// layer's ReLU mask (backward-data, with flipped transposed weights).
//
// One CTA = 128 positions x 128 output channels of one sequence, 128 threads.  The input tile
// (134 rows: the 128 positions and the 3-row halo on each side) is staged "k-group major":
// the 16-byte group g of channels 8g .. 8g+7 of row r sits at g * 2144 + r * 16, so rows are
// 16 bytes apart inside a group.  That is the canonical K-major operand layout without
// swizzling with a stride-dimension offset of 128 bytes (8 rows) and a leading-dimension
// offset of 2144 bytes (one group), and the tap shift becomes a start-address offset of
// t * 16 bytes: the A operand of tap t is rows t .. t + 127.  The weights of a tap arrive
// from HBM in the same layout (prepared once per weight update) by one bulk copy into a
// two-stage ring.  One thread issues 7 taps x 8 K-steps of tcgen05.mma (M = N = 128,
// K = 16, BF16 -> FP32 in tensor memory); the four warps then read the accumulator rows back
// with tcgen05.ld (warp w: positions 32w .. 32w + 31) for the epilogue.
#include <cuda_bf16.h>

#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"
#include "prop.h"
#include "tc.cuh"

namespace mss {

namespace {

constexpr int kCtM = 128;                              // positions per CTA
constexpr int kCtRows = kCtM + 6;                      // with the halo
constexpr uint32_t kCtGroupA = kCtRows * 16;           // bytes of one channel group of the input tile
constexpr uint32_t kCtBytesA = 16 * kCtGroupA;         // 34,304
constexpr uint32_t kCtGroupW = 128 * 16;               // one channel group of a tap's weights
constexpr uint32_t kCtBytesW = 16 * kCtGroupW;         // 32,768 per tap
constexpr uint32_t kCtOffW = (kCtBytesA + 1023) & ~1023u;
constexpr uint32_t kCtOffBar = kCtOffW + 2 * kCtBytesW;
constexpr uint32_t kCtSmem = kCtOffBar + 64;
constexpr int kCtThreads = 128;
constexpr uint32_t kCtIdesc = idesc_bf16_f32(128, 128);
constexpr uint64_t kCtWaitNs = 2000000000ull;

__device__ __forceinline__ void cp_async16_tc(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__global__ void __launch_bounds__(kCtThreads) k_conv_tc(const __nv_bfloat16* __restrict__ in,
                                                        const uint8_t* __restrict__ wcanon,
                                                        const float* __restrict__ bias,
                                                        const __nv_bfloat16* __restrict__ prev,
                                                        const int32_t* __restrict__ lens,
                                                        __nv_bfloat16* __restrict__ out, int32_t rows, int mode,
                                                        int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  const int n = blockIdx.y, p0 = blockIdx.x * kCtM;
  const int len = lens[n];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (p0 >= len) {  // the whole tile lies beyond the sequence: zeros
    for (int e = tid; e < kCtM * 16; e += kCtThreads) {
      const int r = e >> 4, c = e & 15;
      reinterpret_cast<uint4*>(out + ((int64_t)n * rows + p0 + r + 3) * kPropC)[c] = make_uint4(0, 0, 0, 0);
    }
    return;
  }
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kCtOffBar);
  uint64_t* wfull = bar;       // [2]
  uint64_t* wfree = bar + 2;   // [2]
  uint64_t* done = bar + 4;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&wfull[s], 1);
      mbar_init(&wfree[s], 1);
    }
    mbar_init(done, 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, 128);
    tmem_relinquish();
  }
  // input tile, k-group major: chunk (row r, group g) -> g * kCtGroupA + r * 16
  const __nv_bfloat16* inb = in + ((int64_t)n * rows + p0) * kPropC;  // tile row 0 = position p0 - 3
  const uint32_t sA = smem_u32(sm);
  for (int e = tid; e < kCtRows * 16; e += kCtThreads) {
    const int r = e >> 4, g = e & 15;
    cp_async16_tc(sA + g * kCtGroupA + r * 16, inb + r * kPropC + g * 8);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  fence_proxy_async_smem();  // the tensor cores read the tile through the async proxy
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sW = sA + kCtOffW;

  if (tid == 0) {
    int32_t armed[2] = {-1, -1};
    for (int t = 0; t < 2; ++t) {
      armed[t] = 0;
      mbar_arrive_expect_tx(&wfull[t], kCtBytesW);
      tma_load_1d(sm + kCtOffW + t * kCtBytesW, wcanon + (size_t)t * kCtBytesW, kCtBytesW, &wfull[t]);
    }
    bool ok = true;
    int issued = 0;
    for (int t = 0; t < kPropTaps && ok; ++t) {
      const int s = t & 1;
      ok = mbar_wait(&wfull[s], (uint32_t)((t >> 1) & 1), kCtWaitNs);
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kPropC / 16; ++ks)
        tc_mma_bf16(tmem, smem_desc(sA + (2 * ks) * kCtGroupA + t * 16, kCtGroupA, 128),
                    smem_desc(sW + s * kCtBytesW + (2 * ks) * kCtGroupW, kCtGroupW, 128), kCtIdesc,
                    (t > 0 || ks > 0) ? 1u : 0u);
      tc_commit(&wfree[s]);
      issued = t + 1;
      if (t >= 1 && t + 1 < kPropTaps) {  // refill the stage of tap t - 1 with tap t + 1
        const int s1 = (t + 1) & 1;
        ok = mbar_wait(&wfree[s1], (uint32_t)(((t - 1) >> 1) & 1), kCtWaitNs);
        if (!ok) break;
        armed[s1] = ((t + 1) >> 1) & 1;
        mbar_arrive_expect_tx(&wfull[s1], kCtBytesW);
        tma_load_1d(sm + kCtOffW + s1 * kCtBytesW, wcanon + (size_t)(t + 1) * kCtBytesW, kCtBytesW, &wfull[s1]);
      }
    }
    tc_commit(done);  // arrives when every MMA issued above has completed
    if (!ok || issued < kPropTaps) {
      s_bad = 1;
      atomicOr(err, ERR_TIMEOUT);
    }
    for (int s = 0; s < 2; ++s)
      if (armed[s] >= 0 && !mbar_wait(&wfull[s], (uint32_t)armed[s], kCtWaitNs)) atomicOr(err, ERR_TIMEOUT);
  }
  // epilogue: thread = position p0 + tid, 128 channels in four 32-column loads
  const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, kCtWaitNs));
  __syncwarp();
  tc_fence_after();
  const int p = p0 + tid;
  const int64_t orow = ((int64_t)n * rows + p + 3) * kPropC;
  const bool valid = ok && p < len && s_bad == 0;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    uint32_t x[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c), x);
    tmem_wait_ld();
    uint32_t packed[16];
    if (mode == 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float v0 = fmaxf(__uint_as_float(x[2 * j]) + bias[32 * c + 2 * j], 0.f);
        float v1 = fmaxf(__uint_as_float(x[2 * j + 1]) + bias[32 * c + 2 * j + 1], 0.f);
        if (!valid) v0 = v1 = 0.f;
        __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        packed[j] = *reinterpret_cast<uint32_t*>(&h);
      }
    } else {
      const uint4* pv = reinterpret_cast<const uint4*>(prev + orow + 32 * c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 m4 = valid ? pv[q] : make_uint4(0, 0, 0, 0);
        const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
        for (int h2 = 0; h2 < 4; ++h2) {
          const int j = 4 * q + h2;
          const __nv_bfloat162 pm = *reinterpret_cast<const __nv_bfloat162*>(&mw[h2]);
          float v0 = __uint_as_float(x[2 * j]), v1 = __uint_as_float(x[2 * j + 1]);
          if (!(__bfloat162float(pm.x) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(pm.y) > 0.f)) v1 = 0.f;
          __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
          packed[j] = *reinterpret_cast<uint32_t*>(&h);
        }
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(out + orow + 32 * c);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
}

// w[t][in][out] (bf16) -> per tap the B operand B[out][in] in the k-group-major layout:
// byte t * 32768 + (in / 8) * 2048 + out * 16 + (in % 8) * 2
__global__ void k_canon_weights(const __nv_bfloat16* __restrict__ w, uint8_t* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (t, out, group of 8 inputs)
  if (e >= kPropTaps * 128 * 16) return;
  const int t = e / (128 * 16), rem = e - t * 128 * 16, o = rem >> 4, g = rem & 15;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = w[((int64_t)t * 128 + g * 8 + i) * 128 + o];
  *reinterpret_cast<uint4*>(dst + (size_t)t * kCtBytesW + g * kCtGroupW + o * 16) = *reinterpret_cast<uint4*>(v);
}

}  // namespace

int64_t prop_canon_weight_bytes() { return (int64_t)kPropTaps * kCtBytesW; }

cudaError_t prop_canon_weights(const __nv_bfloat16* w, void* dst, cudaStream_t s) {
  const int n = kPropTaps * 128 * 16;
  k_canon_weights<<<(n + 255) / 256, 256, 0, s>>>(w, static_cast<uint8_t*>(dst));
  return cudaGetLastError();
}

cudaError_t prop_conv_tc(const __nv_bfloat16* in, const void* wcanon, const float* bias, const __nv_bfloat16* prev,
                         const int32_t* lens, __nv_bfloat16* out, int32_t n, int32_t rows, int mode, int32_t* err,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((unsigned)((rows - 6) / kCtM), (unsigned)n);
  k_conv_tc<<<grid, kCtThreads, kCtSmem, s>>>(in, static_cast<const uint8_t*>(wcanon), bias, prev, lens, out, rows,
                                               mode, err);
  return cudaGetLastError();
}

}  // namespace mss
