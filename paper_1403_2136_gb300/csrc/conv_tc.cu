// 128 -> 128 convolution of the proposal network on the fifth-generation tensor cores (a8
// forward, a11 backward-data): out[p][co] = sum over taps t and input channels ci of
// in[p + t - 3][ci] * w[t][ci][co], then bias + ReLU + length mask (forward) or the previous
// layer's ReLU mask (backward-data, with flipped transposed weights).
//
// Persistent, warp-specialised kernel, one CTA per SM.  A CTA owns one half of the output
// channels (64) for the whole launch: the 7 taps of that half (112 KB of B operands) are
// copied into shared memory once and stay there.  Work item = 128 positions of one sequence;
// even CTAs take the low half and odd CTAs the high half of the same items, so the partner's
// read of an input tile hits L2.  Roles, linked only by mbarriers:
//   warp 0  producer: per item two TMA tensor copies (channels 0-63 and 64-127, 134 rows of
//           128 B each) into a three-stage ring of input tiles;
//   warp 1  one thread issues the item's 56 MMAs (7 taps x 8 K-steps of M = 128, N = 64,
//           K = 16, BF16 -> FP32) into one of three 64-column tensor-memory accumulators;
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (warp w reads lanes 32 (w mod 4) .. + 31),
//           release it, then bias + ReLU + mask and the BF16 store.
// Each half of an input tile is K-major in the 128-byte swizzled layout (rows of 128 B in
// 1 KB atoms of 8 rows, written swizzled by the TMA unit), so a K-step is a 32-byte start
// offset inside a row and the tap shift is a start offset of t rows (t * 128 B); one staged
// tile serves all 7 taps.  The resident weights use the
// canonical K-major layout without swizzling.  Every wait is time-bounded and reports through
// the error word.
#include <cuda.h>
#include <cudaTypedefs.h>
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

constexpr int kCtM = 128;                              // positions per item
constexpr int kCtN = 64;                               // output channels per CTA
constexpr int kCtRows = kCtM + 6;                      // with the halo
constexpr int kCtStages = 3;
constexpr uint32_t kCtHalfA = 17 * 1024;               // 64 channels x 134 rows of 128 B, whole 1 KB atoms
constexpr uint32_t kCtBytesA = 2 * kCtHalfA;           // 34,816 per stage
constexpr uint32_t kCtTxA = 16 * kCtRows * 16;         // 34,304 bytes land per item
constexpr uint32_t kCtGroupW = kCtN * 16;              // one channel group of a tap's half weights
constexpr uint32_t kCtTapW = 16 * kCtGroupW;           // 16,384 per tap and half
constexpr uint32_t kCtHalfW = kPropTaps * kCtTapW;     // 114,688 per half
constexpr uint32_t kCtOffW = kCtStages * kCtBytesA;
constexpr uint32_t kCtOffBar = kCtOffW + kCtHalfW;
constexpr uint32_t kCtSmem = kCtOffBar + 128;
constexpr int kCtThreads = 192;
constexpr uint32_t kCtTmemCols = 256;                  // power of two >= kCtStages * kCtN
constexpr uint32_t kCtIdesc = idesc_bf16_f32(kCtM, kCtN);
constexpr uint64_t kCtWaitNs = 2000000000ull;
static_assert(kCtSmem + 1024 <= 227 * 1024, "shared memory of the conv CTA");
static_assert(kCtStages * kCtN <= (int)kCtTmemCols, "tensor-memory columns");
static_assert(kCtOffW % 1024 == 0 && kCtHalfA % 1024 == 0 && kCtBytesA % 1024 == 0, "operand alignment");
static_assert(kCtRows * 128 <= (int)kCtHalfA, "input tile half");

// Shared-memory descriptor of a K-major operand in the 128-byte swizzled layout (rows of 128 B,
// 8-row atoms of 1 KB, the 16-byte chunks of row r XOR-ed with r mod 8, as the TMA unit writes
// them with CU_TENSOR_MAP_SWIZZLE_128B into 1 KB-aligned buffers): stride-dimension offset
// 1 KB, layout type 2 (bits 61-63), base offset 0.  The swizzle follows the absolute address
// bits, so a start moved by whole 128-byte rows (the tap shift) or by 32 bytes inside a row
// (a K-step) reads the tile as written (checked against the oracle by the embedding and
// gradient tests).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                      // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride-dimension offset: 8 rows
  d |= (uint64_t)1 << 46;                      // version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// 2-D tiled TMA load of one 64-channel half of an item's input tile (channels x .. x + 63,
// rows y .. y + 133, 128-byte rows in the 128-byte swizzle) completing on bar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

struct ConvItem {
  int n, p0;
  bool live;  // some position of the item lies inside the sequence
};

__device__ __forceinline__ ConvItem conv_item(int j, int ntile, const int32_t* lens) {
  ConvItem it;
  it.n = j / ntile;
  it.p0 = (j - it.n * ntile) * kCtM;
  it.live = it.p0 < lens[it.n];
  return it;
}

__global__ void __launch_bounds__(kCtThreads, 1) k_conv_tc(const __grid_constant__ CUtensorMap tin,
                                                           const uint8_t* __restrict__ wcanon,
                                                           const float* __restrict__ bias,
                                                           const __nv_bfloat16* __restrict__ prev,
                                                           const int32_t* __restrict__ lens,
                                                           __nv_bfloat16* __restrict__ out, int32_t rows,
                                                           int32_t ntile, int32_t items, int mode, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint32_t s_tmem;
  __shared__ int32_t s_live[kCtStages];  // producer -> MMA issuer: the stage's item has live positions
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int half = blockIdx.x & 1, stride = gridDim.x >> 1;
  const int first = blockIdx.x >> 1;
  const int count = first < items ? (items - 1 - first) / stride + 1 : 0;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kCtOffBar);
  uint64_t* wfull = bar;                       // the resident weights have landed
  uint64_t* afull = bar + 1;                   // [kCtStages] input tile of the stage landed
  uint64_t* done = bar + 1 + kCtStages;        // [kCtStages] MMAs of the stage's item completed
  uint64_t* accfree = bar + 1 + 2 * kCtStages; // [kCtStages] epilogue has read the accumulator
  const uint32_t sA = smem_u32(sm);
  const uint32_t sW = sA + kCtOffW;
  if (tid == 0) {
    mbar_init(wfull, 1);
    for (int s = 0; s < kCtStages; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&done[s], 1);
      mbar_init(&accfree[s], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, kCtTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0 && count > 0) {  // producer
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tin)) : "memory");
      mbar_arrive_expect_tx(wfull, kCtHalfW);
      for (int t = 0; t < kPropTaps; ++t)
        tma_load_1d(sm + kCtOffW + t * kCtTapW, wcanon + (size_t)half * kCtHalfW + (size_t)t * kCtTapW, kCtTapW,
                    wfull);
      bool ok = true;
      for (int k = 0; k < count; ++k) {
        const int s = k % kCtStages, u = k / kCtStages;
        if (k >= kCtStages && ok && !mbar_wait(&done[s], (uint32_t)((u - 1) & 1), kCtWaitNs)) {
          ok = false;
          atomicOr(err, ERR_TIMEOUT);
        }
        const ConvItem it = conv_item(first + k * stride, ntile, lens);
        s_live[s] = ok && it.live;  // published by the arrive below (release), read after the wait
        if (ok && it.live) {
          mbar_arrive_expect_tx(&afull[s], kCtTxA);
          const int32_t y = it.n * rows + it.p0;  // padded row of position p0 - 3
#pragma unroll
          for (int h = 0; h < 2; ++h) tma_load_2d(sA + s * kCtBytesA + h * kCtHalfA, &tin, 64 * h, y, &afull[s]);
        } else {
          mbar_arrive(&afull[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && count > 0) {  // MMA issuer
      bool wok = mbar_wait(wfull, 0, kCtWaitNs);
      if (!wok) atomicOr(err, ERR_TIMEOUT);
      for (int k = 0; k < count; ++k) {
        const int s = k % kCtStages, u = k / kCtStages;
        bool go = mbar_wait(&afull[s], (uint32_t)(u & 1), kCtWaitNs);
        if (go && k >= kCtStages) go = mbar_wait(&accfree[s], (uint32_t)((u - 1) & 1), kCtWaitNs);
        if (!go) atomicOr(err, ERR_TIMEOUT);
        tc_fence_after();
        if (wok && go && s_live[s]) {
          const uint32_t a0 = sA + s * kCtBytesA, d = tmem + (uint32_t)(s * kCtN);
#pragma unroll 1
          for (int t = 0; t < kPropTaps; ++t) {
#pragma unroll
            for (int ks = 0; ks < kPropC / 16; ++ks)
              tc_mma_bf16(d, smem_desc_sw128(a0 + (ks >> 2) * kCtHalfA + t * 128 + (ks & 3) * 32),
                          smem_desc(sW + t * kCtTapW + (2 * ks) * kCtGroupW, kCtGroupW, 128), kCtIdesc,
                          (t > 0 || ks > 0) ? 1u : 0u);
          }
          tc_commit(&done[s]);
        } else {
          mbar_arrive(&done[s]);
        }
      }
    }
  } else {  // epilogue: thread = position p0 + 32 (warp mod 4) + lane, the CTA's 64 channels
    const int q = warp & 3;
    for (int k = 0; k < count; ++k) {
      const int s = k % kCtStages, u = k / kCtStages;
      const bool ok = mbar_wait(&done[s], (uint32_t)(u & 1), kCtWaitNs);
      if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
      __syncwarp();
      tc_fence_after();
      uint32_t x[2][32];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * kCtN);
      tmem_ld32(ta, x[0]);
      tmem_ld32(ta + 32, x[1]);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[s]);
      const ConvItem it = conv_item(first + k * stride, ntile, lens);
      const int p = it.p0 + 32 * q + lane;
      const bool valid = ok && it.live && p < lens[it.n];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int ch = half * kCtN + 32 * c;
        const int64_t orow = ((int64_t)it.n * rows + p + 3) * kPropC + ch;
        uint32_t packed[16];
        if (mode == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float v0 = fmaxf(__uint_as_float(x[c][2 * j]) + bias[ch + 2 * j], 0.f);
            float v1 = fmaxf(__uint_as_float(x[c][2 * j + 1]) + bias[ch + 2 * j + 1], 0.f);
            if (!valid) v0 = v1 = 0.f;
            __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            packed[j] = *reinterpret_cast<uint32_t*>(&h);
          }
        } else {
          const uint4* pv = reinterpret_cast<const uint4*>(prev + orow);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const uint4 m4 = valid ? pv[v] : make_uint4(0, 0, 0, 0);
            const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int h2 = 0; h2 < 4; ++h2) {
              const int j = 4 * v + h2;
              const __nv_bfloat162 pm = *reinterpret_cast<const __nv_bfloat162*>(&mw[h2]);
              float v0 = __uint_as_float(x[c][2 * j]), v1 = __uint_as_float(x[c][2 * j + 1]);
              if (!(__bfloat162float(pm.x) > 0.f)) v0 = 0.f;
              if (!(__bfloat162float(pm.y) > 0.f)) v1 = 0.f;
              __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
              packed[j] = *reinterpret_cast<uint32_t*>(&h);
            }
          }
        }
        uint4* dst = reinterpret_cast<uint4*>(out + orow);
#pragma unroll
        for (int v = 0; v < 4; ++v)
          dst[v] = make_uint4(packed[4 * v], packed[4 * v + 1], packed[4 * v + 2], packed[4 * v + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, kCtTmemCols);
  }
}

// w[t][in][out] (bf16) -> per output half h and tap t the B operand B[out][in] in the
// k-group-major layout: byte h * 114688 + t * 16384 + (in / 8) * 1024 + (out % 64) * 16 + (in % 8) * 2
__global__ void k_canon_weights(const __nv_bfloat16* __restrict__ w, uint8_t* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (t, out, group of 8 inputs)
  if (e >= kPropTaps * 128 * 16) return;
  const int t = e / (128 * 16), rem = e - t * 128 * 16, o = rem >> 4, g = rem & 15;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = w[((int64_t)t * 128 + g * 8 + i) * 128 + o];
  *reinterpret_cast<uint4*>(dst + (size_t)(o / kCtN) * kCtHalfW + (size_t)t * kCtTapW + g * kCtGroupW +
                            (o % kCtN) * 16) = *reinterpret_cast<uint4*>(v);
}

}  // namespace

int64_t prop_canon_weight_bytes() { return (int64_t)(kPropC / kCtN) * kCtHalfW; }

cudaError_t prop_canon_weights(const __nv_bfloat16* w, void* dst, cudaStream_t s) {
  const int n = kPropTaps * 128 * 16;
  k_canon_weights<<<(n + 255) / 256, 256, 0, s>>>(w, static_cast<uint8_t*>(dst));
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

cudaError_t prop_conv_tc(const __nv_bfloat16* in, const void* wcanon, const float* bias, const __nv_bfloat16* prev,
                         const int32_t* lens, __nv_bfloat16* out, int32_t n, int32_t rows, int mode, int32_t* err,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtSmem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int32_t ntile = (rows - 6) / kCtM;
  const int64_t items = (int64_t)n * ntile;
  if (items <= 0) return cudaSuccess;
  // row coordinates of the tensor map are 32-bit; the base must be 16-byte aligned
  if ((int64_t)n * rows > INT32_MAX || (reinterpret_cast<uintptr_t>(in) & 15u) != 0) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)kPropC, (cuuint64_t)n * rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kPropC * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {64, (cuuint32_t)kCtRows};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(in), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // one CTA per SM, an even count (the two output halves of an item go to CTAs 2i and 2i + 1)
  const int64_t grid = std::min<int64_t>(std::max(2, sms & ~1), 2 * items);
  k_conv_tc<<<(unsigned)grid, kCtThreads, kCtSmem, s>>>(map, static_cast<const uint8_t*>(wcanon), bias, prev, lens,
                                                         out, rows, ntile, (int32_t)items, mode, err);
  return cudaGetLastError();
}

}  // namespace mss
