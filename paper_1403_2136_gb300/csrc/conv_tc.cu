// 128 -> 128 convolution of the proposal network on the fifth-generation tensor cores (a8
// forward, a11 backward-data): out[p][co] = sum over taps t and input channels ci of
// in[p + t - 3][ci] * w[t][ci][co], then bias + ReLU + length mask (forward) or the previous
// layer's ReLU mask (backward-data, with flipped transposed weights).
//
// The GEMM per item (128 positions of one sequence) is D[co][p] = sum_t W_t[co][:] . X[p+t][:]
// with M = 128 output channels, N = 128 positions, K = 7 taps x 128 input channels, so that
// every MMA has N = 128, where the tensor cores run at their full rate (an MMA of N = 64 runs
// at about 0.7 of it, whether its A operand comes from shared or tensor memory).  The weights
// are the A operand and stay resident for the whole launch: taps 0-5 in tensor memory
// (64 columns per tap: output channel = lane, two input channels per 32-bit column), tap 6 in
// shared memory; the remaining 128 tensor-memory columns hold the accumulator.
//
// Persistent, warp-specialised kernel, one CTA per SM, items strided over the CTAs.  Roles,
// linked only by mbarriers:
//   warp 0  producer: per item two TMA tensor copies (channels 0-63 and 64-127, 134 rows of
//           128 B each) into a three-stage ring of input tiles, and in the backward pass one
//           more (the previous layer's activations at the item's 128 positions, whose sign is
//           the ReLU mask) into a two-slot ring;
//   warp 1  one thread issues the item's 56 MMAs (taps 0-5 with A from tensor memory, tap 6
//           with A from shared memory; 8 K-steps of 16 each) into the accumulator;
//   warps 2-5  epilogue: warp w owns output channels 32 (w mod 4) .. + 31 (its tensor-memory
//           lane quarter); it reads the whole accumulator (thread = channel, 128 positions),
//           releases it, then applies bias + ReLU + length mask (forward) or the ReLU mask
//           staged by the producer (backward) and stores BF16.
// Each half of an input tile is K-major in the 128-byte swizzled layout (rows of 128 B in
// 1 KB atoms of 8 rows, written swizzled by the TMA unit), so a K-step is a 32-byte start
// offset inside a row and the tap shift is a start offset of t rows (t * 128 B); one staged
// tile serves all 7 taps.  Every wait is time-bounded and reports through the error word.
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

constexpr int kCtM = 128;                              // positions per item (the MMA's N)
constexpr int kCtRows = kCtM + 6;                      // with the halo
constexpr int kCtStages = 3;
constexpr uint32_t kCtHalfA = 17 * 1024;               // 64 channels x 134 rows of 128 B, whole 1 KB atoms
constexpr uint32_t kCtBytesA = 2 * kCtHalfA;           // 34,816 per stage
constexpr uint32_t kCtTxA = 16 * kCtRows * 16;         // 34,304 bytes land per item
constexpr int kCtTmemTaps = 6;                         // taps whose weights live in tensor memory
constexpr uint32_t kCtTapCols = kPropC / 2;            // 64 columns per tap (two BF16 per column)
constexpr uint32_t kCtDCol = kCtTmemTaps * kCtTapCols; // 384: the accumulator's first column
constexpr uint32_t kCtTmemCols = 512;
constexpr uint32_t kCtTmemWBytes = kCtTmemTaps * kCtTapCols * kPropC * 4;  // 196,608
constexpr uint32_t kCtW6Bytes = kPropC * kPropC * 2;  // tap 6, canonical K-major: 32,768
constexpr uint32_t kCtOffW6 = kCtStages * kCtBytesA;
constexpr int kCtMaskSlots = 2;
constexpr uint32_t kCtMaskBytes = kCtM * kPropC * 2;    // 128 rows of 256 B, no swizzle
constexpr uint32_t kCtOffMask = kCtOffW6 + kCtW6Bytes;
constexpr uint32_t kCtOffBar = kCtOffMask + kCtMaskSlots * kCtMaskBytes;
constexpr uint32_t kCtSmem = kCtOffBar + 128;
constexpr int kCtThreads = 192;
constexpr uint32_t kCtIdesc = idesc_bf16_f32(kPropC, kCtM);
constexpr uint64_t kCtWaitNs = 2000000000ull;
static_assert(kCtSmem + 1024 <= 227 * 1024, "shared memory of the conv CTA");
static_assert(kCtDCol + kCtM <= kCtTmemCols, "tensor-memory columns");
static_assert(kCtOffW6 % 1024 == 0 && kCtHalfA % 1024 == 0 && kCtBytesA % 1024 == 0 && kCtOffMask % 1024 == 0,
              "operand alignment");
static_assert(kCtRows * 128 <= (int)kCtHalfA, "input tile half");

// D[tmem] (+)= A[tmem] * B[smem]^T (A: M lanes x 16 BF16, two per 32-bit column), one thread
__device__ __forceinline__ void tc_mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 32 consecutive 32-bit columns of this warp's 32 tensor-memory lanes (thread i -> lane i)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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
                                                           const __grid_constant__ CUtensorMap tprev,
                                                           const uint8_t* __restrict__ wprep,
                                                           const float* __restrict__ bias,
                                                           const int32_t* __restrict__ lens,
                                                           __nv_bfloat16* __restrict__ out, int32_t rows,
                                                           int32_t ntile, int32_t items, int mode, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint32_t s_tmem;
  __shared__ int32_t s_live[kCtStages];  // producer -> MMA issuer: the stage's item has live positions
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int first = blockIdx.x, stride = gridDim.x;
  const int count = first < items ? (items - 1 - first) / stride + 1 : 0;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kCtOffBar);
  uint64_t* wfull = bar;                        // tap 6's weights have landed
  uint64_t* afull = bar + 1;                    // [kCtStages] input tile of the stage landed
  uint64_t* afree = bar + 1 + kCtStages;        // [kCtStages] MMAs reading the stage completed
  uint64_t* dfull = bar + 1 + 2 * kCtStages;    // the item's accumulator is complete
  uint64_t* dfree = bar + 2 + 2 * kCtStages;    // the epilogue has read the accumulator
  uint64_t* mfull = bar + 3 + 2 * kCtStages;    // [kCtMaskSlots] backward: the item's mask tile landed
  uint64_t* mfree = bar + 3 + 2 * kCtStages + kCtMaskSlots;  // [kCtMaskSlots] the epilogue is done with it
  const uint32_t sA = smem_u32(sm);
  const uint32_t sW6 = sA + kCtOffW6;
  if (tid == 0) {
    mbar_init(wfull, 1);
    for (int s = 0; s < kCtStages; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&afree[s], 1);
    }
    mbar_init(dfull, 1);
    mbar_init(dfree, 4);
    for (int m = 0; m < kCtMaskSlots; ++m) {
      mbar_init(&mfull[m], 1);
      mbar_init(&mfree[m], 4);
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
  if (warp >= 2) {
    // taps 0-5 of the weights into tensor memory: thread = output channel (its lane), tap t at
    // columns 64 t .. 64 t + 63; the prepared words are [t][column][channel], so a warp's loads
    // are contiguous
    const int co = 32 * (warp & 3) + lane;
    const uint32_t* wt = reinterpret_cast<const uint32_t*>(wprep);
    for (int t = 0; t < kCtTmemTaps; ++t)
#pragma unroll
      for (int c0 = 0; c0 < (int)kCtTapCols; c0 += 32) {
        uint32_t r[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) r[c] = wt[((size_t)t * kCtTapCols + c0 + c) * kPropC + co];
        tmem_st32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(t * kCtTapCols + c0), r);
      }
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    if (lane == 0 && count > 0) {  // producer
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tin)) : "memory");
      if (mode == 1) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tprev)) : "memory");
      mbar_arrive_expect_tx(wfull, kCtW6Bytes);
      tma_load_1d(sm + kCtOffW6, wprep + kCtTmemWBytes, kCtW6Bytes, wfull);
      bool ok = true;
      for (int k = 0; k < count; ++k) {
        const int s = k % kCtStages, u = k / kCtStages;
        if (k >= kCtStages && ok && !mbar_wait(&afree[s], (uint32_t)((u - 1) & 1), kCtWaitNs)) {
          ok = false;
          atomicOr(err, ERR_TIMEOUT);
        }
        const ConvItem it = conv_item(first + k * stride, ntile, lens);
        s_live[s] = ok && it.live;  // published by the arrive below (release), read after the wait
        const int32_t y = it.n * rows + it.p0;  // padded row of position p0 - 3
        if (ok && it.live) {
          mbar_arrive_expect_tx(&afull[s], kCtTxA);
#pragma unroll
          for (int h = 0; h < 2; ++h) tma_load_2d(sA + s * kCtBytesA + h * kCtHalfA, &tin, 64 * h, y, &afull[s]);
        } else {
          mbar_arrive(&afull[s]);
        }
        if (mode == 1) {  // the mask tile of the item: rows of positions p0 .. p0 + 127
          const int m = k % kCtMaskSlots, v = k / kCtMaskSlots;
          if (k >= kCtMaskSlots && ok && !mbar_wait(&mfree[m], (uint32_t)((v - 1) & 1), kCtWaitNs)) {
            ok = false;
            atomicOr(err, ERR_TIMEOUT);
          }
          if (ok && it.live) {
            mbar_arrive_expect_tx(&mfull[m], kCtMaskBytes);
            tma_load_2d(sA + kCtOffMask + m * kCtMaskBytes, &tprev, 0, y + 3, &mfull[m]);
          } else {
            mbar_arrive(&mfull[m]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && count > 0) {  // MMA issuer
      bool wok = mbar_wait(wfull, 0, kCtWaitNs);
      if (!wok) atomicOr(err, ERR_TIMEOUT);
      const uint32_t d = tmem + kCtDCol;
      for (int k = 0; k < count; ++k) {
        const int s = k % kCtStages, u = k / kCtStages;
        bool go = mbar_wait(&afull[s], (uint32_t)(u & 1), kCtWaitNs);
        if (go && k >= 1) go = mbar_wait(dfree, (uint32_t)((k - 1) & 1), kCtWaitNs);
        if (!go) atomicOr(err, ERR_TIMEOUT);
        tc_fence_after();
        if (wok && go && s_live[s]) {
          const uint32_t a0 = sA + s * kCtBytesA;
#pragma unroll 1
          for (int t = 0; t < kCtTmemTaps; ++t) {
#pragma unroll
            for (int ks = 0; ks < kPropC / 16; ++ks)
              tc_mma_bf16_ts(d, tmem + (uint32_t)(t * kCtTapCols + ks * 8),
                             smem_desc_sw128(a0 + (ks >> 2) * kCtHalfA + t * 128 + (ks & 3) * 32), kCtIdesc,
                             (t > 0 || ks > 0) ? 1u : 0u);
          }
#pragma unroll
          for (int ks = 0; ks < kPropC / 16; ++ks)
            tc_mma_bf16(d, smem_desc(sW6 + ks * 256, kCanonLbo, kCanonSbo),
                        smem_desc_sw128(a0 + (ks >> 2) * kCtHalfA + kCtTmemTaps * 128 + (ks & 3) * 32), kCtIdesc,
                        1u);
          tc_commit(&afree[s]);
          tc_commit(dfull);
        } else {
          mbar_arrive(&afree[s]);
          mbar_arrive(dfull);
        }
      }
    }
  } else {  // epilogue: thread = output channel 32 (warp mod 4) + lane, the item's 128 positions
    const int q = warp & 3, co = 32 * q + lane;
    const float b_co = mode == 0 ? bias[co] : 0.f;
    for (int k = 0; k < count; ++k) {
      const bool ok = mbar_wait(dfull, (uint32_t)(k & 1), kCtWaitNs);
      if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
      __syncwarp();
      tc_fence_after();
      uint32_t x[4][32];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + kCtDCol;
#pragma unroll
      for (int c = 0; c < 4; ++c) tmem_ld32(ta + 32 * c, x[c]);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(dfree);
      const ConvItem it = conv_item(first + k * stride, ntile, lens);
      const int len = lens[it.n];
      const int64_t base = ((int64_t)it.n * rows + it.p0 + 3) * kPropC + co;
      const int m = k % kCtMaskSlots;
      bool mok = true;
      if (mode == 1) {
        mok = __all_sync(0xffffffffu, mbar_wait(&mfull[m], (uint32_t)((k / kCtMaskSlots) & 1), kCtWaitNs));
        if (!mok && lane == 0) atomicOr(err, ERR_TIMEOUT);
      }
      const __nv_bfloat16* mk = reinterpret_cast<const __nv_bfloat16*>(sm + kCtOffMask + m * kCtMaskBytes) + co;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int p = it.p0 + 32 * c + j;
          const int64_t o = base + (int64_t)(32 * c + j) * kPropC;
          const bool valid = ok && mok && it.live && p < len;
          float v = __uint_as_float(x[c][j]);
          if (mode == 0)
            v = fmaxf(v + b_co, 0.f);
          else if (!(valid && __bfloat162float(mk[(32 * c + j) * kPropC]) > 0.f))
            v = 0.f;
          if (!valid) v = 0.f;
          out[o] = __float2bfloat16_rn(v);
        }
      if (mode == 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&mfree[m]);
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

// w[t][in][out] (bf16) -> the kernel's resident A operands: for taps 0-5 the tensor-memory
// words [t][column c][out] = (w[t][2c][out], w[t][2c + 1][out]) (low half first), then tap 6
// as a [out][in] K-major tile in the canonical layout without swizzling.  One thread per
// (tap, column, output channel).
__global__ void k_canon_weights(const __nv_bfloat16* __restrict__ w, uint8_t* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kPropTaps * (int)kCtTapCols * kPropC) return;
  const int t = e / ((int)kCtTapCols * kPropC), rem = e - t * (int)kCtTapCols * kPropC;
  const int c = rem / kPropC, o = rem - c * kPropC;
  const __nv_bfloat16 lo = w[((int64_t)t * kPropC + 2 * c) * kPropC + o];
  const __nv_bfloat16 hi = w[((int64_t)t * kPropC + 2 * c + 1) * kPropC + o];
  if (t < kCtTmemTaps) {
    reinterpret_cast<uint32_t*>(dst)[e] =
        (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
  } else {
    __nv_bfloat16* w6 = reinterpret_cast<__nv_bfloat16*>(dst + kCtTmemWBytes);
    w6[canon_offset((uint32_t)o, (uint32_t)(2 * c)) / 2] = lo;
    w6[canon_offset((uint32_t)o, (uint32_t)(2 * c + 1)) / 2] = hi;
  }
}

}  // namespace

int64_t prop_canon_weight_bytes() { return (int64_t)kCtTmemWBytes + kCtW6Bytes; }

cudaError_t prop_canon_weights(const __nv_bfloat16* w, void* dst, cudaStream_t s) {
  const int n = kPropTaps * (int)kCtTapCols * kPropC;
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

cudaError_t prop_tensor_map_rows(CUtensorMap* map, const __nv_bfloat16* base, int64_t nrows, uint32_t box_ch,
                                 uint32_t box_rows, bool swizzle128) {
  // row coordinates of a tensor map are 32-bit; the base must be 16-byte aligned
  if (nrows <= 0 || nrows > INT32_MAX || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)kPropC, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {(cuuint64_t)kPropC * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {box_ch, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return cudaSuccess;
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
  CUtensorMap map, pmap;
  cudaError_t e = prop_tensor_map_rows(&map, in, (int64_t)n * rows, 64, (uint32_t)kCtRows, true);
  if (e != cudaSuccess) return e;
  // backward: the previous layer's activations, whose sign masks the gradient, as 128-row
  // tiles of all 128 channels (256-byte rows, no swizzle); the forward pass passes the input
  // map in its place (unused)
  pmap = map;
  if (mode == 1) {
    if (!prev) return cudaErrorInvalidValue;
    e = prop_tensor_map_rows(&pmap, prev, (int64_t)n * rows, (uint32_t)kPropC, (uint32_t)kCtM, false);
    if (e != cudaSuccess) return e;
  }
  // one CTA per SM (the tensor memory holds one CTA's weights and accumulator)
  const int64_t grid = std::min<int64_t>(std::max(1, sms), items);
  k_conv_tc<<<(unsigned)grid, kCtThreads, kCtSmem, s>>>(map, pmap, static_cast<const uint8_t*>(wcanon), bias, lens,
                                                         out, rows, ntile, (int32_t)items, mode, err);
  return cudaGetLastError();
}

}  // namespace mss
