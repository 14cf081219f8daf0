// Device helpers shared by the libmaxss kernels: inline PTX for PRMT, packed f16 FMA,
// mbarrier and bulk (TMA) copies, and the packed-genome format.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mss {

// Packed genome: base p is 2 bits at word p/16 (bits 2*(p%16)), and a valid bit at word p/32
// (bit p%32) that is 0 for N and for padding.  Code 4 stands for N everywhere.
__device__ __forceinline__ uint32_t genome_code(const uint32_t* g2, const uint32_t* gm, int64_t p) {
  uint32_t c = (g2[p >> 4] >> ((p & 15) * 2)) & 3u;
  uint32_t v = (gm[p >> 5] >> (p & 31)) & 1u;
  return v ? c : 4u;
}

// ASCII -> code: A C G T (either case) -> 0..3, N/n -> 4, other -> 5 (invalid).
__device__ __forceinline__ uint32_t ascii_code(uint32_t ch) {
  switch (ch | 0x20u) {
    case 'a': return 0;
    case 'c': return 1;
    case 'g': return 2;
    case 't': return 3;
    case 'n': return 4;
    default: return 5;
  }
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// relu(a * b + c) on two f16 lanes (the FMA pipe).
__device__ __forceinline__ uint32_t hfma2_relu(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: returns false if the phase has not completed after
// limit_ns nanoseconds of polling (a poll takes about 25 ns).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t addr = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 0) {  // read the clock every 256 polls
      const uint64_t now = global_ns();
      if (it == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
}

// One-dimensional bulk copy global -> shared through the TMA unit, completing on an mbarrier.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Decode a non-negative f16 bit pattern holding an exact integer (0..2048) back to int.
__device__ __forceinline__ int32_t f16_bits_to_int(uint32_t v) {
  v &= 0xFFFFu;
  if (v == 0) return 0;
  int32_t e = (int32_t)((v >> 10) & 31u);  // biased exponent, value = 1.mant * 2^(e-15)
  int32_t sig = (int32_t)(1024u | (v & 0x3FFu));
  int32_t sh = e - 25;                      // value = sig * 2^(e-25)
  return sh >= 0 ? (sig << sh) : (sig >> (-sh));
}

// Top-2 over fragments: (s1, f1) best, (s2, f2) best among fragments != f1.
// Order: higher score, then lower fragment index.  Empty entry: s = -1, f = INT32_MAX.
struct Top2 {
  int32_t s1, f1, s2, f2;
};

__device__ __forceinline__ bool better(int32_t sa, int32_t fa, int32_t sb, int32_t fb) {
  return sa > sb || (sa == sb && fa < fb);
}

// Merge of two top-2 summaries that may share fragments (exact: the second is the best
// entry of either side whose fragment differs from the merged first).
__device__ __forceinline__ Top2 top2_merge(Top2 a, Top2 b) {
  Top2 r;
  if (better(b.s1, b.f1, a.s1, a.f1)) {
    Top2 t = a;
    a = b;
    b = t;
  }
  r.s1 = a.s1;
  r.f1 = a.f1;
  // candidates for second: a.s2 (a's second, fragment != a.f1), and b's best entry whose
  // fragment != a.f1
  int32_t cs = a.s2, cf = a.f2;
  int32_t bs = b.s1, bf = b.f1;
  if (bf == a.f1) {
    bs = b.s2;
    bf = b.f2;
  }
  if (better(bs, bf, cs, cf)) {
    cs = bs;
    cf = bf;
  }
  r.s2 = cs;
  r.f2 = cf;
  return r;
}

__device__ __forceinline__ Top2 top2_shfl_xor(Top2 v, int mask) {
  Top2 o;
  o.s1 = __shfl_xor_sync(0xffffffffu, v.s1, mask);
  o.f1 = __shfl_xor_sync(0xffffffffu, v.f1, mask);
  o.s2 = __shfl_xor_sync(0xffffffffu, v.s2, mask);
  o.f2 = __shfl_xor_sync(0xffffffffu, v.f2, mask);
  return o;
}

__device__ __forceinline__ Top2 top2_empty() { return Top2{-1, 0x7fffffff, -1, 0x7fffffff}; }

// Top-4 over fragments (higher score, then lower fragment), distinct fragments, sorted; empty
// entries s = -1, f = INT32_MAX.  Enough to find both the best fragment other than the first
// and the best one not adjacent to it (at most two fragments are adjacent).  Merging lists
// that share a fragment keeps its larger score, so partial maxima of a fragment split across
// genome chunks merge exactly: a fragment's true score is the largest of its partial maxima,
// and in the chunk holding that maximum fewer than four other fragments can precede it.
struct Top4 {
  int32_t s[4], f[4];
};

__device__ __forceinline__ Top4 top4_empty() {
  Top4 r;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.s[i] = -1, r.f[i] = 0x7fffffff;
  return r;
}

__device__ __forceinline__ Top4 top4_insert(Top4 a, int32_t s, int32_t f) {
  bool dup = false;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (a.f[i] == f) {
      dup = true;
      if (s > a.s[i]) a.s[i] = s;
    }
  if (dup) {  // one entry may have grown: bubble it towards the front
#pragma unroll
    for (int i = 3; i > 0; --i)
      if (better(a.s[i], a.f[i], a.s[i - 1], a.f[i - 1])) {
        const int32_t ts = a.s[i], tf = a.f[i];
        a.s[i] = a.s[i - 1], a.f[i] = a.f[i - 1];
        a.s[i - 1] = ts, a.f[i - 1] = tf;
      }
    return a;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)  // carry the new entry down the list; the last one drops out
    if (better(s, f, a.s[i], a.f[i])) {
      const int32_t ts = a.s[i], tf = a.f[i];
      a.s[i] = s, a.f[i] = f;
      s = ts, f = tf;
    }
  return a;
}

__device__ __forceinline__ Top4 top4_merge(Top4 a, const Top4& b) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (b.s[i] >= 0) a = top4_insert(a, b.s[i], b.f[i]);
  return a;
}

__device__ __forceinline__ Top4 top4_shfl_xor(const Top4& v, int mask) {
  Top4 o;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    o.s[i] = __shfl_xor_sync(0xffffffffu, v.s[i], mask);
    o.f[i] = __shfl_xor_sync(0xffffffffu, v.f[i], mask);
  }
  return o;
}

// ---- packed-lane maximum-scoring-subsequence step (scan and candidate rescoring)
// PRMT selector for the lane pair (genome code c1 at d + k, code c2 at d + D + k).
template <bool F16>
__device__ __forceinline__ uint32_t make_sel(uint32_t c1, uint32_t c2) {
  if (F16) {
    // f16 lane = [low byte 0x00 (byte 4 of {b,a}), high byte = profile byte c, or byte 5 for N]
    uint32_t n1 = c1 < 4 ? c1 : 5u, n2 = c2 < 4 ? c2 : 5u;
    return 4u | (n1 << 4) | (4u << 8) | (n2 << 12);
  } else {
    // int16 lane = [profile byte c (byte 4 = mismatch for N), its sign replicated]
    uint32_t n1 = c1 < 4 ? c1 : 4u, n2 = c2 < 4 ? c2 : 4u;
    return n1 | ((n1 | 8u) << 4) | (n2 << 8) | ((n2 | 8u) << 12);
  }
}

// Profile word of one query base: byte b = score byte of (query base, genome base b).
__device__ __forceinline__ uint32_t profile_word(uint32_t code, uint32_t ma, uint32_t mm) {
  uint32_t w = mm * 0x01010101u;
  if (code < 4) w = (w & ~(0xFFu << (8 * code))) | (ma << (8 * code));
  return w;
}

template <bool F16>
__device__ __forceinline__ uint32_t kadane_step(uint32_t h, uint32_t s) {
  if (F16) return hfma2_relu(h, 0x3C003C00u, s);   // relu(h * 1 + s) on two f16 lanes
  return __viaddmax_s16x2(h, s, 0u);                // max(h + s, 0) on two int16 lanes
}

template <bool F16>
__device__ __forceinline__ int32_t lane_value(uint32_t bits16) {
  if (F16) return f16_bits_to_int(bits16);
  return (int32_t)(int16_t)(bits16 & 0xFFFFu);
}

}  // namespace mss
