// a9: read x fragment scores on the fifth-generation tensor cores with a streaming per-read
// top K in the epilogue (the learned proposal; not in the paper).
//
// score(read, f) = max over the read's two strands of <e_strand, e_f>, BF16 embeddings, FP32
// accumulation; per read the K best fragments, larger score first, ties -> lower fragment.
//
// One CTA = 64 reads (128 sequences: 2i forward, 2i + 1 reverse complement of read i) x a
// contiguous range of 128-fragment tiles.  Warp 16 (one elected lane) streams the fragment
// tiles into a two-stage shared-memory ring with bulk copies and issues the MMAs
// (M = 128 fragments, N = 128 sequences, K = 128, eight K = 16 steps) into one of two
// tensor-memory accumulator stages.  Sixteen epilogue warps read the accumulators back (warp w:
// fragment rows 32 (w mod 4) .. + 31, the 16 reads 16 (w div 4) .. + 15), take the strand
// maximum, and append every score above the read's current threshold to the read's candidate
// buffer in shared memory (one warp vote per tile, then a ballot + one shared atomic per read
// that has a passing score).  When a buffer passes 128 entries the epilogue warps keep
// its K best (warp-wide selection of the K-th largest key) and raise the threshold.  The
// four warps of a group of 16 reads synchronise among themselves only (named barriers) and
// keep the group's thresholds in registers, reloading them after a tile that raised one.  Tiles
// are processed in increasing fragment order, so a later fragment equal to the threshold
// loses the tie and is never appended.  With several CTAs per read block (fragment splits)
// every split writes its K best and k_topk_merge keeps the K best of the splits.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"
#include "prop.h"
#include "tc.cuh"

namespace mss {

namespace {

constexpr int kTcReads = 64;                          // reads per CTA
constexpr int kTcN = 2 * kTcReads;                    // MMA N: sequences per CTA
constexpr int kTcM = 128;                             // MMA M: fragments per tile
constexpr uint32_t kTcTile = kTcM * kPropC * 2;       // bytes of a fragment tile (and of a read block)
constexpr int kTcCap = 256;                           // candidate slots per read
constexpr int kTcEpiWarps = 16;                       // 4 lane quarters x 4 groups of 16 reads
constexpr int kTcThreads = (kTcEpiWarps + 1) * 32;
constexpr uint32_t kTcTmemCols = 2 * kTcN;            // two accumulator stages of N columns
constexpr uint32_t kTcIdesc = idesc_bf16_f32(kTcM, kTcN);
constexpr uint64_t kTcWaitNs = 2000000000ull;

constexpr uint32_t kOffB = 0;
constexpr uint32_t kOffA = kOffB + kTcTile;                       // two stages
constexpr uint32_t kOffKey = kOffA + 2 * kTcTile;                 // uint32 [kTcReads][kTcCap]
constexpr uint32_t kOffFrag = kOffKey + kTcReads * kTcCap * 4;    // int32 [kTcReads][kTcCap]
constexpr uint32_t kOffTheta = kOffFrag + kTcReads * kTcCap * 4;  // uint32 [kTcReads]
constexpr uint32_t kOffCnt = kOffTheta + kTcReads * 4;            // int32 [kTcReads]
constexpr uint32_t kOffBar = kOffCnt + kTcReads * 4;              // 7 mbarriers
constexpr uint32_t kOffMisc = kOffBar + 8 * 8;                    // tensor-memory base, abort flag
constexpr uint32_t kTcSmem = kOffMisc + 16;
static_assert(kTcSmem <= 232448, "fused scoring kernel exceeds the shared memory of a CTA");

struct TcArgs {
  const __nv_bfloat16* breads;  // canonical blocks of kTcN sequences
  const __nv_bfloat16* index;   // canonical tiles of kTcM fragments
  int32_t R;
  int64_t NF;
  int32_t T;    // fragment tiles
  int32_t S;    // splits of the tile range per read block
  int32_t tps;  // tiles per split
  int32_t K;
  int32_t* out_f;     // S == 1: [R][K]
  float* out_s;
  uint32_t* part_key; // S > 1: [S][R][K]
  int32_t* part_f;
  int32_t* err;
};

// order-preserving unsigned key of a float, and back
__device__ __forceinline__ uint32_t score_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_score(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Keep the K best (key desc, fragment asc) of the n <= kTcCap entries of one buffer in its
// first slots; returns the K-th largest key, or 0 (accept everything) with fewer than K.
__device__ uint32_t warp_select(uint32_t* key, int32_t* frag, int n, int K, int lane) {
  if (n <= K) {
    if (n < K) return 0u;
    uint32_t mn = 0xFFFFFFFFu;
    for (int e = lane; e < n; e += 32) mn = min(mn, key[e]);
    return __reduce_min_sync(0xffffffffu, mn);
  }
  constexpr int E = kTcCap / 32;
  uint32_t kk[E];
  int32_t ff[E];
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int e = lane + 32 * t;
    kk[t] = e < n ? key[e] : 0u;
    ff[t] = e < n ? frag[e] : 0x7fffffff;
  }
  __syncwarp();
  // the K-th largest key, bit by bit: the largest T with #(key >= T) >= K
  uint32_t T = 0u;
  for (int bit = 31; bit >= 0; --bit) {
    const uint32_t c = T | (1u << bit);
    uint32_t cnt = 0;
#pragma unroll
    for (int t = 0; t < E; ++t) cnt += kk[t] >= c ? 1u : 0u;
    if ((int)__reduce_add_sync(0xffffffffu, cnt) >= K) T = c;
  }
  bool take[E];
  uint32_t cgt = 0;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    take[t] = kk[t] > T;
    cgt += take[t] ? 1u : 0u;
  }
  int need = K - (int)__reduce_add_sync(0xffffffffu, cgt);
  while (need > 0) {  // entries equal to T: lowest fragments first
    int32_t fm = 0x7fffffff;
#pragma unroll
    for (int t = 0; t < E; ++t)
      if (kk[t] == T && !take[t]) fm = min(fm, ff[t]);
    fm = __reduce_min_sync(0xffffffffu, fm);
#pragma unroll
    for (int t = 0; t < E; ++t)
      if (kk[t] == T && !take[t] && ff[t] == fm) take[t] = true;
    --need;
  }
  int base = 0;
  const uint32_t below = (1u << lane) - 1u;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const uint32_t b = __ballot_sync(0xffffffffu, take[t]);
    if (take[t]) {
      const int pos = base + __popc(b & below);
      key[pos] = kk[t];
      frag[pos] = ff[t];
    }
    base += __popc(b);
  }
  __syncwarp();
  return T;
}

// Write n <= K entries sorted (key desc, fragment asc), padded to K.
__device__ void warp_emit(const uint32_t* key, const int32_t* frag, int n, int K, int lane, int32_t* of, float* os,
                          uint32_t* ok, int32_t* okf) {
  for (int a = lane; a < n; a += 32) {
    const uint32_t ka = key[a];
    const int32_t fa = frag[a];
    int rank = 0;
    for (int b = 0; b < n; ++b) {
      const uint32_t kb = key[b];
      rank += (kb > ka) || (kb == ka && frag[b] < fa);
    }
    if (of) {
      of[rank] = fa;
      os[rank] = key_score(ka);
    } else {
      ok[rank] = ka;
      okf[rank] = fa;
    }
  }
  for (int a = n + lane; a < K; a += 32) {
    if (of) {
      of[a] = -1;
      os[a] = -1e30f;
    } else {
      ok[a] = 0u;
      okf[a] = -1;
    }
  }
}

// The four epilogue warps of a read group (warps 4g .. 4g + 3 append to reads 16g .. 16g + 15
// and compact them) synchronise on their own named barrier 2 + g; the "or" form makes every
// warp of the group take the same decision (abort, or reload the thresholds).
__device__ __forceinline__ bool grp_bar_or(int g, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, 128, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(2 + g)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_score_topk(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rb = blockIdx.x / a.S, split = blockIdx.x - rb * a.S;
  const int r0 = rb * kTcReads;
  const int t0 = split * a.tps;
  const int nt = min(a.T, t0 + a.tps) - t0;
  uint8_t* sB = smem + kOffB;
  uint8_t* sA = smem + kOffA;
  uint32_t* s_key = reinterpret_cast<uint32_t*>(smem + kOffKey);
  int32_t* s_frag = reinterpret_cast<int32_t*>(smem + kOffFrag);
  uint32_t* s_theta = reinterpret_cast<uint32_t*>(smem + kOffTheta);
  int32_t* s_cnt = reinterpret_cast<int32_t*>(smem + kOffCnt);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
  uint64_t* full_b = bar + 0;
  uint64_t* full_a = bar + 1;     // [2]
  uint64_t* mma_done = bar + 3;   // [2]
  uint64_t* tmem_free = bar + 5;  // [2]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kOffMisc);
  volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(smem + kOffMisc + 4);

  if (tid < kTcReads) {
    s_theta[tid] = 0u;
    s_cnt[tid] = 0;
  }
  if (tid == 0) {
    mbar_init(full_b, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full_a[s], 1);
      mbar_init(&mma_done[s], 1);
      mbar_init(&tmem_free[s], kTcEpiWarps);
    }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTcEpiWarps) {
    tmem_alloc(s_tmem, kTcTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == kTcEpiWarps) {
    // ---- producer and MMA issuer
    if (lane == 0 && nt > 0) {
      const uint8_t* gidx = reinterpret_cast<const uint8_t*>(a.index) + (size_t)t0 * kTcTile;
      int32_t armed[2] = {-1, -1};
      mbar_arrive_expect_tx(full_b, kTcTile);
      tma_load_1d(sB, reinterpret_cast<const uint8_t*>(a.breads) + (size_t)rb * kTcTile, kTcTile, full_b);
      for (int j = 0; j < 2 && j < nt; ++j) {
        armed[j] = 0;
        mbar_arrive_expect_tx(&full_a[j], kTcTile);
        tma_load_1d(sA + j * kTcTile, gidx + (size_t)j * kTcTile, kTcTile, &full_a[j]);
      }
      bool ok = mbar_wait(full_b, 0, kTcWaitNs);
      int issued = 0;
      const uint32_t b_addr = smem_u32(sB);
      for (int j = 0; ok && j < nt; ++j) {
        const int s = j & 1;
        ok = mbar_wait(&full_a[s], (uint32_t)((j >> 1) & 1), kTcWaitNs);
        if (ok && j >= 2) ok = mbar_wait(&tmem_free[s], (uint32_t)(((j >> 1) - 1) & 1), kTcWaitNs);
        if (!ok) break;
        tc_fence_after();
        const uint32_t a_addr = smem_u32(sA + s * kTcTile);
#pragma unroll
        for (int ks = 0; ks < kPropC / 16; ++ks)
          tc_mma_bf16(tmem + (uint32_t)(s * kTcN), smem_desc(a_addr + ks * 256, kCanonLbo, kCanonSbo),
                      smem_desc(b_addr + ks * 256, kCanonLbo, kCanonSbo), kTcIdesc, ks > 0 ? 1u : 0u);
        tc_commit(&mma_done[s]);
        issued = j + 1;
        if (j >= 1 && j + 1 < nt) {  // refill the stage of tile j - 1 with tile j + 1
          const int s1 = (j + 1) & 1;
          ok = mbar_wait(&mma_done[s1], (uint32_t)(((j - 1) >> 1) & 1), kTcWaitNs);
          if (!ok) break;
          armed[s1] = ((j + 1) >> 1) & 1;
          mbar_arrive_expect_tx(&full_a[s1], kTcTile);
          tma_load_1d(sA + s1 * kTcTile, gidx + (size_t)(j + 1) * kTcTile, kTcTile, &full_a[s1]);
        }
      }
      if (!ok) {
        *s_abort = 1;
        atomicOr(a.err, ERR_TIMEOUT);
      }
      // drain: the last committed MMA (they complete in order) and every armed copy
      if (issued > 0 &&
          !mbar_wait(&mma_done[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1), kTcWaitNs))
        atomicOr(a.err, ERR_TIMEOUT);
      mbar_wait(full_b, 0, kTcWaitNs);
      for (int s = 0; s < 2; ++s)
        if (armed[s] >= 0 && !mbar_wait(&full_a[s], (uint32_t)armed[s], kTcWaitNs)) atomicOr(a.err, ERR_TIMEOUT);
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads accumulator lanes 32 (w mod 4) .. + 31 (fragments) and
    //      columns 32 (w div 4) .. + 31 (16 reads): strand maximum, threshold, candidate buffers
    const int q = warp & 3, grp = warp >> 2, rbase = 16 * grp;
    const int frow = 32 * q + lane;  // fragment row of this thread in a tile
    // the group's 16 thresholds as floats, kept in registers and reloaded only after a tile
    // in which some warp of the group raised one (key 0, before the first compaction,
    // accepts every score)
    float th[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) th[i] = __int_as_float(0xff800000);
    for (int j = 0; j < nt; ++j) {
      const int s = j & 1;
      // every lane waits (acquire); the tensor-memory loads below need the whole warp
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&mma_done[s], (uint32_t)((j >> 1) & 1), kTcWaitNs));
      if (!ok) *s_abort = 1;
      const int64_t f = (int64_t)(t0 + j) * kTcM + frow;
      if (ok) {
        tc_fence_after();
        // scores are made canonical (-0 -> +0), so on them the float order is the key order
        // and "v > threshold" is "key > threshold key"; rows past the last fragment never pass
        uint32_t x[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * kTcN + 2 * rbase), x);
        tmem_wait_ld();
        float v[16];
        uint32_t m = 0u;  // bit i: this thread's score for read rbase + i passes
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          v[i] = fmaxf(__uint_as_float(x[2 * i]), __uint_as_float(x[2 * i + 1])) + 0.0f;
          m |= (v[i] > th[i] ? 1u : 0u) << i;
        }
        if (f >= a.NF) m = 0u;
        // append, for the reads where some lane passes (a warp-uniform test per read)
        const uint32_t mm = __reduce_or_sync(0xffffffffu, m);
        if (mm) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (mm & (1u << i)) {
              const int r = rbase + i;
              const bool pred = (m >> i) & 1u;
              const uint32_t b = __ballot_sync(0xffffffffu, pred);
              const int leader = __ffs(b) - 1;
              int basepos = 0;
              if (lane == leader) basepos = atomicAdd(&s_cnt[r], __popc(b));
              basepos = __shfl_sync(0xffffffffu, basepos, leader);
              if (pred) {
                const int pos = basepos + __popc(b & ((1u << lane) - 1u));
                s_key[r * kTcCap + pos] = score_key(v[i]);
                s_frag[r * kTcCap + pos] = (int32_t)f;
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tmem_free[s]);
      // every append of the group's reads for this tile is done
      const bool abort = grp_bar_or(grp, *s_abort != 0);
      bool raised = false;
      if (!abort)
        for (int r = rbase + q; r < rbase + 16; r += 4)
          if (s_cnt[r] > kTcCap - kTcM) {
            s_theta[r] = warp_select(s_key + r * kTcCap, s_frag + r * kTcCap, s_cnt[r], a.K, lane);
            if (lane == 0) s_cnt[r] = a.K;
            __syncwarp();
            raised = true;
          }
      // the group's buffers compacted before its next appends; new thresholds are visible
      if (grp_bar_or(grp, raised)) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const uint32_t k = s_theta[rbase + i];
          th[i] = k == 0u ? __int_as_float(0xff800000) : key_score(k);
        }
      }
      if (abort) break;
    }
    // the K best of every read of the group (its buffers are final after the last group barrier)
    for (int r = rbase + q; r < rbase + 16; r += 4) {
      const int rg = r0 + r;
      if (rg >= a.R) continue;
      int n = s_cnt[r];
      if (n > a.K) {
        warp_select(s_key + r * kTcCap, s_frag + r * kTcCap, n, a.K, lane);
        n = a.K;
      }
      __syncwarp();
      if (a.S == 1)
        warp_emit(s_key + r * kTcCap, s_frag + r * kTcCap, n, a.K, lane, a.out_f + (size_t)rg * a.K,
                  a.out_s + (size_t)rg * a.K, nullptr, nullptr);
      else
        warp_emit(s_key + r * kTcCap, s_frag + r * kTcCap, n, a.K, lane, nullptr, nullptr,
                  a.part_key + ((size_t)split * a.R + rg) * a.K, a.part_f + ((size_t)split * a.R + rg) * a.K);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kTcEpiWarps) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcTmemCols);
  }
}

// K best of the S split lists of each read; one warp per read
constexpr int kMergeWarps = 4;
__global__ void __launch_bounds__(kMergeWarps * 32) k_topk_merge(const uint32_t* __restrict__ pk,
                                                                 const int32_t* __restrict__ pf, int32_t R, int32_t S,
                                                                 int32_t K, int32_t* out_f, float* out_s) {
  __shared__ uint32_t s_key[kMergeWarps][kTcCap];
  __shared__ int32_t s_frag[kMergeWarps][kTcCap];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * kMergeWarps + w;
  if (r >= R) return;
  int n = 0;
  for (int s = 0; s < S; ++s) {
    const uint32_t* k = pk + ((size_t)s * R + r) * K;
    const int32_t* f = pf + ((size_t)s * R + r) * K;
    // entries are sorted with the padding (fragment -1) last
    int cnt = 0;
    for (int e = lane; e < K; e += 32) cnt += f[e] >= 0 ? 1 : 0;
    cnt = (int)__reduce_add_sync(0xffffffffu, (uint32_t)cnt);
    for (int e = lane; e < cnt; e += 32) {
      s_key[w][n + e] = k[e];
      s_frag[w][n + e] = f[e];
    }
    n += cnt;
  }
  __syncwarp();
  if (n > K) {
    warp_select(s_key[w], s_frag[w], n, K, lane);
    n = K;
  }
  __syncwarp();
  warp_emit(s_key[w], s_frag[w], n, K, lane, out_f + (size_t)r * K, out_s + (size_t)r * K, nullptr, nullptr);
}

// fp32 embeddings [2R][128] -> BF16 canonical blocks of kTcN sequences (zero beyond 2R)
__global__ void k_pack_reads_canon(const float* __restrict__ er, int32_t R, uint8_t* __restrict__ out,
                                   int64_t nchunks) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nchunks) return;
  const int64_t seq = t >> 4;
  const int kc = (int)(t & 15);
  const int64_t blk = seq / kTcN;
  const int row = (int)(seq - blk * kTcN);
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (seq < 2 * (int64_t)R) {
    const float4 a = *reinterpret_cast<const float4*>(er + seq * kPropC + kc * 8);
    const float4 b = *reinterpret_cast<const float4*>(er + seq * kPropC + kc * 8 + 4);
    __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
    v.x = *reinterpret_cast<uint32_t*>(&p0);
    v.y = *reinterpret_cast<uint32_t*>(&p1);
    v.z = *reinterpret_cast<uint32_t*>(&p2);
    v.w = *reinterpret_cast<uint32_t*>(&p3);
  }
  *reinterpret_cast<uint4*>(out + blk * kTcTile + canon_offset((uint32_t)row, (uint32_t)kc * 8)) = v;
}

// fp32 embeddings of fragments f0 .. f0 + nb - 1 -> BF16 canonical fragment tiles
__global__ void k_store_index_canon(const float* __restrict__ emb, int64_t f0, int32_t nb, uint8_t* __restrict__ index) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * 16) return;
  const int64_t i = t >> 4;
  const int kc = (int)(t & 15);
  const int64_t f = f0 + i;
  const float4 a = *reinterpret_cast<const float4*>(emb + i * kPropC + kc * 8);
  const float4 b = *reinterpret_cast<const float4*>(emb + i * kPropC + kc * 8 + 4);
  __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
  __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
  uint4 v;
  v.x = *reinterpret_cast<uint32_t*>(&p0);
  v.y = *reinterpret_cast<uint32_t*>(&p1);
  v.z = *reinterpret_cast<uint32_t*>(&p2);
  v.w = *reinterpret_cast<uint32_t*>(&p3);
  *reinterpret_cast<uint4*>(index + (f >> 7) * (int64_t)kTcTile + canon_offset((uint32_t)(f & 127), (uint32_t)kc * 8)) =
      v;
}

}  // namespace

int64_t prop_index_bytes(int64_t NF) { return (NF + kTcM - 1) / kTcM * (int64_t)kTcTile; }
int64_t prop_read_block_bytes(int32_t R) { return ((2 * (int64_t)R + kTcN - 1) / kTcN) * (int64_t)kTcTile; }

cudaError_t prop_store_index(const float* emb, int64_t f0, int32_t nb, void* index, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  const int64_t n = (int64_t)nb * 16;
  k_store_index_canon<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(emb, f0, nb, static_cast<uint8_t*>(index));
  return cudaGetLastError();
}

cudaError_t prop_pack_reads(const float* er, int32_t R, void* out, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  const int64_t n = prop_read_block_bytes(R) / kTcTile * kTcN * 16;
  k_pack_reads_canon<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(er, R, static_cast<uint8_t*>(out), n);
  return cudaGetLastError();
}

int32_t prop_score_splits(int32_t R, int64_t NF, int32_t K, int num_sms) {
  const int64_t blocks = (R + kTcReads - 1) / kTcReads;
  const int64_t T = (NF + kTcM - 1) / kTcM;
  int64_t S = (num_sms + blocks - 1) / blocks;  // at least one CTA per SM
  S = std::min<int64_t>(S, kTcCap / std::max(1, K));
  S = std::min<int64_t>(S, T);
  return (int32_t)std::max<int64_t>(1, S);
}

cudaError_t prop_score_topk(const void* breads, int32_t R, const void* index, int64_t NF, int32_t K, int32_t S,
                            int32_t* out_f, float* out_s, uint32_t* part_key, int32_t* part_f, int32_t* err,
                            cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  if (K < 1 || K > kTcCap - kTcM || S < 1 || (int64_t)S * K > kTcCap || NF < 1) return cudaErrorInvalidValue;
  TcArgs a;
  a.breads = static_cast<const __nv_bfloat16*>(breads);
  a.index = static_cast<const __nv_bfloat16*>(index);
  a.R = R;
  a.NF = NF;
  a.T = (int32_t)((NF + kTcM - 1) / kTcM);
  a.tps = (a.T + S - 1) / S;
  a.S = (a.T + a.tps - 1) / a.tps;
  a.K = K;
  a.out_f = out_f;
  a.out_s = out_s;
  a.part_key = part_key;
  a.part_f = part_f;
  a.err = err;
  if (a.S > 1 && (!part_key || !part_f)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_score_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (R + kTcReads - 1) / kTcReads;
  k_score_topk<<<(unsigned)(blocks * a.S), kTcThreads, kTcSmem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || a.S == 1) return e;
  k_topk_merge<<<(unsigned)((R + kMergeWarps - 1) / kMergeWarps), kMergeWarps * 32, 0, s>>>(part_key, part_f, R, a.S,
                                                                                           K, out_f, out_s);
  return cudaGetLastError();
}

}  // namespace mss
