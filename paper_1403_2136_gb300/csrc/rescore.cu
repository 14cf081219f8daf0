// a10: exact rescoring of the learned proposal's candidate fragments.
//
// For each read and each of its K candidate fragments f, the same quantity as the exhaustive
// scan ("First phase of MaxSSmap"): the maximum, over the diagonals d in [fF, (f+1)F) and
// both strands, of the maximum-scoring subsequence of the substitution scores along d.  Then
// the best and second-best fragment among the candidates (higher score, then lower fragment)
// and the best diagonal/strand inside the best one (+ strand first, then smaller d); with the
// neighbour rule of the context the second is the best candidate not adjacent to the best.
//
// k_rescore_scan: one CTA per read; the read's two strands sit in a shared-memory profile;
// each pass covers 2048 diagonals of two candidates at once (each half of the CTA: 128
// threads x 8 packed lane pairs (d, d + 8) per strand), with each half's genome window
// expanded into PRMT selector words laid out [position mod 16][position div 16] (four
// positions' codes per multiply, as in the exhaustive scan) and the recurrence in packed
// 16-bit lanes (f16 FMA-relu when exact, else int16 DPX add-max), as in the exhaustive scan.
// k_rescore_pick: one warp per read; top-2 over the candidate maxima, then a plain int32
// rescan of the best fragment for its best diagonal and strand.
#include <algorithm>

#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"
#include "prop.h"

namespace mss {

namespace {

template <bool B>
struct BoolTagRs {
  static constexpr bool value = B;
};

constexpr int kRsThreads = 256;
constexpr int kRsHalf = kRsThreads / 2;         // threads per candidate
constexpr int kRsD = 8;                         // lane pairs per thread and strand
constexpr int kRsSpan = 2 * kRsD;               // diagonals per thread
constexpr int kRsTile = kRsHalf * kRsSpan;      // diagonals per pass and candidate (2048)

struct RsArgs {
  const uint32_t* g2;
  const uint32_t* gm;
  int64_t F;
  const char* reads;
  const int64_t* offsets;
  const int32_t* idx;
  int32_t R;
  int32_t max_len;
  const int32_t* cand;   // [R][K]; entries < 0 are skipped
  int32_t K;
  int32_t* cand_max;     // [R][K] out: exact score of each candidate (-1 for skipped)
  int32_t* err;
  int32_t W;             // selector columns
  uint32_t prof_match, prof_mismatch, mm_word;
};

inline int32_t rs_mpad(int32_t m) { return std::max(kRsD, (m + kRsD - 1) / kRsD * kRsD); }
__host__ __device__ inline size_t rs_prof_bytes(int32_t max_len) {
  const int32_t mp = max_len < kRsD ? kRsD : (max_len + kRsD - 1) / kRsD * kRsD;
  return ((size_t)(mp + 1) * 2 * 4 + 15) & ~(size_t)15;  // one padding row: read one step ahead
}
inline int rs_cols(int32_t max_len) { return (kRsTile + rs_mpad(max_len) + 2 * kRsD + kRsSpan - 1) / kRsSpan; }
inline size_t rs_smem(int32_t max_len) {
  return rs_prof_bytes(max_len) + 2 * (size_t)kRsSpan * rs_cols(max_len) * 4 + 16;
}

template <bool F16>
__global__ void __launch_bounds__(kRsThreads, 3) k_rescore_scan(RsArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int tid = threadIdx.x, lane = tid & 31;
  const int half = tid >> 7, ltid = tid & (kRsHalf - 1);
  const int i = blockIdx.x;
  const int ridx = a.idx ? a.idx[i] : i;
  const int64_t off = a.offsets[ridx];
  const int64_t l = a.offsets[ridx + 1] - off;
  const int32_t m = l < 0 ? 0 : (l > a.max_len ? a.max_len : (int32_t)l);
  if (l > a.max_len && tid == 0) atomicOr(a.err, ERR_BAD_LEN);
  const int mpad = max(kRsD, (m + kRsD - 1) / kRsD * kRsD);
  const int W = a.W;
  uint32_t* prof = reinterpret_cast<uint32_t*>(smem);                                 // [mpad + 1][2]
  uint32_t* sel = reinterpret_cast<uint32_t*>(smem + rs_prof_bytes(a.max_len)) + half * kRsSpan * W;
  int32_t* s_best = reinterpret_cast<int32_t*>(smem + rs_prof_bytes(a.max_len) + 2 * (size_t)kRsSpan * W * 4);

  // profile rows k = 0..mpad: word q = 0 forward, q = 1 reverse complement
  for (int e = tid; e < (mpad + 1) * 2; e += kRsThreads) {
    const int k = e >> 1, q = e & 1;
    uint32_t code = 4;
    if (k < m) {
      code = ascii_code((uint8_t)a.reads[off + (q ? m - 1 - k : k)]);
      if (code == 5) {
        atomicOr(a.err, ERR_BAD_CHAR);
        code = 4;
      }
      if (q && code < 4) code = 3 - code;
    }
    prof[e] = profile_word(code, a.prof_match, a.prof_mismatch);
  }
  if (tid < 2) s_best[tid] = 0;
  const uint32_t mmw = a.mm_word;
  const int ncols = (kRsTile + mpad + kRsD + kRsSpan - 1) / kRsSpan;
  const int ntile = (int)((a.F + kRsTile - 1) / kRsTile);
  const int nfull = m / kRsD * kRsD, rem = m - nfull;
  const int last_parity = (m - 1) & 1;

  for (int c0 = 0; c0 < a.K; c0 += 2) {
    // this half's candidate (the second half idles when K is odd)
    const int c = c0 + half;
    const int32_t f = c < a.K ? a.cand[(int64_t)i * a.K + c] : -1;
    for (int tt = 0; tt < ntile; ++tt) {
      const int64_t ts = (int64_t)f * a.F + (int64_t)tt * kRsTile;
      const int64_t lim = a.F - (int64_t)tt * kRsTile;  // pass positions p < lim are diagonals of f
      __syncthreads();  // the previous pass has finished reading the selectors
      if (f >= 0) {
        // selector column col: positions P = col*16 .. P+15 and their partners at +8, one byte
        // per position (the 2-bit code, or the N code where the valid bit is 0), four
        // positions per word built with carry-free multiplies
        for (int col = ltid; col < ncols; col += kRsHalf) {
          const int64_t q = ts + (int64_t)col * kRsSpan;
          const int64_t w2 = q >> 4, wm = q >> 5;
          const int sh = 2 * (int)(q & 15);
          const uint32_t g0 = a.g2[w2], g1 = a.g2[w2 + 1], g2w = a.g2[w2 + 2];
          const uint32_t lo = (uint32_t)(((((uint64_t)g1) << 32) | g0) >> sh);   // positions 0..15
          const uint32_t hi = (uint32_t)(((((uint64_t)g2w) << 32) | g1) >> sh);  // positions 16..31
          const uint32_t vw = (uint32_t)(((((uint64_t)a.gm[wm + 1]) << 32) | a.gm[wm]) >> (int)(q & 31));
          uint32_t nb[3 * kRsD / 4];
#pragma unroll
          for (int k = 0; k < 3 * kRsD / 4; ++k) {
            const uint32_t b = prmt(k < 4 ? lo : hi, 0u, 0x4440u | (uint32_t)(k & 3));
            const uint32_t codes = ((((b * 4097u) & 0x000F000Fu) * 65u) & 0x03030303u);
            const uint32_t vs = ((((vw >> (4 * k)) & 0xFu) * 0x00204081u) & 0x01010101u);
            nb[k] = codes + (F16 ? 5u : 4u) * (0x01010101u - vs);
          }
#pragma unroll
          for (int r = 0; r < kRsSpan; ++r) {
            const uint32_t t2 =
                prmt(nb[r >> 2], nb[(r + kRsD) >> 2], (uint32_t)(r & 3) | ((uint32_t)(4 + (r & 3)) << 4) | 0x8800u);
            sel[r * W + col] = F16 ? t2 * 16u + 0x0404u : t2 * 17u + 0x8080u;
          }
        }
      }
      __syncthreads();
      if (f >= 0) {
        uint32_t win[kRsD], H[2][kRsD], M[2][kRsD];
#pragma unroll
        for (int j = 0; j < kRsD; ++j) win[j] = sel[j * W + ltid];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int j = 0; j < kRsD; ++j) H[q][j] = 0u, M[q][j] = 0u;
        uint2 pnext = reinterpret_cast<const uint2*>(prof)[0];
        // blocks of 8 steps (pair j of step k0 + u reads win[(j + u) % 8]), the last one cut
        // at the read's length
        auto block = [&](int k0, auto tail, int nvalid) {
          constexpr bool kTail = decltype(tail)::value;
          const int kk = k0 + kRsD;
          const uint32_t* sp = sel + (kk % kRsSpan) * W + ltid + kk / kRsSpan;
          const uint2* pp = reinterpret_cast<const uint2*>(prof) + k0 + 1;
#pragma unroll
          for (int u = 0; u < kRsD; ++u) {
            if (kTail && u >= nvalid) break;
            const uint32_t pw[2] = {pnext.x, pnext.y};
            pnext = pp[u];
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
              for (int j = 0; j < kRsD; ++j) {
                const uint32_t s = prmt(pw[q], mmw, win[(j + u) % kRsD]);
                const uint32_t h = kadane_step<F16>(H[q][j], s);
                if ((u & 1) != (j & 1)) M[q][j] = __vimax3_s16x2(M[q][j], H[q][j], h);
                H[q][j] = h;
              }
            win[u] = sp[u * W];
          }
        };
        for (int k0 = 0; k0 < nfull; k0 += kRsD) block(k0, BoolTagRs<false>{}, kRsD);
        if (rem > 0) block(nfull, BoolTagRs<true>{}, rem);
        // the pairs of the last step's parity hold one value not yet folded
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int j = 0; j < kRsD; ++j)
            if ((j & 1) == last_parity) M[q][j] = __vimax3_s16x2(M[q][j], H[q][j], 0u);

        // this thread's diagonals: pass positions ltid*16 + j (low lane) and + 8 + j (high lane)
        const int p0 = ltid * kRsSpan;
        uint32_t x = 0u;
#pragma unroll
        for (int j = 0; j < kRsD; ++j) {
          const uint32_t mask =
              ((p0 + j < lim) ? 0x0000FFFFu : 0u) | ((p0 + kRsD + j < lim) ? 0xFFFF0000u : 0u);
          x = __vimax3_s16x2(x, M[0][j] & mask, M[1][j] & mask);
        }
        int32_t v = max(lane_value<F16>(x & 0xFFFFu), lane_value<F16>(x >> 16));
        v = __reduce_max_sync(0xffffffffu, v);
        if (lane == 0 && v > 0) atomicMax(&s_best[half], v);
      }
    }
    __syncthreads();
    if (ltid == 0 && c < a.K) {
      a.cand_max[(int64_t)i * a.K + c] = f >= 0 ? s_best[half] : -1;
      s_best[half] = 0;  // the next pair's first pass starts after a barrier
    }
  }
}

constexpr int kPickWarps = 4;
constexpr int kPickChunk = 512;

struct PickArgs {
  const uint32_t* g2;
  const uint32_t* gm;
  int64_t F;
  const char* reads;
  const int64_t* offsets;
  const int32_t* idx;
  int32_t R;
  int32_t max_len;
  const int32_t* cand;
  const int32_t* cand_max;
  int32_t K;
  int32_t match, mismatch;
  int32_t exclude_neighbors;
  void* hits;
};

__global__ void __launch_bounds__(kPickWarps * 32) k_rescore_pick(PickArgs a) {
  __shared__ uint8_t s_gen[kPickWarps][kPickChunk + MSS_MAX_READ_LEN + 16];
  __shared__ uint8_t s_q[kPickWarps][2][MSS_MAX_READ_LEN];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * kPickWarps + wib;
  if (i >= a.R) return;
  const int ridx = a.idx ? a.idx[i] : i;
  const int64_t off = a.offsets[ridx];
  const int64_t l = a.offsets[ridx + 1] - off;
  const int32_t m = l < 0 ? 0 : (l > a.max_len ? a.max_len : (int32_t)l);

  Top4 t4 = top4_empty();
  for (int c = lane; c < a.K; c += 32) {
    const int32_t f = a.cand[(int64_t)i * a.K + c];
    if (f < 0) continue;
    t4 = top4_insert(t4, a.cand_max[(int64_t)i * a.K + c], f);
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) t4 = top4_merge(t4, top4_shfl_xor(t4, s));
  // the best candidate and the second: the next one, or with the neighbour rule the first one
  // not adjacent to the best
  Top2 acc{t4.s[0], t4.f[0], -1, 0x7fffffff};
#pragma unroll
  for (int j = 3; j >= 1; --j) {
    const bool adjacent = t4.f[j] == t4.f[0] - 1 || t4.f[j] == t4.f[0] + 1;
    if (t4.s[j] >= 0 && !(a.exclude_neighbors && adjacent)) acc.s2 = t4.s[j], acc.f2 = t4.f[j];
  }

  int32_t bestK = -1, bestS = 0;
  int64_t bestD = 0;
  if (acc.s1 >= 0) {
    for (int k = lane; k < m; k += 32) {
      uint32_t cf = ascii_code((uint8_t)a.reads[off + k]);
      if (cf > 4) cf = 4;
      s_q[wib][0][k] = (uint8_t)cf;
      s_q[wib][1][m - 1 - k] = (uint8_t)(cf < 4 ? 3 - cf : 4);
    }
    const int64_t d_lo = (int64_t)acc.f1 * a.F, d_hi = d_lo + a.F;
    for (int sg = 0; sg < 2; ++sg) {
      for (int64_t d0 = d_lo; d0 < d_hi; d0 += kPickChunk) {
        const int64_t nd = (d_hi - d0 < (int64_t)kPickChunk) ? d_hi - d0 : (int64_t)kPickChunk;
        __syncwarp();
        for (int64_t x = lane; x < nd + m; x += 32) s_gen[wib][x] = (uint8_t)genome_code(a.g2, a.gm, d0 + x);
        __syncwarp();
        for (int64_t x = lane; x < nd; x += 32) {
          int32_t h = 0, mx = 0;
          for (int k = 0; k < m; ++k) {
            const uint32_t qc = s_q[wib][sg][k], gc = s_gen[wib][x + k];
            h += (qc < 4 && qc == gc) ? a.match : a.mismatch;
            h = max(h, 0);
            mx = max(mx, h);
          }
          if (mx > bestK) {  // lanes visit (strand, d) in increasing order
            bestK = mx;
            bestS = sg;
            bestD = d0 + x;
          }
        }
      }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const int32_t oK = __shfl_xor_sync(0xffffffffu, bestK, s);
      const int32_t oS = __shfl_xor_sync(0xffffffffu, bestS, s);
      const int64_t oD = __shfl_xor_sync(0xffffffffu, bestD, s);
      if (oK > bestK || (oK == bestK && (oS < bestS || (oS == bestS && oD < bestD)))) {
        bestK = oK;
        bestS = oS;
        bestD = oD;
      }
    }
  }
  if (lane == 0) {
    mss_hit h;
    h.best_frag = acc.s1 < 0 ? -1 : acc.f1;
    h.best_score = acc.s1 < 0 ? 0 : acc.s1;
    h.second_frag = acc.s2 < 0 ? -1 : acc.f2;
    h.second_score = acc.s2 < 0 ? 0 : acc.s2;
    h.offset = bestD;
    h.strand = bestS;
    const bool repeat = (h.best_score == 0) || (10LL * h.second_score >= 9LL * h.best_score);
    h.flags = repeat ? MSS_HIT_REPEAT : 0;
    reinterpret_cast<mss_hit*>(a.hits)[i] = h;
  }
}

}  // namespace

cudaError_t prop_rescore(const uint32_t* g2, const uint32_t* gm, int64_t F, const char* reads, const int64_t* offsets,
                         const int32_t* idx, int32_t R, int32_t max_len, const int32_t* cand, int32_t K,
                         int32_t match, int32_t mismatch, int32_t exclude_neighbors, void* hits,
                         int32_t* cand_scores, int32_t* err, int num_sms, cudaStream_t s) {
  (void)num_sms;
  if (R <= 0 || K <= 0) return cudaSuccess;
  if (max_len < 1 || max_len > MSS_MAX_READ_LEN || !cand_scores) return cudaErrorInvalidValue;
  RsArgs a;
  a.g2 = g2;
  a.gm = gm;
  a.F = F;
  a.reads = reads;
  a.offsets = offsets;
  a.idx = idx;
  a.R = R;
  a.max_len = max_len;
  a.cand = cand;
  a.K = K;
  a.cand_max = cand_scores;
  a.err = err;
  a.W = rs_cols(max_len);
  const bool f16 = f16_path_exact(max_len, match, mismatch);
  if (f16) {
    a.prof_match = (int_to_f16_bits(match) >> 8) & 0xFFu;
    a.prof_mismatch = (int_to_f16_bits(mismatch) >> 8) & 0xFFu;
    a.mm_word = a.prof_mismatch << 8;
  } else {
    a.prof_match = (uint32_t)match & 0xFFu;
    a.prof_mismatch = (uint32_t)mismatch & 0xFFu;
    a.mm_word = a.prof_mismatch * 0x01010101u;
  }
  const size_t smem = rs_smem(max_len);
  const void* fn = f16 ? reinterpret_cast<const void*>(&k_rescore_scan<true>)
                       : reinterpret_cast<const void*>(&k_rescore_scan<false>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  e = cudaLaunchKernel(fn, dim3((unsigned)R), dim3(kRsThreads), args, smem, s);
  if (e != cudaSuccess) return e;
  PickArgs b;
  b.g2 = g2;
  b.gm = gm;
  b.F = F;
  b.reads = reads;
  b.offsets = offsets;
  b.idx = idx;
  b.R = R;
  b.max_len = max_len;
  b.cand = cand;
  b.cand_max = cand_scores;
  b.K = K;
  b.match = match;
  b.mismatch = mismatch;
  b.exclude_neighbors = exclude_neighbors;
  b.hits = hits;
  k_rescore_pick<<<(unsigned)((R + kPickWarps - 1) / kPickWarps), kPickWarps * 32, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace mss
