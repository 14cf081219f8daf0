// a3-a5: maximum-scoring-subsequence scan of every read (both strands) along every diagonal,
// per-fragment maxima and the per-read top-2 fragments; then the best-fragment rescan that
// recovers the best diagonal and strand.
//
// Method ("First phase of MaxSSmap", "Maximum scoring subsequence"): for a read q and
// diagonal d, the substitution scores s_k = score(q[k], g[d+k]) are reduced by the linear
// maximum-scoring-subsequence scan H = max(H + s, 0), M = max(M, H); fragment f keeps the
// maximum M over its diagonals [fF, (f+1)F) (windows run into the next fragment); the read
// keeps the best and the second-best fragment.
//
// GB300 design (not the paper's thread-per-fragment layout):
//   * one work item = a group of RQ query sequences (RQ/2 reads x 2 strands) against one
//     chunk of the genome; persistent CTAs pull items from a device queue, longest reads
//     first;
//   * a CTA tile is NT*2D consecutive diagonals; thread t owns diagonals t*2D + [0, 2D) as D
//     packed 16-bit lane pairs (d, d + D) per query;
//   * the 2-bit genome of a tile is staged by a bulk (TMA) copy into a double buffer and
//     expanded once into PRMT selector words laid out [lane row][thread column] so that a warp
//     reads 32 consecutive words (the same idea as the paper's transposed genome, Figure 2,
//     done in shared memory);
//   * the query profile (one byte per genome base per read position) sits in shared memory
//     and is read as warp-wide broadcasts;
//   * score generation is one PRMT per lane pair; the recurrence H runs either as a packed
//     int16 DPX add-max (variant 0, any scores) or as a packed f16 FMA with relu on the FMA
//     pipe (variant 1, exact for small integer scores); the running maximum M is a packed
//     3-input DPX max every second step;
//   * per-fragment maxima go through warp redux + shared-memory atomics into a ring of
//     fragment slots, and completed fragments are folded by warp shuffles into a top-2
//     summary per read; chunks are merged exactly by the finalize kernel.
#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"

namespace mss {

template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

// D lane pairs per thread, NT threads, reads up to MAXL bases (selector rows sized for it)
template <int D, int NT, int MAXL>
struct ScanGeo {
  static constexpr int kSpan = 2 * D;                                     // diagonals per thread
  static constexpr int kTile = NT * kSpan;                                // diagonals per tile
  static constexpr int kSelCols = (kTile + MAXL + 2 * D + kSpan - 1) / kSpan;
  static constexpr int kSelWords = kSpan * kSelCols;                      // one selector buffer
  static constexpr int kRawPos = ((kTile + MAXL + 4 * D + 16 + 127) / 128) * 128;
  static constexpr uint32_t kRawG2Bytes = kRawPos / 4;
  static constexpr uint32_t kRawGmBytes = kRawPos / 8;
  static constexpr uint32_t kRawBytes = kRawG2Bytes + kRawGmBytes;
};

struct SmemLayout {
  size_t prof, profn, sel, raw, ring, top, mbar, misc, total;
};

// pssm: a second profile array holds, per read position and query, the word a genome N
// selects (the position's mismatch score)
template <int D, int RQ, int NT, int MAXL>
__host__ __device__ inline SmemLayout scan_layout(int32_t max_len, int32_t ring_slots, bool pssm) {
  using Geo = ScanGeo<D, NT, MAXL>;
  SmemLayout L;
  size_t mpad_max = (size_t)((max_len + 7) & ~7);
  L.prof = 0;
  L.profn = L.prof + (mpad_max + 1) * RQ * 4;  // one padding row: the scan reads one row ahead
  L.sel = L.profn + (pssm ? (mpad_max + 1) * RQ * 4 : 0);
  L.raw = L.sel + 2 * (size_t)Geo::kSelWords * 4;  // two selector buffers (tile t and t+1)
  L.raw = (L.raw + 127) & ~(size_t)127;
  L.ring = L.raw + 2 * (size_t)Geo::kRawBytes;
  L.top = L.ring + (size_t)(RQ / 2) * ring_slots * 4;
  L.top = (L.top + 15) & ~(size_t)15;
  L.mbar = L.top + (size_t)(RQ / 2) * sizeof(Top4);
  L.misc = L.mbar + 16;                     // item (4 B), read lengths at +16, offsets at +32
  L.total = L.misc + 32 + (size_t)(RQ / 2) * 8;
  return L;
}

// STEP = 1: every read base; STEP = 2: every other read base ("MaxSSmap_fast"), so step k of
// diagonal d compares read base STEP*k with genome base d + STEP*k.
// PSSM: position-specific scores from base qualities ("Incorporating base qualities and
// position specific scoring matrix"), int16 lanes only: the profile bytes and the genome-N word
// come from the read position's quality.
template <bool F16, int D, int RQ, int NT, int MAXL, int MINB, int STEP, bool PSSM>
__global__ void __launch_bounds__(NT, MINB) k_scan(ScanArgs a) {
  using Geo = ScanGeo<D, NT, MAXL>;
  constexpr int RG = RQ / 2;
  constexpr int SPAN = Geo::kSpan;
  constexpr int TILE = Geo::kTile;
  constexpr int W = Geo::kSelCols;
  constexpr int BS = D / STEP;  // steps per block: a block consumes D genome positions
  static_assert(RQ % 4 == 0, "profile rows are read as uint4");
  static_assert(STEP == 1 || STEP == 2, "read step 1 or 2");
  static_assert(BS % 2 == 0, "the running max is updated every second step");
  static_assert(!(PSSM && F16), "position-specific scores run on the int16 lanes");
  static_assert(RG <= 4, "read lengths occupy 16 bytes of the misc area");

  extern __shared__ __align__(128) uint8_t smem[];
  const SmemLayout L = scan_layout<D, RQ, NT, MAXL>(a.max_len, a.ring_slots, PSSM);
  uint32_t* prof = reinterpret_cast<uint32_t*>(smem + L.prof);
  uint32_t* profn = reinterpret_cast<uint32_t*>(smem + L.profn);
  uint32_t* const sel_base = reinterpret_cast<uint32_t*>(smem + L.sel);
  uint8_t* raw = smem + L.raw;
  int32_t* ring = reinterpret_cast<int32_t*>(smem + L.ring);
  Top4* top = reinterpret_cast<Top4*>(smem + L.top);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
  int32_t* s_item = reinterpret_cast<int32_t*>(smem + L.misc);
  int32_t* s_len = reinterpret_cast<int32_t*>(smem + L.misc + 16);      // [RG]
  int64_t* s_off = reinterpret_cast<int64_t*>(smem + L.misc + 32);      // [RG]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = a.ring_slots;
  const uint32_t mmw = a.mm_word;

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity[2] = {0u, 0u};
  int32_t armed[2] = {-1, -1};  // thread 0: parity of the last phase armed on each mbarrier
  bool timed_out = false;
  constexpr uint64_t kWaitLimitNs = 2000000000ull;  // a tile's copy completes in microseconds

  for (;;) {
    if (tid == 0) *s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = *s_item;
    if (item >= a.n_items) break;
    const int g = item / a.n_chunks;
    const int c = item - g * a.n_chunks;

    if (tid < RG) {
      const int p = g * RG + tid;
      int32_t len = 0;
      int64_t off = 0;
      if (p < a.R) {
        const int ridx = a.order[p];
        off = a.offsets[ridx];
        int64_t l = a.offsets[ridx + 1] - off;
        len = l < 0 ? 0 : (l > a.max_len ? a.max_len : (int32_t)l);
      }
      s_len[tid] = len;
      s_off[tid] = off;
      top[tid] = top4_empty();
    }
    for (int e = tid; e < RG * S; e += NT) ring[e] = 0;
    __syncthreads();

    int32_t mmax = 0;
#pragma unroll
    for (int r = 0; r < RG; ++r) mmax = max(mmax, s_len[r]);
    const int nsteps = (mmax + STEP - 1) / STEP;
    const int mpad = max(BS, (nsteps + BS - 1) / BS * BS);

    // query profile: prof[k * RQ + q] for step k (read base STEP*k), q = 2r (forward) or 2r + 1
    // (reverse complement)
    for (int e = tid; e < mpad * RQ; e += NT) {
      const int k = e / RQ, q = e - k * RQ, r = q >> 1;
      const int len = s_len[r];
      const int kr = STEP * k;
      uint32_t code = 4;
      uint32_t pma = a.prof_match, pmm = a.prof_mismatch;
      if (kr < len) {
        const int64_t pos = s_off[r] + ((q & 1) ? (len - 1 - kr) : kr);
        if (PSSM) {  // the base's own quality (the reverse strand's base k is read base len-1-k)
          int Q = (int)(uint8_t)a.quals[pos] - 33;
          if (Q < 0 || Q >= kQualLevels) {
            atomicOr(a.err, ERR_BAD_QUAL);
            Q = 0;
          }
          pma = (uint32_t)a.qtab[2 * Q] & 0xFFu;
          pmm = (uint32_t)a.qtab[2 * Q + 1] & 0xFFu;
        }
        code = ascii_code((uint8_t)a.reads[pos]);
        if (code == 5) {
          atomicOr(a.err, ERR_BAD_CHAR);
          code = 4;
        }
        if ((q & 1) && code < 4) code = 3 - code;
      }
      prof[e] = profile_word(code, pma, pmm);
      if (PSSM) profn[e] = pmm * 0x01010101u;
    }

    const int64_t c0 = (int64_t)c * a.chunk_len;
    const int64_t c1 = min(c0 + a.chunk_len, a.Gp);
    const int ntiles = (int)((c1 - c0 + TILE - 1) / TILE);
    const int32_t f_lo = (int32_t)(c0 / a.F);
    const int32_t f_end = (int32_t)((c1 - 1) / a.F) + 1;
    int32_t fold_next = f_lo;
    // fragment of the current tile start and of this thread's first diagonal, with remainders,
    // advanced by TILE per tile without dividing again
    const int64_t tile_step_q = TILE / a.F, tile_step_rem = TILE % a.F;
    int64_t tile_frag = c0 / a.F, tile_rem = c0 - tile_frag * a.F;
    int64_t th_frag = (c0 + (int64_t)tid * SPAN) / a.F;
    int64_t th_rem = c0 + (int64_t)tid * SPAN - th_frag * a.F;

    auto issue = [&](int t, int buf) {
      const int64_t ts = c0 + (int64_t)t * TILE;
      uint8_t* dst = raw + buf * Geo::kRawBytes;
      fence_proxy_async_smem();
      armed[buf] = (int32_t)parity[buf];
      mbar_arrive_expect_tx(&mbar[buf], Geo::kRawBytes);
      tma_load_1d(dst, reinterpret_cast<const uint8_t*>(a.g2) + ts / 4, Geo::kRawG2Bytes, &mbar[buf]);
      tma_load_1d(dst + Geo::kRawG2Bytes, reinterpret_cast<const uint8_t*>(a.gm) + ts / 8, Geo::kRawGmBytes,
                  &mbar[buf]);
    };
    auto fold = [&](int r, int32_t lo, int32_t hi) {  // fragments [lo, hi) of read r, one warp
      if (hi - lo <= 8) {  // the usual case (F >= a tile / 8): one lane inserts them in order
        if (lane == 0) {
          Top4 t = top[r];
          for (int32_t f = lo; f < hi; ++f) {
            const int slot = r * S + (int)(f % S);
            t = top4_insert(t, ring[slot], f);
            ring[slot] = 0;
          }
          top[r] = t;
        }
        __syncwarp();
        return;
      }
      Top4 acc = top4_empty();
      for (int32_t base = lo; base < hi; base += 32) {
        const int32_t f = base + lane;
        if (f < hi) {
          const int slot = r * S + (int)(f % S);
          const int32_t v = ring[slot];
          ring[slot] = 0;
          acc = top4_insert(acc, v, f);
        }
      }
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) acc = top4_merge(acc, top4_shfl_xor(acc, m));
      if (lane == 0) top[r] = top4_merge(top[r], acc);
    };

    __syncthreads();  // profile and ring ready
    if (tid == 0) issue(0, 0);

    for (int t = 0; t < ntiles; ++t) {
      const int buf = t & 1;
      // selector buffer of this tile: written by the expansion below, read by the scan; the
      // other buffer may still be read by warps finishing tile t-1 (one barrier per tile)
      uint32_t* const sel = sel_base + buf * Geo::kSelWords;
      if (tid == 0 && t + 1 < ntiles) issue(t + 1, buf ^ 1);
      if (!mbar_wait(&mbar[buf], parity[buf], kWaitLimitNs)) timed_out = true;
      parity[buf] ^= 1u;

      // expand the staged 2-bit genome into selector words: sel[row * W + col] is the
      // selector of tile position p = col * SPAN + row (codes at p and p + D)
      {
        const uint32_t* rg2 = reinterpret_cast<const uint32_t*>(raw + buf * Geo::kRawBytes);
        const uint32_t* rgm = reinterpret_cast<const uint32_t*>(raw + buf * Geo::kRawBytes + Geo::kRawG2Bytes);
        // one selector column per thread: positions P .. P + SPAN - 1 and their partners at
        // +D; their 2-bit codes and valid bits fit in two aligned words each.  One byte per
        // position, n = the 2-bit code, or the N code where the valid bit is 0 (packed N and
        // padding carry code 0), four positions per word, built with carry-free multiplies:
        // bytes of 4 codes -> 2-bit fields 8 bits apart; 4 valid bits -> bit 0 of 4 bytes
        auto nbytes = [&](uint64_t gw, uint32_t vw, int k) {
          const uint32_t b = prmt(k < 4 ? (uint32_t)gw : (uint32_t)(gw >> 32), 0u, 0x4440u | (uint32_t)(k & 3));
          const uint32_t codes = ((((b * 4097u) & 0x000F000Fu) * 65u) & 0x03030303u);
          const uint32_t vs = ((((vw >> (4 * k)) & 0xFu) * 0x00204081u) & 0x01010101u);
          return codes + (F16 ? 5u : 4u) * (0x01010101u - vs);
        };
        auto window = [&](int P, uint64_t& gw, uint32_t& vw) {
          gw = ((((uint64_t)rg2[(P >> 4) + 1]) << 32) | rg2[P >> 4]) >> (2 * (P & 15));
          vw = (uint32_t)(((((uint64_t)rgm[(P >> 5) + 1]) << 32) | rgm[P >> 5]) >> (P & 31));
        };
        // bytes [n(P + r), n(P + r + D), 0, 0] (the zero bytes replicate the sign of a byte
        // <= 5), then the selector word of make_sel with one multiply-add
        auto selector = [&](uint32_t na, uint32_t nbw, int r) {
          const uint32_t t2 = prmt(na, nbw, (uint32_t)(r & 3) | ((uint32_t)(4 + (r & 3)) << 4) | 0x8800u);
          return F16 ? t2 * 16u + 0x0404u : t2 * 17u + 0x8080u;
        };
        {
          const int col = tid;  // the tile's own columns: one per thread
          uint64_t gw;
          uint32_t vw;
          window(col * SPAN, gw, vw);
          uint32_t nb[3 * D / 4];
#pragma unroll
          for (int k = 0; k < 3 * D / 4; ++k) nb[k] = nbytes(gw, vw, k);
#pragma unroll
          for (int r = 0; r < SPAN; ++r) sel[r * W + col] = selector(nb[r >> 2], nb[(r + D) >> 2], r);
        }
        // the columns past the tile (the window's overhang) selector by selector, spread over
        // the threads, so that no thread builds two whole columns
        const int ncols = (TILE + STEP * mpad + D + SPAN - 1) / SPAN;
        for (int e = tid; e < (ncols - NT) * SPAN; e += NT) {
          const int col = NT + e / SPAN, r = e % SPAN;
          uint64_t gw;
          uint32_t vw;
          window(col * SPAN, gw, vw);
          sel[r * W + col] = selector(nbytes(gw, vw, r >> 2), nbytes(gw, vw, (r + D) >> 2), r);
        }
      }
      __syncthreads();

      const int64_t ts = c0 + (int64_t)t * TILE;
      {
        const int64_t tf = tile_frag;  // = ts / F
        const int32_t done = (int32_t)(tf < (int64_t)f_end ? tf : (int64_t)f_end);  // fragments < done are complete
        if (warp < RG && done > fold_next) fold(warp, fold_next, done);
        fold_next = max(fold_next, done);
      }

      // ---- the scan of this tile
      uint32_t win[D];
#pragma unroll
      for (int j = 0; j < D; ++j) win[j] = sel[j * W + tid];
      // H: latest Kadane value per lane pair; M: running maximum.  Each pair folds two new H
      // values into M with one 3-input max every second step; pairs with odd j fold on even
      // steps and pairs with even j on odd steps, so every step carries the same mix of
      // integer-pipe (PRMT, max) and FMA-pipe (H update) instructions.
      uint32_t H[RQ][D], M[RQ][D];
#pragma unroll
      for (int q = 0; q < RQ; ++q)
#pragma unroll
        for (int j = 0; j < D; ++j) H[q][j] = 0u, M[q][j] = 0u;

      // profile row of the next step, loaded one step ahead (hides the shared-memory latency,
      // also across block boundaries; the row after the last is padding)
      uint4 pnext[RQ / 4], nnext[RQ / 4];
#pragma unroll
      for (int v = 0; v < RQ / 4; ++v) {
        pnext[v] = reinterpret_cast<const uint4*>(prof)[v];
        if (PSSM) nnext[v] = reinterpret_cast<const uint4*>(profn)[v];
      }

      // whole blocks of BS steps, then the last block cut at the group's longest read: steps
      // past it would only score padding (mismatches), which lowers H and never raises M
      const int nfull = nsteps / BS * BS;
      const int rem = nsteps - nfull;
      auto block = [&](int k0, auto tail, int nvalid) {
        constexpr bool kTail = decltype(tail)::value;
        // positions entering the window during this block: p = tid*SPAN + STEP*k0 + D + i,
        // i < D, all in one selector row band and one column; pair j of step k = k0 + u reads
        // position tid*SPAN + STEP*k + j, kept in win[(j + STEP*u) % D] (STEP*k0 is a
        // multiple of D)
        const int kk = STEP * k0 + D;
        const uint32_t* sp = sel + (kk % SPAN) * W + tid + kk / SPAN;
        const uint4* pp = reinterpret_cast<const uint4*>(prof + (k0 + 1) * RQ);
        const uint4* pn = reinterpret_cast<const uint4*>(profn + (k0 + 1) * RQ);
#pragma unroll
        for (int u = 0; u < BS; ++u) {
          if (kTail && u >= nvalid) break;  // the same for every thread of the CTA
          uint32_t pw[RQ], nw[RQ];
#pragma unroll
          for (int v = 0; v < RQ / 4; ++v) {
            pw[4 * v + 0] = pnext[v].x;
            pw[4 * v + 1] = pnext[v].y;
            pw[4 * v + 2] = pnext[v].z;
            pw[4 * v + 3] = pnext[v].w;
            if (PSSM) {
              nw[4 * v + 0] = nnext[v].x;
              nw[4 * v + 1] = nnext[v].y;
              nw[4 * v + 2] = nnext[v].z;
              nw[4 * v + 3] = nnext[v].w;
            }
          }
#pragma unroll
          for (int v = 0; v < RQ / 4; ++v) {
            pnext[v] = pp[u * (RQ / 4) + v];
            if (PSSM) nnext[v] = pn[u * (RQ / 4) + v];
          }
#pragma unroll
          for (int q = 0; q < RQ; ++q) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
              const uint32_t s = prmt(pw[q], PSSM ? nw[q] : mmw, win[(j + STEP * u) % D]);
              const uint32_t h = kadane_step<F16>(H[q][j], s);
              if ((u & 1) != (j & 1)) M[q][j] = __vimax3_s16x2(M[q][j], H[q][j], h);
              H[q][j] = h;
            }
          }
#pragma unroll
          for (int e = 0; e < STEP; ++e) win[(STEP * u + e) % D] = sp[(STEP * u + e) * W];
        }
      };
      for (int k0 = 0; k0 < nfull; k0 += BS) block(k0, BoolTag<false>{}, BS);
      if (rem > 0) block(nfull, BoolTag<true>{}, rem);
      // step u folds into pair j's maximum when u and j differ in parity (blocks have an even
      // number of steps, so u's parity is the step's): after the last step, the pairs of its
      // parity hold one value not yet folded
      const int last_parity = (nsteps - 1) & 1;
#pragma unroll
      for (int q = 0; q < RQ; ++q)
#pragma unroll
        for (int j = 0; j < D; ++j)
          if ((j & 1) == last_parity) M[q][j] = __vimax3_s16x2(M[q][j], H[q][j], 0u);

      // ---- per-fragment maxima of this thread's 2D diagonals
      const int64_t ds = ts + (int64_t)tid * SPAN;
      const int32_t fA = (int32_t)th_frag;          // = ds / F
      const int64_t bnd = ds - th_rem + a.F;        // start of fragment fA + 1
      const bool split = th_rem + SPAN > a.F;
      // advance the per-tile and per-thread fragment positions by one tile
      tile_rem += tile_step_rem;
      tile_frag += tile_step_q + (tile_rem >= a.F ? 1 : 0);
      if (tile_rem >= a.F) tile_rem -= a.F;
      th_rem += tile_step_rem;
      th_frag += tile_step_q + (th_rem >= a.F ? 1 : 0);
      if (th_rem >= a.F) th_rem -= a.F;
      const int32_t fA0 = __shfl_sync(0xffffffffu, fA, 0);
      const bool uni = __all_sync(0xffffffffu, (fA == fA0) && !split);
      uint32_t maskA[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const uint32_t lo = (ds + j < bnd) ? 0x0000FFFFu : 0u;
        const uint32_t hi = (ds + D + j < bnd) ? 0xFFFF0000u : 0u;
        maskA[j] = split ? (lo | hi) : 0xFFFFFFFFu;
      }
      // the maxima are non-negative, so their 16-bit patterns (f16 or int16) order like their
      // values: reduce the patterns, decode once
#pragma unroll
      for (int r = 0; r < RG; ++r) {
        uint32_t xa = 0u, xb = 0u;
        if (!split) {
#pragma unroll
          for (int j = 0; j < D; ++j) xa = __vimax3_s16x2(xa, M[2 * r][j], M[2 * r + 1][j]);
        } else {
#pragma unroll
          for (int j = 0; j < D; ++j) {
            xa = __vimax3_s16x2(xa, M[2 * r][j] & maskA[j], M[2 * r + 1][j] & maskA[j]);
            xb = __vimax3_s16x2(xb, M[2 * r][j] & ~maskA[j], M[2 * r + 1][j] & ~maskA[j]);
          }
        }
        const uint32_t pa = max(xa & 0xFFFFu, xa >> 16);
        if (uni) {
          const uint32_t pm = __reduce_max_sync(0xffffffffu, pa);
          if (lane == 0) {
            const int32_t v = lane_value<F16>(pm);
            if (v > 0) atomicMax(&ring[r * S + (int)(fA0 % S)], v);
          }
        } else {
          const int32_t vA = lane_value<F16>(pa);
          const int32_t vB = lane_value<F16>(max(xb & 0xFFFFu, xb >> 16));
          if (vA > 0) atomicMax(&ring[r * S + (int)(fA % S)], vA);
          if (vB > 0) atomicMax(&ring[r * S + (int)((fA + 1) % S)], vB);
        }
      }
    }
    __syncthreads();  // every fragment slot of the last tile is final

    if (warp < RG && f_end > fold_next) fold(warp, fold_next, f_end);
    __syncthreads();
    if (tid < RG) {
      const int p = g * RG + tid;
      const Top4 v = top[tid];
      int4* dst = a.partial + ((size_t)p * a.n_chunks + c) * 2;   // top-4 of this chunk
      dst[0] = make_int4(v.s[0], v.f[0], v.s[1], v.f[1]);
      dst[1] = make_int4(v.s[2], v.f[2], v.s[3], v.f[3]);
    }
    // the next item rewrites the profile, ring and summaries only after the barrier at its top
  }
  if (timed_out) atomicOr(a.err, ERR_TIMEOUT);
  // never leave with a bulk copy in flight: thread 0 waits (bounded) for the last phase it
  // armed on each buffer; phases that were already waited on return at once
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < 2; ++b)
      if (armed[b] >= 0 && !mbar_wait(&mbar[b], (uint32_t)armed[b], kWaitLimitNs)) atomicOr(a.err, ERR_TIMEOUT);
  }
}

// ---------------------------------------------------------------- host side of the scan
// (f16, D, RQ, NT, MAXL, min CTAs per SM, read step, position-specific scores)
#define MSS_SCAN_VARIANTS(X)               \
  X(false, 4, 8, 256, 512, 2, 1, false)    \
  X(true, 4, 8, 256, 512, 2, 1, false)     \
  X(false, 8, 4, 256, 512, 2, 1, false)    \
  X(true, 8, 4, 256, 512, 2, 1, false)     \
  X(false, 4, 4, 256, 512, 2, 1, false)    \
  X(true, 4, 4, 256, 512, 2, 1, false)     \
  X(false, 4, 8, 256, 2432, 2, 1, false)   \
  X(true, 4, 8, 256, 2432, 2, 1, false)    \
  X(false, 8, 4, 256, 2432, 2, 1, false)   \
  X(true, 8, 4, 256, 2432, 2, 1, false)    \
  X(false, 4, 4, 256, 2432, 2, 1, false)   \
  X(true, 4, 4, 256, 2432, 2, 1, false)    \
  X(false, 8, 4, 256, 512, 2, 2, false)    \
  X(true, 8, 4, 256, 512, 2, 2, false)     \
  X(false, 8, 4, 256, 2432, 2, 2, false)   \
  X(true, 8, 4, 256, 2432, 2, 2, false)    \
  X(false, 8, 4, 256, 512, 2, 1, true)     \
  X(false, 8, 4, 256, 2432, 2, 1, true)    \
  X(false, 8, 4, 128, 512, 4, 1, false)    \
  X(true, 8, 4, 128, 512, 4, 1, false)     \
  X(false, 8, 4, 128, 2432, 4, 1, false)   \
  X(true, 8, 4, 128, 2432, 4, 1, false)

// reads up to 512 bases use selector rows sized for 512 (less shared memory per CTA)
static int maxl_of(int32_t max_len) { return max_len <= 512 ? 512 : 2432; }

template <bool F16, int D, int RQ, int NT, int MAXL, int MINB, int STEP, bool PSSM>
static const void* scan_fn() {
  return reinterpret_cast<const void*>(&k_scan<F16, D, RQ, NT, MAXL, MINB, STEP, PSSM>);
}

static const void* pick_scan(const ScanConfig& c) {
  const int ml = maxl_of(c.max_len);
#define X(f, d, rq, nt, mx, mb, st, ps)                                                            \
  if (c.variant == (f ? 1 : 0) && c.pairs == d && c.queries == rq && c.threads == nt && ml == mx && \
      c.step == st && c.pssm == ps)                                                                \
    return scan_fn<f, d, rq, nt, mx, mb, st, ps>();
  MSS_SCAN_VARIANTS(X)
#undef X
  return nullptr;
}

bool scan_supported(const ScanConfig& c) { return pick_scan(c) != nullptr; }

int64_t scan_tile_diags(const ScanConfig& c) { return (int64_t)c.threads * 2 * c.pairs; }

size_t scan_smem_bytes(const ScanConfig& c, int32_t max_len, int32_t ring_slots) {
  const int ml = maxl_of(max_len);
#define X(f, d, rq, nt, mx, mb, st, ps)                                            \
  if (c.pairs == d && c.queries == rq && c.threads == nt && ml == mx)              \
    return scan_layout<d, rq, nt, mx>(max_len, ring_slots, c.pssm).total;
  MSS_SCAN_VARIANTS(X)
#undef X
  return 0;
}

int scan_ring_slots(const ScanConfig& c, int64_t F) {
  int64_t tile = scan_tile_diags(c);
  int64_t per_tile = (tile + F - 1) / F;
  int64_t s = 2 * per_tile + 4;
  return (int)((s + 3) & ~3);  // multiple of 4 keeps the summaries 16-byte aligned
}

cudaError_t scan_max_ctas_per_sm(const ScanConfig& c, size_t smem, int* out) {
  const void* fn = pick_scan(c);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, c.threads, smem);
}

cudaError_t launch_scan(const ScanConfig& c, const ScanArgs& a, int grid, size_t smem, cudaStream_t s) {
  const void* fn = pick_scan(c);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<ScanArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(c.threads), args, smem, s);
}

// ---------------------------------------------------------------- finalize: merge + rescan
// One warp per read: merge the chunk summaries, then rescan the best fragment on both strands
// with plain int32 arithmetic to find the best diagonal (ties: + strand first, then smallest
// d).  The rescan costs 2*F*m cells per read (1/NF of the scan).
constexpr int kFinWarps = 4;
constexpr int kFinChunk = 512;   // diagonals staged per pass (and the granularity of the early stop)

__global__ void __launch_bounds__(kFinWarps * 32) k_finalize(FinalArgs a) {
  __shared__ uint8_t s_gen[kFinWarps][kFinChunk + MSS_MAX_READ_LEN + 16];
  __shared__ uint8_t s_q[kFinWarps][2][MSS_MAX_READ_LEN];
  __shared__ uint8_t s_qual[kFinWarps][MSS_MAX_READ_LEN];  // Phred values, read order (quals only)
  __shared__ int8_t s_tab[kQualLevels][2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (a.quals)
    for (int e = threadIdx.x; e < 2 * kQualLevels; e += blockDim.x) s_tab[e >> 1][e & 1] = (int8_t)a.qtab[e];
  __syncthreads();
  const int p = blockIdx.x * kFinWarps + wib;
  if (p >= a.R) return;
  const int ridx = a.order[p];
  const int64_t off = a.offsets[ridx];
  int64_t l = a.offsets[ridx + 1] - off;
  const int32_t m = l < 0 ? 0 : (l > MSS_MAX_READ_LEN ? MSS_MAX_READ_LEN : (int32_t)l);

  Top4 t4 = top4_empty();
  for (int c = lane; c < a.n_chunks; c += 32) {
    const int4 v0 = a.partial[((size_t)p * a.n_chunks + c) * 2];
    const int4 v1 = a.partial[((size_t)p * a.n_chunks + c) * 2 + 1];
    Top4 v;
    v.s[0] = v0.x, v.f[0] = v0.y, v.s[1] = v0.z, v.f[1] = v0.w;
    v.s[2] = v1.x, v.f[2] = v1.y, v.s[3] = v1.z, v.f[3] = v1.w;
    t4 = top4_merge(t4, v);
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) t4 = top4_merge(t4, top4_shfl_xor(t4, s));
  // the best fragment and the second: the next entry, or with the neighbour rule the first
  // entry not adjacent to the best (at most two entries are adjacent, so the top-4 holds it)
  Top2 acc{t4.s[0], t4.f[0], -1, 0x7fffffff};
#pragma unroll
  for (int i = 3; i >= 1; --i) {
    const bool adjacent = t4.f[i] == t4.f[0] - 1 || t4.f[i] == t4.f[0] + 1;
    if (t4.s[i] >= 0 && !(a.exclude_neighbors && adjacent)) acc.s2 = t4.s[i], acc.f2 = t4.f[i];
  }

  for (int k = lane; k < m; k += 32) {
    uint32_t cf = ascii_code((uint8_t)a.reads[off + k]);
    if (cf > 4) cf = 4;
    s_q[wib][0][k] = (uint8_t)cf;
    s_q[wib][1][m - 1 - k] = (uint8_t)(cf < 4 ? 3 - cf : 4);
    if (a.quals) {
      int Q = (int)(uint8_t)a.quals[off + k] - 33;
      s_qual[wib][k] = (uint8_t)(Q < 0 || Q >= kQualLevels ? 0 : Q);
    }
  }
  __syncwarp();

  const int32_t f1 = acc.f1;
  int32_t bestK = -1, bestS = 0;
  int64_t bestD = 0;
  const int64_t d_lo = (int64_t)f1 * a.F, d_hi = d_lo + a.F;
  // (strand, d) in increasing order, chunk by chunk: the answer is the first pair whose score
  // is the fragment's score, so the rescan stops after the first chunk in which some lane
  // reached it (every earlier chunk scored less); without such a chunk it runs to the end and
  // the self-check below reports the mismatch
  bool found = false;
  for (int sg = 0; sg < 2 && !found; ++sg) {
    for (int64_t d0 = d_lo; d0 < d_hi && !found; d0 += kFinChunk) {
      const int64_t nd = (d_hi - d0 < (int64_t)kFinChunk) ? d_hi - d0 : (int64_t)kFinChunk;
      __syncwarp();
      for (int64_t i = lane; i < nd + m; i += 32) s_gen[wib][i] = (uint8_t)genome_code(a.g2, a.gm, d0 + i);
      __syncwarp();
      for (int64_t i = lane; i < nd; i += 32) {
        int32_t h = 0, mx = 0;
        if (a.quals) {  // position-specific scores (the reverse strand's base k is read base m-1-k)
          for (int k = 0; k < m; ++k) {
            const uint32_t qc = s_q[wib][sg][k], gc = s_gen[wib][i + k];
            const int Q = s_qual[wib][sg ? m - 1 - k : k];
            h += (qc < 4 && qc == gc) ? s_tab[Q][0] : s_tab[Q][1];
            h = max(h, 0);
            mx = max(mx, h);
          }
        } else {
          for (int k = 0; k < m; k += a.step) {
            const uint32_t qc = s_q[wib][sg][k], gc = s_gen[wib][i + k];
            h += (qc < 4 && qc == gc) ? a.match : a.mismatch;
            h = max(h, 0);
            mx = max(mx, h);
          }
        }
        if (mx > bestK) {  // lanes visit (strand, d) in increasing order
          bestK = mx;
          bestS = sg;
          bestD = d0 + i;
        }
      }
      found = __any_sync(0xffffffffu, bestK == acc.s1);
    }
  }
  // warp argmax: larger K, then smaller strand, then smaller d
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
  if (lane == 0) {
    if (bestK != acc.s1) atomicOr(a.err, ERR_SELFCHECK);
    mss_hit h;
    h.best_frag = acc.f1;
    h.best_score = acc.s1;
    h.second_frag = acc.s2 < 0 ? -1 : acc.f2;
    h.second_score = acc.s2 < 0 ? 0 : acc.s2;
    h.offset = bestD;
    h.strand = bestS;
    const bool repeat = (h.best_score == 0) || (10LL * h.second_score >= 9LL * h.best_score);
    h.flags = repeat ? MSS_HIT_REPEAT : 0;
    reinterpret_cast<mss_hit*>(a.hits)[ridx] = h;
  }
}

cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t s) {
  if (a.R <= 0) return cudaSuccess;
  const int blocks = (a.R + kFinWarps - 1) / kFinWarps;
  k_finalize<<<blocks, kFinWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mss
