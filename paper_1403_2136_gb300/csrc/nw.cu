// a6: phase two, Needleman-Wunsch of each read against the genome around its best diagonal
// ("Second phase of MaxSSmap": match 5, mismatch -4, gap -26 by default).
//
// Alignment model: glocal (the read end to end, genome ends free) with affine gaps (Gotoh),
// a gap of length k costing open + (k-1)*extend, inside the window [d-W, d+m+W) clipped to the
// genome and the band |j - i - (d - window start)| <= W around the seed diagonal d.
//
// GB300 layout: one warp per read, rows of the band processed in order; lane l holds band
// cells 4l..4l+3.  The diagonal and vertical terms come from the previous row (own registers
// and one shuffle); the horizontal gap term E is a max-plus prefix over the row,
// E(b) = open - ext + b*ext + max_{b'<b}(H'(b') - b'*ext), which equals the Gotoh recurrence
// whenever open <= ext (a warp shuffle scan).  One direction byte per cell goes to a per-warp
// scratch area and a single lane walks the traceback.
#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"

namespace mss {

constexpr int kNwWarps = 4;
constexpr int kNwCells = 4;                 // band cells per lane
constexpr int kNwRow = 32 * kNwCells;       // bytes per traceback row
constexpr int32_t kNeg = -(1 << 29);        // "minus infinity" (finite scores stay far above kNeg/2)

__device__ __forceinline__ int32_t clampneg(int32_t x) { return x < kNeg / 2 ? kNeg : x; }

// Per-warp scratch: (max_len + 1) direction rows of 128 bytes, then the traceback ops
// (at most m + window length <= 2m + 2W).  Rounded to 128 bytes so that every warp's rows stay
// aligned for the 4-byte stores.
int64_t nw_scratch_per_warp(int32_t max_len, int32_t band) {
  const int64_t bytes = (int64_t)(max_len + 1) * kNwRow + 2 * (int64_t)max_len + 2 * (int64_t)band + 64;
  return (bytes + 127) / 128 * 128;
}

__global__ void __launch_bounds__(kNwWarps * 32) k_nw(NwArgs a) {
  __shared__ uint8_t s_q[kNwWarps][MSS_MAX_READ_LEN];
  __shared__ uint8_t s_w[kNwWarps][MSS_MAX_READ_LEN + 2 * 64 + 16];
  __shared__ uint8_t s_qual[kNwWarps][MSS_MAX_READ_LEN];  // Phred values in strand order (quals only)
  __shared__ int16_t s_tab[kQualLevels][2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (a.quals)
    for (int e = threadIdx.x; e < 2 * kQualLevels; e += blockDim.x) s_tab[e >> 1][e & 1] = a.qtab[e];
  __syncthreads();
  const int gw = blockIdx.x * kNwWarps + wib;
  if (gw >= a.n_warps) return;
  uint8_t* tb = a.scratch + (int64_t)gw * a.scratch_per_warp;
  char* opsbuf = reinterpret_cast<char*>(tb + (int64_t)(a.max_len + 1) * kNwRow);
  const int32_t W = a.band, B = 2 * a.band;  // band cells b = 0..B
  const int32_t go = a.gap_open, ge = a.gap_extend;

  for (int r = gw; r < a.R; r += a.n_warps) {
    const mss_hit hit = reinterpret_cast<const mss_hit*>(a.hits)[r];
    const int64_t off = a.offsets[r];
    int64_t l = a.offsets[r + 1] - off;
    const int32_t m = l < 1 ? 0 : (l > a.max_len ? a.max_len : (int32_t)l);
    mss_aln out;
    out.score = MSS_NW_NONE;
    out.cigar_len = 0;
    const int64_t d = hit.offset;
    int64_t ws = d - W;
    if (ws < 0) ws = 0;
    int64_t we = d + m + W;
    if (we > a.G) we = a.G;
    const int32_t L = (int32_t)(we > ws ? we - ws : 0);
    const int32_t offc = (int32_t)(d - ws);
    out.gstart = out.gend = ws;

    __syncwarp();
    for (int k = lane; k < m; k += 32) {
      uint32_t cf;
      if (hit.strand) {
        cf = ascii_code((uint8_t)a.reads[off + m - 1 - k]);
        cf = cf < 4 ? 3 - cf : 4;
      } else {
        cf = ascii_code((uint8_t)a.reads[off + k]);
        if (cf > 4) cf = 4;
      }
      s_q[wib][k] = (uint8_t)cf;
      if (a.quals) {
        int Q = (int)(uint8_t)a.quals[off + (hit.strand ? m - 1 - k : k)] - 33;
        if (Q < 0 || Q >= kQualLevels) {
          atomicOr(a.err, ERR_BAD_QUAL);
          Q = 0;
        }
        s_qual[wib][k] = (uint8_t)Q;
      }
    }
    for (int j = lane; j < L; j += 32) s_w[wib][j] = (uint8_t)genome_code(a.g2, a.gm, ws + j);
    __syncwarp();

    // row 0: H = 0 on in-band columns 0..L (leading genome bases are free)
    int32_t Hp[kNwCells], Fp[kNwCells];
#pragma unroll
    for (int c = 0; c < kNwCells; ++c) {
      const int32_t b = kNwCells * lane + c;
      const int32_t j = offc - W + b;
      const bool valid = (b <= B) && j >= 0 && j <= L;
      Hp[c] = valid ? 0 : kNeg;
      Fp[c] = kNeg;
    }
    for (int32_t i = 1; i <= m; ++i) {
      const uint32_t qc = s_q[wib][i - 1];
      int32_t row_match = a.match, row_mismatch = a.mismatch;
      if (a.quals) {  // position-specific scores of this read base
        const int Q = s_qual[wib][i - 1];
        row_match = s_tab[Q][0];
        row_mismatch = s_tab[Q][1];
      }
      const int32_t Hn = __shfl_down_sync(0xffffffffu, Hp[0], 1);
      const int32_t Fn = __shfl_down_sync(0xffffffffu, Fp[0], 1);
      int32_t Hd[kNwCells], Fc[kNwCells], Dg[kNwCells], Hup[kNwCells];
      bool valid[kNwCells];
#pragma unroll
      for (int c = 0; c < kNwCells; ++c) {
        const int32_t b = kNwCells * lane + c;
        const int32_t j = i + offc - W + b;
        valid[c] = (b <= B) && j >= 0 && j <= L;
        const int32_t hu = (c + 1 < kNwCells) ? Hp[c + 1] : (lane < 31 ? Hn : kNeg);
        const int32_t fu = (c + 1 < kNwCells) ? Fp[c + 1] : (lane < 31 ? Fn : kNeg);
        int32_t dg = kNeg;
        if (valid[c] && j >= 1 && Hp[c] > kNeg / 2) {
          const uint32_t gc = s_w[wib][j - 1];
          dg = Hp[c] + ((qc < 4 && qc == gc) ? row_match : row_mismatch);
        }
        const int32_t f = clampneg(max(hu + go, fu + ge));
        Hup[c] = hu;
        Dg[c] = dg;
        Fc[c] = valid[c] ? f : kNeg;
        Hd[c] = valid[c] ? max(dg, Fc[c]) : kNeg;
      }
      // E: exclusive max-plus prefix of Y(b) = H'(b) - b*ext along the row
      int32_t Y[kNwCells];
      int32_t lmax = kNeg;
#pragma unroll
      for (int c = 0; c < kNwCells; ++c) {
        const int32_t b = kNwCells * lane + c;
        Y[c] = Hd[c] > kNeg / 2 ? Hd[c] - b * ge : kNeg;
        lmax = max(lmax, Y[c]);
      }
      int32_t incl = lmax;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= s) incl = max(incl, o);
      }
      int32_t run = __shfl_up_sync(0xffffffffu, incl, 1);
      if (lane == 0) run = kNeg;
      int32_t Hc[kNwCells], Ec[kNwCells];
#pragma unroll
      for (int c = 0; c < kNwCells; ++c) {
        const int32_t b = kNwCells * lane + c;
        const int32_t e = run > kNeg / 2 ? go - ge + b * ge + run : kNeg;
        Ec[c] = valid[c] ? clampneg(e) : kNeg;
        Hc[c] = valid[c] ? max(Hd[c], Ec[c]) : kNeg;
        run = max(run, Y[c]);
      }
      // direction bytes: bits 0-1 source of H (0 diagonal, 1 E, 2 F), bit 2 E opened from H,
      // bit 3 F opened from H
      const int32_t Hl = __shfl_up_sync(0xffffffffu, Hc[kNwCells - 1], 1);
      uint32_t packed = 0;
#pragma unroll
      for (int c = 0; c < kNwCells; ++c) {
        const int32_t hleft = (c > 0) ? Hc[c - 1] : (lane > 0 ? Hl : kNeg);
        uint32_t src = (Dg[c] > kNeg / 2 && Hc[c] == Dg[c]) ? 0u : (Hc[c] == Ec[c] ? 1u : 2u);
        const uint32_t eo = (Ec[c] > kNeg / 2 && Ec[c] == hleft + go) ? 4u : 0u;
        const uint32_t fo = (Fc[c] > kNeg / 2 && Fc[c] == Hup[c] + go) ? 8u : 0u;
        packed |= (src | eo | fo) << (8 * c);
      }
      reinterpret_cast<uint32_t*>(tb + (int64_t)i * kNwRow)[lane] = packed;
#pragma unroll
      for (int c = 0; c < kNwCells; ++c) {
        Hp[c] = Hc[c];
        Fp[c] = Fc[c];
      }
    }
    // best end cell of the last row: highest score, then smallest column (= smallest b)
    int32_t bv = kNeg, bb = 0x7fffffff;
#pragma unroll
    for (int c = 0; c < kNwCells; ++c) {
      const int32_t b = kNwCells * lane + c;
      if (m > 0 && Hp[c] > kNeg / 2 && (Hp[c] > bv)) {
        bv = Hp[c];
        bb = b;
      }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const int32_t ov = __shfl_xor_sync(0xffffffffu, bv, s);
      const int32_t ob = __shfl_xor_sync(0xffffffffu, bb, s);
      if (ov > bv || (ov == bv && ob < bb)) {
        bv = ov;
        bb = ob;
      }
    }
    __syncwarp();
    if (lane == 0) {
      char* cig = a.cigars + (int64_t)r * a.cigar_stride;
      if (bv > kNeg / 2) {
        out.score = bv;
        int32_t i = m, b = bb, state = 0, nops = 0;
        const int32_t jend = m + offc - W + bb;
        while (i > 0) {
          const uint32_t dir = tb[(int64_t)i * kNwRow + b];
          if (state == 0) {
            const uint32_t src = dir & 3u;
            if (src == 0) {
              opsbuf[nops++] = 'M';
              --i;
            } else {
              state = (int)src;
            }
          } else if (state == 1) {
            opsbuf[nops++] = 'D';
            state = (dir & 4u) ? 0 : 1;
            --b;
          } else {
            opsbuf[nops++] = 'I';
            state = (dir & 8u) ? 0 : 2;
            --i;
            ++b;
          }
        }
        const int32_t jstart = offc - W + b;
        out.gstart = ws + jstart;
        out.gend = ws + jend;
        // run-length encode in forward order
        int32_t len = 0;
        bool overflow = false;
        int32_t k = nops - 1;
        while (k >= 0) {
          const char op = opsbuf[k];
          int32_t run = 0;
          while (k >= 0 && opsbuf[k] == op) {
            ++run;
            --k;
          }
          char tmp[12];
          int t = 0;
          do {
            tmp[t++] = (char)('0' + run % 10);
            run /= 10;
          } while (run > 0);
          if (len + t + 1 >= a.cigar_stride) {
            overflow = true;
            break;
          }
          while (t > 0) cig[len++] = tmp[--t];
          cig[len++] = op;
        }
        if (overflow) {
          out.cigar_len = -1;
          if (a.cigar_stride > 0) cig[0] = 0;
        } else {
          out.cigar_len = len;
          cig[len] = 0;
        }
      } else if (a.cigar_stride > 0) {
        cig[0] = 0;
      }
      reinterpret_cast<mss_aln*>(a.alns)[r] = out;
    }
    __syncwarp();
  }
}

cudaError_t launch_nw(const NwArgs& a, int grid_warps, cudaStream_t s) {
  if (a.R <= 0) return cudaSuccess;
  const int blocks = (grid_warps + kNwWarps - 1) / kNwWarps;
  k_nw<<<blocks, kNwWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mss
