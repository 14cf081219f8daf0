/*
 * CPU oracle for the MaxSSmap hot path — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded statement of what the mapping computes, written from the
 * paper (Turki & Roshan, "MaxSSmap", arXiv 1403.2136).  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * Sections followed:
 *   - "Maximum scoring subsequence" (Methods/Background): the maximum-sum contiguous run of
 *     substitution scores, empty run allowed (so the score is >= 0), found in linear time by
 *     the Bentley / Bates-Constable scan.
 *   - "First phase of MaxSSmap": the read slides over every fixed-size fragment, with the
 *     window allowed to run into the next fragment (junctions); best and second fragment;
 *     mapped iff second/best < 0.9.
 *   - "Coalescent global memory access": fragment f = genome bases [fF, fF+F), the genome
 *     padded with N up to a multiple of F (Figure 2 toy genome).
 *   - "Second phase of MaxSSmap": Needleman-Wunsch of the read against the region found in
 *     phase one, match 5, mismatch -4, gap -26 by default.
 *
 * Readings where the paper is silent:
 *   - both strands are scanned; the reverse strand is the reverse complement of the read;
 *   - only diagonals d in [0, Gp) exist (no left overhang);
 *   - per-fragment argmax tie: strand + before -, then smallest d;
 *   - best fragment ties -> lowest index; second = best among the other fragments, ties ->
 *     lowest index; with a single fragment, second = -1 and its score 0;
 *   - repeat flag iff best == 0 or 10*second >= 9*best (the exact integer form of >= 0.9);
 *   - phase two is glocal (read end to end, genome ends free) affine-gap (Gotoh) alignment
 *     in the window [d-W, d+m+W) clipped to the genome, restricted to the band
 *     |j - i - (d - window start)| <= W; linear gap -26 is open = extend = -26.
 *
 * Parity pins (tests/test_oracle_*.py): brute-force enumeration of all substrings on tiny
 * inputs, exact-substring and all-mismatch invariants, reverse-complement symmetry, the
 * Figure 2 toy layout, planted repeats, closed forms printed in the paper, hand-worked and
 * brute-force-enumerated alignments.
 */
#ifndef MSS_ORACLE_H
#define MSS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 'A','C','G','T' (either case) -> 0..3, 'N'/'n' -> 4, anything else -> -1 */
int orc_base_code(int c);

/* maximum scoring subsequence of x[0..n), empty run allowed (Bentley / Bates-Constable) */
int64_t orc_mss(const int32_t* x, int64_t n);

/* maximum scoring subsequence along one diagonal: read codes q[0..m) against padded genome
   codes g[d .. d+m) (codes 0..3 bases, 4 = N); s = match iff q[k]==g[d+k] and both < 4 */
int32_t orc_diag_score(const uint8_t* q, int32_t m, const uint8_t* g, int64_t d, int32_t match, int32_t mismatch);

/* the same with the read sampled at positions 0, step, 2 step, ... ("MaxSSmap_fast" considers
   every other nucleotide of the read: step 2); step 1 is orc_diag_score */
int32_t orc_diag_score_step(const uint8_t* q, int32_t m, const uint8_t* g, int64_t d, int32_t match,
                            int32_t mismatch, int32_t step);

typedef struct {
  int32_t best_frag;
  int32_t second_frag;
  int32_t best_score;
  int32_t second_score;
  int64_t offset;     /* best diagonal d of the best fragment (genome index of read base 0) */
  int32_t strand;     /* 0 = read as given, 1 = reverse complement */
  int32_t flags;      /* bit 0: repeat / unmapped (best == 0 or 10*second >= 9*best) */
} orc_hit;

/*
 * Phase one for one read: every diagonal d in [0, Gp) of both strands, fragment maxima,
 * top-2.  genome: ASCII (len G), read: ASCII (len m).  frag_scores (optional, NF entries)
 * receives S(f).  Returns 0, or -1 for an invalid character / size.
 */
int orc_map_read(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                 int32_t mismatch, orc_hit* out, int32_t* frag_scores);

/* phase one whose second fragment is the best one not adjacent to the best (|f - best| > 1);
   second = -1 (score 0) when no such fragment exists */
int orc_map_read_excl(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                      int32_t mismatch, orc_hit* out, int32_t* frag_scores);

/* phase one with the read sampled every step bases (1 or 2; 2 = "MaxSSmap_fast"), on both
   strands (the reverse strand is sampled after reverse complementing) */
int orc_map_read_step(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                      int32_t mismatch, int32_t step, orc_hit* out, int32_t* frag_scores);

/* Base qualities ("Incorporating base qualities and position specific scoring matrix"):
   x = 1 - 10^(-Q/10) for Phred+33 quality character qual_char; *ma = match * x * scale and
   *mm = mismatch * x / 3 * scale, rounded to the nearest integer (halves away from zero).
   Returns -1 for a character outside '!'..'~' or scale < 1. */
int orc_pssm_scores(int32_t qual_char, int32_t match, int32_t mismatch, int32_t scale, int32_t* ma, int32_t* mm);

/* phase one with those position-specific scores (read base k of the reverse complement takes
   the quality of read base m - 1 - k); N never matches and scores the position's mismatch */
int orc_map_read_pssm(const char* genome, int64_t G, int64_t F, const char* read, const char* quals, int32_t m,
                      int32_t match, int32_t mismatch, int32_t scale, orc_hit* out, int32_t* frag_scores);

/* reverse complement of codes (4 stays 4) */
void orc_revcomp(const uint8_t* q, int32_t m, uint8_t* out);

typedef struct {
  int32_t score;       /* alignment score, or ORC_NW_NONE when no in-band alignment exists */
  int32_t cigar_len;   /* characters written to cigar (NUL not counted) */
  int64_t gstart;      /* genome index of the first aligned genome base */
  int64_t gend;        /* one past the last aligned genome base */
} orc_aln;

#define ORC_NW_NONE (-2147483647 - 1)

/*
 * Phase two (primary reading): glocal affine-gap alignment of q (codes, already on the
 * chosen strand) in the window [d-W, d+m+W) clipped to [0, G), banded |j-i-off| <= W.
 * Gap of length k costs open + (k-1)*extend.  Traceback ties: diagonal, then gap in read
 * (D), then gap in genome (I); a gap is closed (opened from H) in preference to extended;
 * among equal end scores the smallest end column.  cigar receives "<n><op>..." (op in M,I,D),
 * at most cigar_cap-1 characters plus NUL.  Returns 0 or -1 (bad arguments / cap too small).
 */
int orc_nw_banded(const uint8_t* gcodes, int64_t G, const uint8_t* q, int32_t m, int64_t d, int32_t W,
                  int32_t match, int32_t mismatch, int32_t gap_open, int32_t gap_extend, orc_aln* out,
                  char* cigar, int32_t cigar_cap);

/*
 * Phase two, literal variant of the paper's wording: the region starts at the best
 * fragment's first base and spans ceil(m/F) fragments to the right (clipped to G); unbanded
 * glocal alignment with the same scoring and tie rules.
 */
int orc_nw_literal(const uint8_t* gcodes, int64_t G, int64_t F, int32_t best_frag, const uint8_t* q, int32_t m,
                   int32_t match, int32_t mismatch, int32_t gap_open, int32_t gap_extend, orc_aln* out,
                   char* cigar, int32_t cigar_cap);

/* ASCII genome -> codes (0..4); returns -1 on an invalid character */
int orc_encode(const char* s, int64_t n, uint8_t* out);

/* Map a batch of reads (concatenated ASCII, offsets[R+1]) and align each with the banded
   reading: convenience loop over orc_map_read + orc_nw_banded for the tests and the CPU
   baseline.  cigars: R slots of cigar_cap bytes.  Returns 0 or the first error. */
int orc_map_batch(const char* genome, int64_t G, int64_t F, const char* reads, const int64_t* offsets, int32_t R,
                  int32_t match, int32_t mismatch, int32_t nw_match, int32_t nw_mismatch, int32_t gap_open,
                  int32_t gap_extend, int32_t W, orc_hit* hits, orc_aln* alns, char* cigars, int32_t cigar_cap);
int orc_nw_banded_pssm(const uint8_t* gcodes, int64_t G, const uint8_t* q, const int32_t* ma, const int32_t* mm,
                       int32_t m, int64_t d, int32_t W, int32_t gap_open, int32_t gap_extend, orc_aln* out,
                       char* cigar, int32_t cigar_cap);
int orc_map_batch_pssm(const char* genome, int64_t G, int64_t F, const char* reads, const char* quals,
                       const int64_t* offsets, int32_t R, int32_t match, int32_t mismatch, int32_t scale,
                       int32_t nw_match, int32_t nw_mismatch, int32_t gap_open, int32_t gap_extend, int32_t W,
                       orc_hit* hits, orc_aln* alns, char* cigars, int32_t cigar_cap);
int orc_map_batch_step(const char* genome, int64_t G, int64_t F, const char* reads, const int64_t* offsets,
                       int32_t R, int32_t match, int32_t mismatch, int32_t step, int32_t nw_match,
                       int32_t nw_mismatch, int32_t gap_open, int32_t gap_extend, int32_t W, orc_hit* hits,
                       orc_aln* alns, char* cigars, int32_t cigar_cap);

#ifdef __cplusplus
}
#endif
#endif
