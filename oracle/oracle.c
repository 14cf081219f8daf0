/*
 * CPU oracle for the MaxSSmap hot path — TEST INFRASTRUCTURE ONLY (see oracle.h for the
 * sections of the paper it follows and the readings it takes).  Plain loops, no blocking,
 * no fusion, no reordering; int64 arithmetic throughout.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int orc_base_code(int c) {
  switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    case 'N': case 'n': return 4;
    default: return -1;
  }
}

int orc_encode(const char* s, int64_t n, uint8_t* out) {
  for (int64_t i = 0; i < n; ++i) {
    int c = orc_base_code((unsigned char)s[i]);
    if (c < 0) return -1;
    out[i] = (uint8_t)c;
  }
  return 0;
}

void orc_revcomp(const uint8_t* q, int32_t m, uint8_t* out) {
  for (int32_t k = 0; k < m; ++k) {
    uint8_t c = q[m - 1 - k];
    out[k] = (uint8_t)(c < 4 ? 3 - c : 4);
  }
}

/* Maximum scoring subsequence ("Maximum scoring subsequence", Methods): the best sum of a
   contiguous run x_i..x_j, where the empty run (sum 0) is allowed.  Linear scan: the best
   run ending at position k is max(best ending at k-1, 0) + x_k; the answer is the largest
   of those and 0. */
int64_t orc_mss(const int32_t* x, int64_t n) {
  int64_t ending_here = 0; /* best sum of a run ending at the current position, or 0 (empty) */
  int64_t best = 0;
  for (int64_t k = 0; k < n; ++k) {
    ending_here = ending_here + x[k];
    if (ending_here < 0) ending_here = 0;
    if (ending_here > best) best = ending_here;
  }
  return best;
}

/* substitution scores of the read against the genome window that starts at diagonal d, at
   read positions 0, step, 2 step, ... (step 1: every base; step 2: "MaxSSmap_fast", every other
   nucleotide of the read); returns how many scores were written */
static int32_t diag_scores_pos(const uint8_t* q, int32_t m, const uint8_t* g, int64_t d, int32_t match,
                               int32_t mismatch, int32_t step, const int32_t* ma, const int32_t* mm, int32_t* x) {
  int32_t n = 0;
  for (int32_t k = 0; k < m; k += step) {
    uint8_t a = q[k], b = g[d + k];
    int32_t sm = ma ? ma[k] : match, sx = mm ? mm[k] : mismatch; /* position-specific when given */
    x[n++] = (a < 4 && a == b) ? sm : sx;
  }
  return n;
}

static int32_t diag_scores(const uint8_t* q, int32_t m, const uint8_t* g, int64_t d, int32_t match,
                           int32_t mismatch, int32_t step, int32_t* x) {
  return diag_scores_pos(q, m, g, d, match, mismatch, step, 0, 0, x);
}

/* One ungapped read-vs-genome diagonal ("First phase of MaxSSmap"): the substitution score
   sequence of the read against the genome window starting at d, then its maximum scoring
   subsequence. */
int32_t orc_diag_score_step(const uint8_t* q, int32_t m, const uint8_t* g, int64_t d, int32_t match,
                            int32_t mismatch, int32_t step) {
  int32_t* x = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t n = diag_scores(q, m, g, d, match, mismatch, step, x);
  int64_t v = orc_mss(x, n);
  free(x);
  return (int32_t)v;
}

int32_t orc_diag_score(const uint8_t* q, int32_t m, const uint8_t* g, int64_t d, int32_t match, int32_t mismatch) {
  return orc_diag_score_step(q, m, g, d, match, mismatch, 1);
}

int orc_map_read(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                 int32_t mismatch, orc_hit* out, int32_t* frag_scores) {
  return orc_map_read_step(genome, G, F, read, m, match, mismatch, 1, out, frag_scores);
}

static int map_read_impl(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                         int32_t mismatch, int32_t step, const int32_t* const* ma, const int32_t* const* mm,
                         int32_t exclude_neighbors, orc_hit* out, int32_t* frag_scores);

int orc_map_read_step(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                      int32_t mismatch, int32_t step, orc_hit* out, int32_t* frag_scores) {
  return map_read_impl(genome, G, F, read, m, match, mismatch, step, 0, 0, 0, out, frag_scores);
}

/* Top-2 with the neighbours of the best fragment excluded (the paper does not say whether the
   fragment next to the best may count as the second; this is the alternative reading): the
   second is the best fragment f with |f - best| > 1. */
int orc_map_read_excl(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                      int32_t mismatch, orc_hit* out, int32_t* frag_scores) {
  return map_read_impl(genome, G, F, read, m, match, mismatch, 1, 0, 0, 1, out, frag_scores);
}

/* "Incorporating base qualities and position specific scoring matrix": a base of Phred
   quality Q is right with probability x = 1 - 10^(-Q/10); a match against it scores
   match * x and a mismatch mismatch * x / 3.  Fixed point: both times scale, rounded to the
   nearest integer with halves away from zero. */
static int32_t round_half_away(double v) { return (int32_t)(v < 0 ? -floor(-v + 0.5) : floor(v + 0.5)); }

int orc_pssm_scores(int32_t qual_char, int32_t match, int32_t mismatch, int32_t scale, int32_t* ma, int32_t* mm) {
  int32_t Q = qual_char - 33; /* Phred+33 */
  if (Q < 0 || Q > 93 || scale < 1) return -1;
  double x = 1.0 - pow(10.0, -Q / 10.0);
  *ma = round_half_away((double)scale * match * x);
  *mm = round_half_away((double)scale * mismatch * x / 3.0);
  return 0;
}

int orc_map_read_pssm(const char* genome, int64_t G, int64_t F, const char* read, const char* quals, int32_t m,
                      int32_t match, int32_t mismatch, int32_t scale, orc_hit* out, int32_t* frag_scores) {
  if (m <= 0 || !quals) return -1;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)m);
  if (!buf) return -2;
  int32_t *maf = buf, *mmf = buf + m, *mar = buf + 2 * m, *mmr = buf + 3 * m;
  for (int32_t k = 0; k < m; ++k) {
    if (orc_pssm_scores((unsigned char)quals[k], match, mismatch, scale, &maf[k], &mmf[k]) != 0) {
      free(buf);
      return -1;
    }
  }
  for (int32_t k = 0; k < m; ++k) { /* the reverse complement's base k is read base m - 1 - k */
    mar[k] = maf[m - 1 - k];
    mmr[k] = mmf[m - 1 - k];
  }
  const int32_t* ma[2] = {maf, mar};
  const int32_t* mm[2] = {mmf, mmr};
  int rc = map_read_impl(genome, G, F, read, m, match, mismatch, 1, ma, mm, 0, out, frag_scores);
  free(buf);
  return rc;
}

static int map_read_impl(const char* genome, int64_t G, int64_t F, const char* read, int32_t m, int32_t match,
                         int32_t mismatch, int32_t step, const int32_t* const* ma, const int32_t* const* mm,
                         int32_t exclude_neighbors, orc_hit* out, int32_t* frag_scores) {
  if (G <= 0 || F <= 0 || m <= 0 || !out || (step != 1 && step != 2)) return -1;
  int64_t NF = (G + F - 1) / F;
  int64_t Gp = NF * F;
  /* genome codes, padded with N up to Gp + m - 1 ("Coalescent global memory access": the last
     fragment is padded with N; the junction window of the last diagonals runs past it) */
  int64_t glen = Gp + m;
  uint8_t* g = (uint8_t*)malloc((size_t)glen);
  uint8_t* q[2];
  q[0] = (uint8_t*)malloc((size_t)m);
  q[1] = (uint8_t*)malloc((size_t)m);
  int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)NF);
  int64_t* arg_d = (int64_t*)malloc(sizeof(int64_t) * (size_t)NF);
  int32_t* arg_s = (int32_t*)malloc(sizeof(int32_t) * (size_t)NF);
  int32_t* x = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int rc = 0;
  if (!g || !q[0] || !q[1] || !S || !arg_d || !arg_s || !x) { rc = -2; goto done; }
  if (orc_encode(genome, G, g) != 0) { rc = -1; goto done; }
  for (int64_t i = G; i < glen; ++i) g[i] = 4;
  if (orc_encode(read, m, q[0]) != 0) { rc = -1; goto done; }
  orc_revcomp(q[0], m, q[1]);

  for (int64_t f = 0; f < NF; ++f) { S[f] = -1; arg_d[f] = -1; arg_s[f] = -1; }
  /* every strand, every diagonal; fragment f owns diagonals [fF, (f+1)F) and reads genome
     bases up to (f+1)F + m - 1 (the junction into the right neighbour) */
  for (int32_t sg = 0; sg < 2; ++sg) {
    for (int64_t d = 0; d < Gp; ++d) {
      int32_t n = diag_scores_pos(q[sg], m, g, d, match, mismatch, step, ma ? ma[sg] : 0, mm ? mm[sg] : 0, x);
      int32_t K = (int32_t)orc_mss(x, n);
      int64_t f = d / F;
      if (K > S[f]) { /* strictly greater: + strand before -, then the smallest d */
        S[f] = K;
        arg_d[f] = d;
        arg_s[f] = sg;
      }
    }
  }
  /* top two fragments: ties go to the lowest index */
  int64_t b1 = 0;
  for (int64_t f = 1; f < NF; ++f)
    if (S[f] > S[b1]) b1 = f;
  int64_t b2 = -1;
  for (int64_t f = 0; f < NF; ++f) {
    if (f == b1) continue;
    if (exclude_neighbors && (f == b1 - 1 || f == b1 + 1)) continue;
    if (b2 < 0 || S[f] > S[b2]) b2 = f;
  }
  out->best_frag = (int32_t)b1;
  out->best_score = S[b1];
  out->second_frag = (int32_t)b2;
  out->second_score = b2 >= 0 ? S[b2] : 0;
  out->offset = arg_d[b1];
  out->strand = arg_s[b1];
  /* "mapped if the ratio of the second best to best score is below .9" */
  int repeat = (out->best_score == 0) || ((int64_t)10 * out->second_score >= (int64_t)9 * out->best_score);
  out->flags = repeat ? 1 : 0;
  if (frag_scores)
    for (int64_t f = 0; f < NF; ++f) frag_scores[f] = S[f];
done:
  free(g); free(q[0]); free(q[1]); free(S); free(arg_d); free(arg_s); free(x);
  return rc;
}

/* ------------------------------------------------------------------------------------------
 * Phase two: Needleman-Wunsch ("Second phase of MaxSSmap") with affine gaps (Gotoh).
 * H = best score of an alignment of q[0..i) ending at window column j in any state,
 * E = ... ending with a gap in the read (genome base against '-', CIGAR D),
 * F = ... ending with a gap in the genome (read base against '-', CIGAR I).
 * ------------------------------------------------------------------------------------------ */
#define NEG_INF (INT64_MIN / 4)

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

static int in_band(int64_t i, int64_t j, int64_t off, int64_t W) {
  if (W < 0) return 1; /* unbanded */
  int64_t t = j - i - off;
  return t >= -W && t <= W;
}

static int append_run(char* cigar, int32_t cap, int32_t* len, int32_t n, char op) {
  char tmp[16];
  int t = 0;
  int32_t v = n;
  do { tmp[t++] = (char)('0' + v % 10); v /= 10; } while (v > 0);
  if (*len + t + 1 >= cap) return -1;
  while (t > 0) cigar[(*len)++] = tmp[--t];
  cigar[(*len)++] = op;
  cigar[*len] = 0;
  return 0;
}

/* w: window codes [0..L), q: read codes [0..m), off: window column of read base 0 on the
   seed diagonal, W < 0: unbanded. */
static int nw_core(const uint8_t* w, int64_t L, const uint8_t* q, int32_t m, int64_t off, int64_t W, int32_t match,
                   int32_t mismatch, const int32_t* ma, const int32_t* mm, int32_t gap_open, int32_t gap_extend,
                   int64_t wstart, orc_aln* out, char* cigar, int32_t cigar_cap) {
  int64_t cols = L + 1;
  int64_t cells = (int64_t)(m + 1) * cols;
  int64_t* H = (int64_t*)malloc(sizeof(int64_t) * (size_t)cells);
  int64_t* E = (int64_t*)malloc(sizeof(int64_t) * (size_t)cells);
  int64_t* Fm = (int64_t*)malloc(sizeof(int64_t) * (size_t)cells);
  char* ops = (char*)malloc((size_t)(m + L + 2));
  if (!H || !E || !Fm || !ops) { free(H); free(E); free(Fm); free(ops); return -2; }
#define AT(A, i, j) A[(int64_t)(i) * cols + (j)]
  for (int64_t j = 0; j <= L; ++j) {
    AT(H, 0, j) = in_band(0, j, off, W) ? 0 : NEG_INF; /* leading genome bases are free */
    AT(E, 0, j) = NEG_INF;
    AT(Fm, 0, j) = NEG_INF;
  }
  for (int64_t i = 1; i <= m; ++i) {
    for (int64_t j = 0; j <= L; ++j) {
      if (!in_band(i, j, off, W)) {
        AT(H, i, j) = AT(E, i, j) = AT(Fm, i, j) = NEG_INF;
        continue;
      }
      int64_t diag = NEG_INF, e = NEG_INF, f;
      if (j >= 1) {
        uint8_t a = q[i - 1], b = w[j - 1];
        int32_t s = (a < 4 && a == b) ? (ma ? ma[i - 1] : match) : (mm ? mm[i - 1] : mismatch);
        if (AT(H, i - 1, j - 1) > NEG_INF / 2) diag = AT(H, i - 1, j - 1) + s;
        e = max2(AT(H, i, j - 1) + gap_open, AT(E, i, j - 1) + gap_extend);
      }
      f = max2(AT(H, i - 1, j) + gap_open, AT(Fm, i - 1, j) + gap_extend);
      if (e < NEG_INF / 2) e = NEG_INF;
      if (f < NEG_INF / 2) f = NEG_INF;
      AT(E, i, j) = e;
      AT(Fm, i, j) = f;
      AT(H, i, j) = max2(diag, max2(e, f));
    }
  }
  /* read end to end, genome end free: best cell of the last row, smallest column on ties */
  int64_t jbest = -1;
  for (int64_t j = 0; j <= L; ++j) {
    if (AT(H, m, j) <= NEG_INF / 2) continue;
    if (jbest < 0 || AT(H, m, j) > AT(H, m, jbest)) jbest = j;
  }
  out->cigar_len = 0;
  if (cigar && cigar_cap > 0) cigar[0] = 0;
  if (jbest < 0) {
    out->score = ORC_NW_NONE;
    out->gstart = out->gend = wstart;
    free(H); free(E); free(Fm); free(ops);
    return 0;
  }
  out->score = (int32_t)AT(H, m, jbest);
  /* traceback: state 0 = H, 1 = E (D), 2 = F (I) */
  int64_t i = m, j = jbest;
  int state = 0;
  int64_t nops = 0;
  while (i > 0) {
    if (state == 0) {
      int64_t h = AT(H, i, j);
      if (j >= 1 && AT(H, i - 1, j - 1) > NEG_INF / 2) {
        uint8_t a = q[i - 1], b = w[j - 1];
        int32_t s = (a < 4 && a == b) ? (ma ? ma[i - 1] : match) : (mm ? mm[i - 1] : mismatch);
        if (h == AT(H, i - 1, j - 1) + s) {
          ops[nops++] = 'M';
          --i; --j;
          continue;
        }
      }
      if (h == AT(E, i, j)) { state = 1; continue; }
      state = 2; /* h == F */
      continue;
    } else if (state == 1) {
      ops[nops++] = 'D';
      int64_t e = AT(E, i, j);
      state = (e == AT(H, i, j - 1) + gap_open) ? 0 : 1;
      --j;
    } else {
      ops[nops++] = 'I';
      int64_t f = AT(Fm, i, j);
      state = (f == AT(H, i - 1, j) + gap_open) ? 0 : 2;
      --i;
    }
  }
  out->gstart = wstart + j;
  out->gend = wstart + jbest;
  /* run-length encode in forward order */
  int32_t len = 0;
  int rc = 0;
  if (cigar && cigar_cap > 0) {
    int64_t k = nops - 1;
    while (k >= 0) {
      char op = ops[k];
      int32_t run = 0;
      while (k >= 0 && ops[k] == op) { ++run; --k; }
      if (append_run(cigar, cigar_cap, &len, run, op) != 0) { rc = -1; break; }
    }
  }
  out->cigar_len = len;
#undef AT
  free(H); free(E); free(Fm); free(ops);
  return rc;
}

int orc_nw_banded(const uint8_t* gcodes, int64_t G, const uint8_t* q, int32_t m, int64_t d, int32_t W,
                  int32_t match, int32_t mismatch, int32_t gap_open, int32_t gap_extend, orc_aln* out,
                  char* cigar, int32_t cigar_cap) {
  if (G <= 0 || m <= 0 || W < 0 || d < 0 || !out) return -1;
  int64_t ws = d - W;
  if (ws < 0) ws = 0;
  int64_t we = d + m + W;
  if (we > G) we = G;
  int64_t L = we - ws;
  if (L < 0) L = 0;
  int64_t off = d - ws;
  return nw_core(gcodes + ws, L, q, m, off, W, match, mismatch, 0, 0, gap_open, gap_extend, ws, out, cigar,
                 cigar_cap);
}

/* the banded reading with position-specific match / mismatch scores of the read bases
   (ma[i], mm[i] for read base i; gaps as given, already in the same fixed point) */
int orc_nw_banded_pssm(const uint8_t* gcodes, int64_t G, const uint8_t* q, const int32_t* ma, const int32_t* mm,
                       int32_t m, int64_t d, int32_t W, int32_t gap_open, int32_t gap_extend, orc_aln* out,
                       char* cigar, int32_t cigar_cap) {
  if (G <= 0 || m <= 0 || W < 0 || d < 0 || !out || !ma || !mm) return -1;
  int64_t ws = d - W;
  if (ws < 0) ws = 0;
  int64_t we = d + m + W;
  if (we > G) we = G;
  int64_t L = we - ws;
  if (L < 0) L = 0;
  int64_t off = d - ws;
  return nw_core(gcodes + ws, L, q, m, off, W, 0, 0, ma, mm, gap_open, gap_extend, ws, out, cigar, cigar_cap);
}

int orc_nw_literal(const uint8_t* gcodes, int64_t G, int64_t F, int32_t best_frag, const uint8_t* q, int32_t m,
                   int32_t match, int32_t mismatch, int32_t gap_open, int32_t gap_extend, orc_aln* out,
                   char* cigar, int32_t cigar_cap) {
  if (G <= 0 || F <= 0 || m <= 0 || best_frag < 0 || !out) return -1;
  int64_t ws = (int64_t)best_frag * F;
  int64_t nfr = ((int64_t)m + F - 1) / F;
  int64_t we = ws + nfr * F;
  if (we > G) we = G;
  if (ws > G) ws = G;
  return nw_core(gcodes + ws, we - ws, q, m, 0, -1, match, mismatch, 0, 0, gap_open, gap_extend, ws, out, cigar,
                 cigar_cap);
}

int orc_map_batch(const char* genome, int64_t G, int64_t F, const char* reads, const int64_t* offsets, int32_t R,
                  int32_t match, int32_t mismatch, int32_t nw_match, int32_t nw_mismatch, int32_t gap_open,
                  int32_t gap_extend, int32_t W, orc_hit* hits, orc_aln* alns, char* cigars, int32_t cigar_cap) {
  return orc_map_batch_step(genome, G, F, reads, offsets, R, match, mismatch, 1, nw_match, nw_mismatch, gap_open,
                            gap_extend, W, hits, alns, cigars, cigar_cap);
}

int orc_map_batch_step(const char* genome, int64_t G, int64_t F, const char* reads, const int64_t* offsets,
                       int32_t R, int32_t match, int32_t mismatch, int32_t step, int32_t nw_match,
                       int32_t nw_mismatch, int32_t gap_open, int32_t gap_extend, int32_t W, orc_hit* hits,
                       orc_aln* alns, char* cigars, int32_t cigar_cap) {
  uint8_t* g = (uint8_t*)malloc((size_t)G);
  if (!g) return -2;
  if (orc_encode(genome, G, g) != 0) { free(g); return -1; }
  for (int32_t r = 0; r < R; ++r) {
    int32_t m = (int32_t)(offsets[r + 1] - offsets[r]);
    int rc = orc_map_read_step(genome, G, F, reads + offsets[r], m, match, mismatch, step, &hits[r], 0);
    if (rc != 0) { free(g); return rc; }
    if (alns) {
      uint8_t* q = (uint8_t*)malloc((size_t)m);
      uint8_t* qs = (uint8_t*)malloc((size_t)m);
      orc_encode(reads + offsets[r], m, q);
      if (hits[r].strand == 1) orc_revcomp(q, m, qs); else memcpy(qs, q, (size_t)m);
      rc = orc_nw_banded(g, G, qs, m, hits[r].offset, W, nw_match, nw_mismatch, gap_open, gap_extend, &alns[r],
                         cigars ? cigars + (int64_t)r * cigar_cap : 0, cigars ? cigar_cap : 0);
      free(q); free(qs);
      if (rc != 0) { free(g); return rc; }
    }
  }
  free(g);
  return 0;
}

/* Both phases with base qualities (quals: Phred+33, same offsets as the reads; scale: the
   fixed point of the scores; phase two gaps are multiplied by scale). */
int orc_map_batch_pssm(const char* genome, int64_t G, int64_t F, const char* reads, const char* quals,
                       const int64_t* offsets, int32_t R, int32_t match, int32_t mismatch, int32_t scale,
                       int32_t nw_match, int32_t nw_mismatch, int32_t gap_open, int32_t gap_extend, int32_t W,
                       orc_hit* hits, orc_aln* alns, char* cigars, int32_t cigar_cap) {
  uint8_t* g = (uint8_t*)malloc((size_t)G);
  if (!g) return -2;
  if (orc_encode(genome, G, g) != 0) { free(g); return -1; }
  for (int32_t r = 0; r < R; ++r) {
    int32_t m = (int32_t)(offsets[r + 1] - offsets[r]);
    int rc = orc_map_read_pssm(genome, G, F, reads + offsets[r], quals + offsets[r], m, match, mismatch, scale,
                               &hits[r], 0);
    if (rc != 0) { free(g); return rc; }
    if (alns) {
      uint8_t* q = (uint8_t*)malloc((size_t)m);
      uint8_t* qs = (uint8_t*)malloc((size_t)m);
      int32_t* sc = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)m);
      int32_t *ma = sc, *mm = sc + m, *mas = sc + 2 * m, *mms = sc + 3 * m;
      orc_encode(reads + offsets[r], m, q);
      for (int32_t k = 0; k < m; ++k)
        orc_pssm_scores((unsigned char)quals[offsets[r] + k], nw_match, nw_mismatch, scale, &ma[k], &mm[k]);
      if (hits[r].strand == 1) {
        orc_revcomp(q, m, qs);
        for (int32_t k = 0; k < m; ++k) { mas[k] = ma[m - 1 - k]; mms[k] = mm[m - 1 - k]; }
      } else {
        memcpy(qs, q, (size_t)m);
        memcpy(mas, ma, sizeof(int32_t) * (size_t)m);
        memcpy(mms, mm, sizeof(int32_t) * (size_t)m);
      }
      rc = orc_nw_banded_pssm(g, G, qs, mas, mms, m, hits[r].offset, W, gap_open * scale, gap_extend * scale,
                              &alns[r], cigars ? cigars + (int64_t)r * cigar_cap : 0, cigars ? cigar_cap : 0);
      free(q); free(qs); free(sc);
      if (rc != 0) { free(g); return rc; }
    }
  }
  free(g);
  return 0;
}
