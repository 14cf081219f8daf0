/*
 * Seeded synthetic genome and read generator.
 *
 * Shared input source for the CPU oracle and the CUDA path.  It holds none of the
 * mapping arithmetic (no scoring, no Kadane, no alignment): it only draws genomes and
 * reads with the shapes of the paper's workloads (Section "Data simulation": reads with
 * 10-30% divergence and gaps up to 30 bp in the read or the genome; Section "Applications
 * on real data": short, very divergent ancient reads).
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014) expands the user seed into the
 * 256-bit state of xoshiro256** (Blackman and Vigna 2018).  Both are written from their
 * published definitions.  Everything is integer arithmetic, so the output is identical on
 * x86_64 and aarch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

/* uniform integer in [0, n) by 128-bit multiply-high (Lemire), n >= 1 */
static uint64_t rng_below(rng_t* r, uint64_t n) {
  unsigned __int128 p = (unsigned __int128)rng_next(r) * n;
  return (uint64_t)(p >> 64);
}

/* uniform in [0, 1) with 53 random bits */
static double rng_unit(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* Bernoulli with probability p given as an integer threshold on 2^32 */
static int rng_bern32(rng_t* r, uint32_t thr) { return (uint32_t)(rng_next(r) >> 32) < thr; }

static uint32_t prob_to_thr(double p) {
  if (p <= 0) return 0;
  if (p >= 1) return 0xFFFFFFFFu;
  return (uint32_t)(p * 4294967296.0);
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

/* one base with GC content gc (threshold form so that the draw is platform independent) */
static char rng_base_gc(rng_t* r, uint32_t gc_thr) {
  uint32_t u = (uint32_t)(rng_next(r) >> 32);
  int gc = u < gc_thr;
  int bit = (int)((rng_next(r) >> 63) & 1);
  return gc ? (bit ? 'G' : 'C') : (bit ? 'T' : 'A');
}

static char comp_base(char c) {
  switch (c) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return 'N';
  }
}

/* a different base than c, uniformly among the other three (N maps to a uniform base) */
static char rng_other_base(rng_t* r, char c) {
  int k = (int)rng_below(r, 3);
  int ci = (c == 'A') ? 0 : (c == 'C') ? 1 : (c == 'G') ? 2 : (c == 'T') ? 3 : -1;
  if (ci < 0) return BASES[rng_below(r, 4)];
  int o = k >= ci ? k + 1 : k;
  return BASES[o];
}

/*
 * Genome.
 *   G            length
 *   gc           GC fraction of i.i.d. background bases
 *   copy_frac    fraction of G made of exact copies of earlier segments (lengths U[copy_min, copy_max])
 *   fam_frac     fraction of G covered by interspersed repeats: copies of fam_count consensus
 *                sequences of length fam_len, each copy at fam_div substitution divergence
 *   n_frac       fraction of G covered by N runs of length U[n_min, n_max]
 * Returns 0 on success.  out must hold G bytes.
 */
int gen_genome(uint64_t seed, int64_t G, double gc, double copy_frac, int64_t copy_min, int64_t copy_max,
               double fam_frac, int32_t fam_count, int32_t fam_len, double fam_div, double n_frac, int64_t n_min,
               int64_t n_max, char* out) {
  if (G <= 0 || !out) return -1;
  rng_t r;
  rng_seed(&r, seed);
  uint32_t gc_thr = prob_to_thr(gc);
  for (int64_t i = 0; i < G; ++i) out[i] = rng_base_gc(&r, gc_thr);

  /* interspersed repeat families */
  if (fam_frac > 0 && fam_count > 0 && fam_len > 0 && fam_len < G) {
    char* fam = (char*)malloc((size_t)fam_count * fam_len);
    if (!fam) return -2;
    for (int64_t i = 0; i < (int64_t)fam_count * fam_len; ++i) fam[i] = rng_base_gc(&r, gc_thr);
    int64_t n_copies = (int64_t)(fam_frac * (double)G / fam_len);
    uint32_t div_thr = prob_to_thr(fam_div);
    for (int64_t c = 0; c < n_copies; ++c) {
      int64_t f = (int64_t)rng_below(&r, (uint64_t)fam_count);
      int64_t pos = (int64_t)rng_below(&r, (uint64_t)(G - fam_len));
      int rc = (int)((rng_next(&r) >> 63) & 1);
      for (int64_t k = 0; k < fam_len; ++k) {
        char b = rc ? comp_base(fam[f * fam_len + (fam_len - 1 - k)]) : fam[f * fam_len + k];
        if (rng_bern32(&r, div_thr)) b = rng_other_base(&r, b);
        out[pos + k] = b;
      }
    }
    free(fam);
  }

  /* exact segment copies */
  if (copy_frac > 0 && copy_max >= copy_min && copy_min > 0 && 2 * copy_max < G) {
    int64_t budget = (int64_t)(copy_frac * (double)G);
    while (budget > 0) {
      int64_t len = copy_min + (int64_t)rng_below(&r, (uint64_t)(copy_max - copy_min + 1));
      if (len > budget) len = budget;
      int64_t src = (int64_t)rng_below(&r, (uint64_t)(G - len));
      int64_t dst = (int64_t)rng_below(&r, (uint64_t)(G - len));
      if ((dst < src + len) && (src < dst + len)) continue; /* overlapping copy: redraw */
      memmove(out + dst, out + src, (size_t)len);
      budget -= len;
    }
  }

  /* N runs */
  if (n_frac > 0 && n_max >= n_min && n_min > 0 && n_max < G) {
    int64_t budget = (int64_t)(n_frac * (double)G);
    while (budget > 0) {
      int64_t len = n_min + (int64_t)rng_below(&r, (uint64_t)(n_max - n_min + 1));
      if (len > budget) len = budget;
      int64_t pos = (int64_t)rng_below(&r, (uint64_t)(G - len));
      memset(out + pos, 'N', (size_t)len);
      budget -= len;
    }
  }
  return 0;
}

/*
 * Reads.
 *   lengths[R]          exact final length of each read
 *   sub_lo, sub_hi      substitution probability, drawn per read uniformly in [sub_lo, sub_hi]
 *   gap_mode            0: no gaps; 1: exactly one gap, length U[gap_min, gap_max];
 *                       2: U{0..gap_count_max} gaps, length geometric(gap_p) truncated to gap_max
 *   deam_rate           C->T at 5' read positions i < deam_len with prob deam_rate*(deam_len-i)/deam_len
 *   strand: 50/50; a reverse read is the reverse complement of the simulated forward read
 * Outputs: reads (concatenated, offsets[R+1]), true start (leftmost genome base covered),
 * strand (0 +, 1 -), number of substitutions and gap bases drawn.
 * The source span is required to be free of N.  Returns 0 on success.
 */
int gen_reads(uint64_t seed, const char* genome, int64_t G, int32_t R, const int32_t* lengths, double sub_lo,
              double sub_hi, int32_t gap_mode, int32_t gap_count_max, int32_t gap_min, int32_t gap_max, double gap_p,
              double deam_rate, int32_t deam_len, char* reads, int64_t* offsets, int64_t* true_start,
              int8_t* true_strand, int32_t* n_sub, int32_t* n_gap, int32_t* true_rel) {
  rng_t r;
  rng_seed(&r, seed ^ 0x5EEDF00Dull);
  /* prefix count of N for span checks */
  int64_t* ncount = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
  if (!ncount) return -2;
  ncount[0] = 0;
  for (int64_t i = 0; i < G; ++i) ncount[i + 1] = ncount[i] + (genome[i] == 'N' || genome[i] == 'n');
  int32_t maxlen = 0;
  for (int32_t i = 0; i < R; ++i) maxlen = lengths[i] > maxlen ? lengths[i] : maxlen;
  char* buf = (char*)malloc((size_t)maxlen + 8);
  int32_t* rel = (int32_t*)malloc(sizeof(int32_t) * ((size_t)maxlen + 8));
  if (!buf || !rel) { free(buf); free(rel); free(ncount); return -2; }
  offsets[0] = 0;
  for (int32_t i = 0; i < R; ++i) {
    int32_t m = lengths[i];
    /* draw gap events: position in read (1..m-1), kind (0 = insertion in read, 1 = deletion) and length */
    int32_t ng = 0, gpos[8], gkind[8], glen[8];
    if (gap_mode == 1) {
      ng = 1;
    } else if (gap_mode == 2) {
      ng = (int32_t)rng_below(&r, (uint64_t)gap_count_max + 1);
      if (ng > 8) ng = 8;
    }
    int64_t del_total = 0;
    int32_t ins_total = 0;
    for (int32_t g = 0; g < ng; ++g) {
      gpos[g] = m > 1 ? 1 + (int32_t)rng_below(&r, (uint64_t)(m - 1)) : 0;
      gkind[g] = (int32_t)((rng_next(&r) >> 63) & 1);
      if (gap_mode == 1) {
        glen[g] = gap_min + (int32_t)rng_below(&r, (uint64_t)(gap_max - gap_min + 1));
      } else {
        int32_t L = 1;
        uint32_t thr = prob_to_thr(1.0 - gap_p); /* continue with probability 1-p */
        while (L < gap_max && rng_bern32(&r, thr)) ++L;
        glen[g] = L;
      }
      if (gkind[g] == 1) del_total += glen[g]; else ins_total += glen[g];
    }
    /* sort events by read position (insertion sort, ng <= 8) */
    for (int32_t a = 1; a < ng; ++a)
      for (int32_t b = a; b > 0 && gpos[b] < gpos[b - 1]; --b) {
        int32_t t;
        t = gpos[b]; gpos[b] = gpos[b - 1]; gpos[b - 1] = t;
        t = gkind[b]; gkind[b] = gkind[b - 1]; gkind[b - 1] = t;
        t = glen[b]; glen[b] = glen[b - 1]; glen[b - 1] = t;
      }
    int64_t span = (int64_t)m + del_total; /* upper bound on genome bases consumed */
    if (span > G) { free(buf); free(rel); free(ncount); return -3; }
    int64_t start = -1;
    for (int attempt = 0; attempt < 100000; ++attempt) {
      int64_t s = (int64_t)rng_below(&r, (uint64_t)(G - span + 1));
      if (ncount[s + span] - ncount[s] == 0) { start = s; break; }
    }
    if (start < 0) { free(buf); free(rel); free(ncount); return -4; }
    double p = sub_lo + (sub_hi - sub_lo) * rng_unit(&r);
    uint32_t sub_thr = prob_to_thr(p);
    int32_t k = 0, ev = 0, subs = 0, gapb = 0;
    int64_t gp = start;
    while (k < m) {
      while (ev < ng && gpos[ev] == k) {
        if (gkind[ev] == 1) {
          gp += glen[ev];
          gapb += glen[ev];
        } else {
          for (int32_t t = 0; t < glen[ev] && k < m; ++t) {
            rel[k] = -1;                       /* an inserted base has no genome position */
            buf[k++] = BASES[rng_below(&r, 4)];
            ++gapb;
          }
        }
        ++ev;
      }
      if (k >= m) break;
      rel[k] = (int32_t)(gp - start);
      char b = genome[gp++];
      if (b >= 'a' && b <= 'z') b = (char)(b - 32);
      if (rng_bern32(&r, sub_thr)) { b = rng_other_base(&r, b); ++subs; }
      buf[k++] = b;
    }
    int rc = (int)((rng_next(&r) >> 63) & 1);
    char* dst = reads + offsets[i];
    if (rc) {
      for (int32_t t = 0; t < m; ++t) dst[t] = comp_base(buf[m - 1 - t]);
    } else {
      memcpy(dst, buf, (size_t)m);
    }
    /* true position of each base in the forward-strand orientation of the read (SAM's SEQ),
       relative to true_start; -1 for inserted bases */
    if (true_rel) memcpy(true_rel + offsets[i], rel, sizeof(int32_t) * (size_t)m);
    if (deam_rate > 0 && deam_len > 0) {
      for (int32_t t = 0; t < deam_len && t < m; ++t) {
        double pr = deam_rate * (double)(deam_len - t) / (double)deam_len;
        if (dst[t] == 'C' && rng_bern32(&r, prob_to_thr(pr))) dst[t] = 'T';
      }
    }
    offsets[i + 1] = offsets[i] + m;
    if (true_start) true_start[i] = start;
    if (true_strand) true_strand[i] = (int8_t)rc;
    if (n_sub) n_sub[i] = subs;
    if (n_gap) n_gap[i] = gapb;
  }
  free(buf);
  free(rel);
  free(ncount);
  return 0;
}

/* read lengths: mode 0 constant a; mode 1 uniform choice from list[0..n); mode 2 round(lognormal(ln a_med, sigma))
   clipped to [lo, hi] (sigma given in thousandths to keep the ABI integer) */
int gen_lengths(uint64_t seed, int32_t R, int32_t mode, const int32_t* list, int32_t n, double median, double sigma,
                int32_t lo, int32_t hi, int32_t* out) {
  rng_t r;
  rng_seed(&r, seed ^ 0x1E47115ull);
  for (int32_t i = 0; i < R; ++i) {
    if (mode == 0) {
      out[i] = list[0];
    } else if (mode == 1) {
      out[i] = list[rng_below(&r, (uint64_t)n)];
    } else {
      /* Box-Muller on two uniform draws */
      double u1 = rng_unit(&r), u2 = rng_unit(&r);
      if (u1 < 1e-300) u1 = 1e-300;
      double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
      double v = median * exp(sigma * z);
      int32_t L = (int32_t)floor(v + 0.5);
      if (L < lo) L = lo;
      if (L > hi) L = hi;
      out[i] = L;
    }
  }
  return 0;
}
