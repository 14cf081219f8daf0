// SAM text and mapping quality of mapped reads (host code; "Mapping qualities, read lengths,
// SAM output, and source code").
//
// MAPQ = -100 log2(p), p = second-best / best fragment score (the probability that the
// mapping is wrong, as the paper defines it), rounded to the nearest integer and capped at
// 254 (SAM's largest defined value); 254 when the second score is 0, 0 when the best score is
// 0 or not above the second.  A read is reported mapped only when phase one did not flag it
// (second / best < 0.9, i.e. MAPQ above 15.2) and phase two found an in-band alignment.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "../../include/maxss.h"

int32_t mss_mapq(int32_t best_score, int32_t second_score) {
  if (best_score <= 0) return 0;
  if (second_score <= 0) return 254;
  if (second_score >= best_score) return 0;
  const double q = -100.0 * log2((double)second_score / (double)best_score);
  const long v = lround(q);
  return v > 254 ? 254 : (int32_t)v;
}

namespace {

char comp_base(char c) {
  switch (c) {
    case 'A': case 'a': return 'T';
    case 'C': case 'c': return 'G';
    case 'G': case 'g': return 'C';
    case 'T': case 't': return 'A';
    default: return 'N';
  }
}

char upper_base(char c) { return (c >= 'a' && c <= 'z') ? (char)(c - 32) : c; }

void append_int(std::string& s, int64_t v) {
  char b[32];
  snprintf(b, sizeof(b), "%lld", (long long)v);
  s += b;
}

}  // namespace

int64_t mss_format_sam(const char* ref_name, int64_t ref_len, const char* reads, const int64_t* offsets, int32_t R,
                       const mss_hit* hits, const mss_aln* alns, const char* cigars, int32_t cigar_stride,
                       int32_t header, char* out, int64_t cap) {
  if (!ref_name || !*ref_name || ref_len < 1 || R < 0 || (R > 0 && (!reads || !offsets || !hits || !alns)))
    return MSS_EINVAL;
  if (cigars && cigar_stride < 1) return MSS_EINVAL;
  for (const char* p = ref_name; *p; ++p)
    if (*p == '\t' || *p == '\n' || *p == ' ') return MSS_EINVAL;
  std::string s;
  if (header) {
    s += "@HD\tVN:1.6\tSO:unsorted\n@SQ\tSN:";
    s += ref_name;
    s += "\tLN:";
    append_int(s, ref_len);
    s += "\n@PG\tID:maxss\tPN:maxss\n";
  }
  for (int32_t r = 0; r < R; ++r) {
    const int64_t off = offsets[r], m = offsets[r + 1] - offsets[r];
    if (m < 0) return MSS_EINVAL;
    const mss_hit& h = hits[r];
    const mss_aln& a = alns[r];
    const bool aligned = a.score != MSS_NW_NONE && a.cigar_len >= 0 && a.gstart >= 0 && a.gstart < ref_len;
    const bool mapped = !(h.flags & MSS_HIT_REPEAT) && aligned;
    const bool rev = mapped && h.strand == 1;
    s += 'r';
    append_int(s, r);
    s += '\t';
    append_int(s, mapped ? (rev ? 16 : 0) : 4);
    s += '\t';
    if (mapped) {
      s += ref_name;
      s += '\t';
      append_int(s, a.gstart + 1);
      s += '\t';
      append_int(s, mss_mapq(h.best_score, h.second_score));
      s += '\t';
      if (cigars && a.cigar_len > 0 && a.cigar_len < cigar_stride)
        s.append(cigars + (int64_t)r * cigar_stride, (size_t)a.cigar_len);
      else
        s += '*';
    } else {
      s += "*\t0\t0\t*";
    }
    s += "\t*\t0\t0\t";
    if (m == 0) {
      s += '*';
    } else if (rev) {  // SEQ on the forward genome strand
      for (int64_t k = m - 1; k >= 0; --k) s += comp_base(reads[off + k]);
    } else {
      for (int64_t k = 0; k < m; ++k) s += upper_base(reads[off + k]);
    }
    s += "\t*";
    if (mapped) {
      s += "\tAS:i:";
      append_int(s, a.score);
    }
    s += "\tZM:i:";
    append_int(s, h.best_score);
    s += "\tXS:i:";
    append_int(s, h.second_score);
    s += '\n';
  }
  const int64_t n = (int64_t)s.size();
  if (out && cap > n) {
    memcpy(out, s.data(), (size_t)n);
    out[n] = '\0';
  }
  return n;
}
