/*
 * maxss.h — C ABI of libmaxss, a GB300 (sm_103a) implementation of the MaxSSmap hot path
 * (Turki & Roshan, "MaxSSmap: A GPU program for mapping divergent short reads to genomes
 * with the maximum scoring subsequence", arXiv 1403.2136).
 *
 * Phase one ("First phase of MaxSSmap"): for every read, on both strands, the maximum
 * scoring subsequence (section "Maximum scoring subsequence": the best-sum contiguous run of
 * match/mismatch scores, empty run allowed) along every ungapped diagonal d of the genome;
 * fragment f (section "Coalescent global memory access": fixed-size disjoint fragments, the
 * last one padded with N) owns diagonals [fF, (f+1)F) and its windows run into the next
 * fragment (junctions, Figure 1); per read the best and second-best fragment, and the repeat
 * test second/best >= 0.9.  Phase two ("Second phase of MaxSSmap"): Needleman-Wunsch of the
 * read against the genome around the best diagonal.
 *
 * Conventions for every entry point:
 *   - return MSS_OK (0) or a negative mss_status; mss_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread);
 *   - no call aborts or exits the process, and nothing falls back to the CPU;
 *   - the caller owns every input and output buffer; the context owns the packed genome and
 *     its device workspaces;
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream);
 *   - *_device entry points take device pointers, enqueue work on the stream and return
 *     without synchronising; errors found on the device are reported by mss_sync();
 *     the other entry points take host pointers, copy in and out, and synchronise.
 *   - base characters: A C G T N in either case; anything else is MSS_EINVAL.
 */
#ifndef MAXSS_H
#define MAXSS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MSS_API __attribute__((visibility("default")))
#else
#define MSS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mss_status;

#define MSS_OK 0
#define MSS_EINVAL (-1)     /* bad argument, bad character, bad size */
#define MSS_ENOMEM (-2)     /* device or host allocation failed */
#define MSS_ECUDA (-3)      /* a CUDA runtime call failed */
#define MSS_EREADLEN (-4)   /* read length 0 or above the context's maximum (at most 2432) */
#define MSS_EOVERFLOW (-5)  /* max_read_len * match would overflow the 16-bit scan lanes */
#define MSS_ETIMEOUT (-6)   /* a bounded device wait gave up */
#define MSS_ESTATE (-7)     /* inconsistent internal state (a self-check failed) */

/* Longest read accepted.  The paper's kernel holds a (m+16)x4x5-byte query profile in 48 KB
   of shared memory, which caps m at 2432 ("Shared memory"); the cap is kept here as the
   validity bound of the ABI. */
#define MSS_MAX_READ_LEN 2432

/* Score of an mss_aln for which no in-band alignment exists. */
#define MSS_NW_NONE (-2147483647 - 1)

typedef struct mss_ctx mss_ctx;

typedef struct {
  int64_t frag_len;     /* F: diagonals per fragment, 16 <= F <= 2^20 (0 = default 2048) */
  int32_t max_read_len; /* longest read that will be mapped, 1..MSS_MAX_READ_LEN (0 = 2432) */
  int32_t reserved;     /* must be 0 */
} mss_genome_params;

typedef struct {
  int32_t match;    /* score of an identical A/C/G/T pair, 1..127 */
  int32_t mismatch; /* score of any other pair (N never matches), -128..0 */
} mss_score_params;

/* Per-read result of phase one (32 bytes). */
typedef struct {
  int32_t best_frag;    /* fragment with the highest score; ties -> lowest index */
  int32_t second_frag;  /* best among the other fragments (ties -> lowest), -1 if only one */
  int32_t best_score;   /* S(best_frag) >= 0 */
  int32_t second_score; /* S(second_frag), 0 if there is no second fragment */
  int64_t offset;       /* diagonal d of best_frag attaining best_score: genome index of read
                           base 0 on the chosen strand; ties -> + strand first, then smallest d */
  int32_t strand;       /* 0: read as given, 1: reverse complement */
  int32_t flags;        /* bit 0 (MSS_HIT_REPEAT): best == 0 or 10*second >= 9*best */
} mss_hit;

#define MSS_HIT_REPEAT 1

typedef struct {
  int32_t match;      /* default 5 ("Second phase of MaxSSmap") */
  int32_t mismatch;   /* default -4 */
  int32_t gap_open;   /* cost of the first base of a gap, default -26 (linear = open == extend) */
  int32_t gap_extend; /* cost of each further base; require gap_open <= gap_extend <= 0 */
  int32_t band;       /* W, 0..63: cells with |j - i - (d - window start)| <= W */
  int32_t reserved;   /* must be 0 */
} mss_nw_params;

/* Per-read result of phase two (24 bytes). */
typedef struct {
  int32_t score;     /* alignment score, MSS_NW_NONE if no in-band alignment exists */
  int32_t cigar_len; /* characters written (without the NUL); -1 if the slot was too small */
  int64_t gstart;    /* genome index of the first aligned genome base */
  int64_t gend;      /* one past the last aligned genome base */
} mss_aln;

typedef struct {
  int64_t genome_len;   /* G */
  int64_t frag_len;     /* F */
  int64_t num_frags;    /* NF = ceil(G / F) */
  int64_t padded_len;   /* Gp = NF * F */
  int32_t max_read_len;
  int32_t num_sms;
} mss_genome_info;

/* Scan configuration: chosen by mss_autotune() or set directly. */
typedef struct {
  int32_t variant;       /* 0: int16 DPX add-max-relu (any scores); 1: f16 add-relu on the FMA
                            pipe + DPX running max (exact when max_read_len*match <= 2048 and the
                            scores are small integers); -1 = pick automatically */
  int32_t pairs;         /* diagonal pairs per thread: 4 or 8 (0 = default 8) */
  int32_t queries;       /* query sequences (read strands) per CTA: 4 or 8 (0 = default: 4 with
                            8 pairs, else 8); 8 pairs with 8 queries is not built */
  int32_t ctas_per_sm;   /* persistent CTAs per SM (0 = occupancy maximum) */
  int32_t min_items_per_cta; /* split the genome into chunks until there are this many work
                                items per CTA (0 = default 4) */
  int32_t threads;       /* threads per CTA: 256 or 128 (0 = default 256); 128 is built for 8
                            pairs x 4 queries at read step 1 without base qualities */
} mss_tune;

/* Load and 2-bit pack a genome (host ASCII, length len >= 1).  Creates *out. */
MSS_API mss_status mss_load_genome(mss_ctx** out, const char* seq, int64_t len, const mss_genome_params* p,
                           void* stream);
/* Same, with the ASCII genome already in device memory. */
MSS_API mss_status mss_load_genome_device(mss_ctx** out, const char* d_seq, int64_t len, const mss_genome_params* p,
                                  void* stream);
MSS_API mss_status mss_get_info(const mss_ctx* ctx, mss_genome_info* info);
/* Change F after loading (the packed genome does not depend on F). */
MSS_API mss_status mss_set_frag_len(mss_ctx* ctx, int64_t frag_len);
/* Read step of phase one ("MaxSSmap_fast" paragraph: the faster version considers every other
   nucleotide of the read): 1 = every read base (default), 2 = read bases 0, 2, 4, ... only,
   i.e. step k of diagonal d compares read base 2k with genome base d + 2k, on each strand
   after reverse complementing.  Fragment maxima, top-2, the repeat flag and the best
   diagonal follow from those scores; phase two (nw_align) always aligns the whole read.
   Step 2 runs with the default scan shape (8 lane pairs x 4 query strands); other mss_tune
   shapes make the mapping calls fail with MSS_EINVAL.  Errors: MSS_EINVAL for a null ctx or
   a step other than 1 or 2. */
MSS_API mss_status mss_set_read_step(mss_ctx* ctx, int32_t step);
/* Second-fragment rule ("First phase of MaxSSmap" keeps the second-best fragment to flag
   repeats; the paper does not say whether the best fragment's neighbours may be that second).
   0 (default): any fragment other than the best.  1: the best fragment f with |f - best| > 1
   (-1 and score 0 when none exists); the repeat flag follows the chosen second.  Applies to
   mss_map_reads*, mss_map_align and mss_map_reads_proposed.  Errors: MSS_EINVAL for a null ctx
   or a rule other than 0 or 1. */
MSS_API mss_status mss_set_second_rule(mss_ctx* ctx, int32_t exclude_neighbors);
MSS_API int32_t mss_get_read_step(const mss_ctx* ctx);  /* -1 for a null ctx */
MSS_API mss_status mss_set_tune(mss_ctx* ctx, const mss_tune* t);
MSS_API mss_status mss_get_tune(const mss_ctx* ctx, mss_tune* t);

/*
 * Phase one for R reads (host buffers): reads = concatenated ASCII, offsets[R+1] (int64,
 * offsets[0] = 0, non-decreasing), each length 1..max_read_len.  out[R] receives the hits in
 * input order.  Synchronous.
 */
MSS_API mss_status mss_map_reads(mss_ctx* ctx, const char* reads, const int64_t* offsets, int32_t R,
                         const mss_score_params* sp, mss_hit* out, void* stream);
/*
 * Phase one, device buffers: d_reads, d_offsets[R+1], d_out[R] in device memory.  max_len
 * is a host-side upper bound on the read lengths (<= the context's max_read_len).  The work
 * is enqueued on the stream (as one CUDA graph when the stream is not the legacy default
 * stream); the context may be reused only in stream order.  Device-side errors (bad
 * character, bad length) are reported by mss_sync().
 */
MSS_API mss_status mss_map_reads_device(mss_ctx* ctx, const char* d_reads, const int64_t* d_offsets, int32_t R,
                                int32_t max_len, const mss_score_params* sp, mss_hit* d_out, void* stream);

/*
 * Phase two for R reads (host buffers): hits from phase one, alignments out[R], CIGAR strings
 * into cigar_buf (R slots of cigar_stride bytes, NUL-terminated, ops M/I/D).  Glocal (read
 * end to end, genome ends free) affine-gap alignment of the read on hits[r].strand in the
 * window [offset-W, offset+m+W) clipped to the genome, banded around the seed diagonal;
 * traceback ties prefer a match/mismatch step, then a gap in the read (D), then a gap in the
 * genome (I); a gap is closed in preference to extended; equal end scores -> smallest end.
 */
MSS_API mss_status nw_align(mss_ctx* ctx, const char* reads, const int64_t* offsets, int32_t R, const mss_hit* hits,
                    const mss_nw_params* np, mss_aln* out, char* cigar_buf, int32_t cigar_stride, void* stream);
/* Phase two, device buffers (enqueued, see mss_map_reads_device). */
MSS_API mss_status nw_align_device(mss_ctx* ctx, const char* d_reads, const int64_t* d_offsets, int32_t R,
                           int32_t max_len, const mss_hit* d_hits, const mss_nw_params* np, mss_aln* d_out,
                           char* d_cigar_buf, int32_t cigar_stride, void* stream);

/*
 * nw_align_device with no allocation of any kind (the paper has no counterpart; this is a
 * deployment interface).  For callers that cannot call cudaMalloc: code running inside CUDA
 * stream capture, latency-critical serving loops, and processes whose device memory belongs
 * to a pool allocator.  Same arguments and results as nw_align_device; the traceback scratch
 * is a fixed 4 MiB array in the library's device image (held by every GPU that loads the
 * library until exit), so long reads get fewer concurrent traceback slots, never a failure,
 * as long as one slot fits (always true up to MSS_MAX_READ_LEN and band 63; otherwise
 * MSS_EINVAL).  The array's device address is looked up on the first call on each device:
 * make that first call outside any stream capture.  All calls share the array, so calls
 * that may run concurrently on the GPU race and must be ordered by the caller.
 */
MSS_API mss_status nw_align_device_noalloc(mss_ctx* ctx, const char* d_reads, const int64_t* d_offsets, int32_t R,
                                           int32_t max_len, const mss_hit* d_hits, const mss_nw_params* np,
                                           mss_aln* d_out, char* d_cigar_buf, int32_t cigar_stride, void* stream);

/*
 * Both phases for R reads with host buffers and one upload: reads/offsets as in
 * mss_map_reads; hits[R], alns[R] and cigar_buf (R slots of cigar_stride bytes) receive the
 * results.  Synchronous.  This is the end-to-end call (host -> device -> host).
 */
MSS_API mss_status mss_map_align(mss_ctx* ctx, const char* reads, const int64_t* offsets, int32_t R,
                                 const mss_score_params* sp, const mss_nw_params* np, mss_hit* hits, mss_aln* alns,
                                 char* cigar_buf, int32_t cigar_stride, void* stream);

/* Wait for the stream and return the first device-side error recorded since the last call. */
MSS_API mss_status mss_sync(mss_ctx* ctx, void* stream);

/*
 * Pick the scan configuration (and, when allow_frag_len is non-zero, F among 1024, 2048,
 * 4096, 8192) by timing phase one on the given device reads.  The result is stored in the
 * context.  Changing F changes which fragments exist, so results depend on it.
 */
MSS_API mss_status mss_autotune(mss_ctx* ctx, const char* d_reads, const int64_t* d_offsets, int32_t R, int32_t max_len,
                        const mss_score_params* sp, int32_t allow_frag_len, void* stream);

/*
 * Kernel timing of the scan: when enabled, every phase-one call records two CUDA events on its
 * stream immediately around the scan kernel (inside the captured graph as event nodes).
 * mss_scan_time_ms() waits for the last recorded pair and returns the scan kernel's duration.
 */
MSS_API mss_status mss_scan_timing(mss_ctx* ctx, int32_t enable);
MSS_API mss_status mss_scan_time_ms(mss_ctx* ctx, float* ms);

/* Number of kernel launches enqueued by this context since it was created. */
MSS_API int64_t mss_launch_count(const mss_ctx* ctx);

/* Copy genome codes [start, start+n) (0..3 = ACGT, 4 = N/padding) into host memory, decoded
   from the packed device genome (a check of the packing kernel). */
MSS_API mss_status mss_genome_codes(const mss_ctx* ctx, int64_t start, int64_t n, uint8_t* out);

/*
 * Throughput probes of the packed 16-bit instructions the scan uses, in warp-instructions per
 * SM clock (at the clock the device reports as its maximum), each from 16 independent chains
 * per thread: rates[0] packed int16 DPX add-max, [1] f16x2 FMA with relu, [2] PRMT and f16x2
 * FMA-relu interleaved (the integer and FMA pipes both busy: the two-pipe peak of the scan's
 * roofline), [3] PRMT, [4] three-input packed int16 max, [5] the scan's own mix (2 PRMT +
 * 2 FMA-relu + 1 three-input max per two lane pairs), [6] DPX add-max and FMA-relu
 * interleaved.  The first min(n_rates, 7) slots are filled; clk_mhz receives the clock used.
 * Allocates a small device buffer for the duration of the call.  MSS_EINVAL for null
 * pointers or n_rates < 1, MSS_ECUDA on a CUDA failure.
 */
MSS_API mss_status mss_probe_pipes(double* rates, int32_t n_rates, double* clk_mhz);

/*
 * Self-check of failure detection (a property of this library, not of the paper's method):
 * every device wait of the kernels here is bounded and, when it gives up, sets an error bit
 * that the next synchronising call returns as MSS_ETIMEOUT instead of hanging.  This call
 * launches one block that waits limit_us microseconds (1 .. 1,000,000) on an mbarrier phase
 * that nothing completes, with the same bounded wait the scan uses, then synchronises the
 * stream.  Returns MSS_ETIMEOUT when the wait gave up as designed (the error word is cleared
 * and the context stays usable), MSS_EINVAL for a null context or a limit out of range,
 * MSS_ECUDA on a launch failure.
 */
MSS_API mss_status mss_check_wait_timeout(mss_ctx* ctx, uint32_t limit_us, void* stream);

/* ==========================================================================================
 * Learned fragment proposal (a step added to the method; the paper has none).  A small 1-D
 * CNN (one-hot bases -> 4 x conv1d(128 channels, kernel 7, "same", ReLU) -> max (or mean) over
 * positions -> L2 norm; BF16 weights, FP32 accumulation) embeds reads and genome fragments.
 * The dot product ranks fragments per read (maximum over the read's two strands); the exact
 * scan then runs only on the top K fragments, and reads whose best proposal score is below a
 * threshold fall back to the exhaustive scan.  Trained on labels produced by the exhaustive
 * scan (softmax cross-entropy of the true best fragment against the other candidates,
 * AdamW on FP32 master weights).
 * ========================================================================================== */
typedef struct mss_prop mss_prop;

/* Create a model with deterministic random weights (uniform(+-sqrt(6/fan_in)), biases 0.01). */
MSS_API mss_status mss_prop_create(mss_prop** out, uint64_t seed, void* stream);
MSS_API void mss_prop_free(mss_prop* p);
/* Number of parameters and the flat fp32 layout: W1 [7][4][128], b1 [128], then for layers
   2..4: W [7][128 in][128 out], b [128].  get/set copy host <-> device; n must equal
   mss_prop_param_count() (else MSS_EINVAL). */
MSS_API int64_t mss_prop_param_count(void);
MSS_API mss_status mss_prop_get_params(const mss_prop* p, float* host, int64_t n);
MSS_API mss_status mss_prop_set_params(mss_prop* p, const float* host, int64_t n);
/* Pooling of the last layer's outputs over a sequence's positions (a reading the proposal
   leaves open): MSS_POOL_MAX (the default) keeps each channel's maximum (the first position
   on ties) and routes its gradient there; MSS_POOL_MEAN takes each channel's mean over the
   sequence's positions (FP32 sum / length) and spreads the gradient with weight 1 / length.
   The setting applies to every later embedding, gradient and training step and is saved in
   checkpoints; an index built under another pooling (or other weights) must be rebuilt.
   MSS_EINVAL for another value.  mss_prop_get_pooling returns -1 for a null model. */
#define MSS_POOL_MAX 0
#define MSS_POOL_MEAN 1
MSS_API mss_status mss_prop_set_pooling(mss_prop* p, int32_t pooling);
MSS_API int32_t mss_prop_get_pooling(const mss_prop* p);
/* Input codes for the network (device buffers, codes 0..3 = ACGT, 4 = N/padding, row stride
   ld): reads (d_idx selects reads, d_strand 1 = reverse complement; both may be NULL) and
   genome windows [start, start + len). */
MSS_API mss_status mss_prop_read_codes(mss_prop* p, const char* d_reads, const int64_t* d_offsets,
                                       const int32_t* d_idx, const int8_t* d_strand, int32_t n, int32_t ld,
                                       uint8_t* d_codes, int32_t* d_lens, void* stream);
MSS_API mss_status mss_prop_window_codes(mss_prop* p, const mss_ctx* ctx, const int64_t* d_starts, int32_t n,
                                         int32_t len, int32_t ld, uint8_t* d_codes, int32_t* d_lens, void* stream);
/* Embeddings of n code sequences (lengths <= maxlen <= ld) into d_emb [n][128] (fp32).
   MSS_EINVAL for n < 0 or maxlen outside [1, ld]; MSS_ETIMEOUT if a bounded wait of a
   tensor-core kernel gave up (the model stays usable). */
MSS_API mss_status mss_prop_embed_device(mss_prop* p, const uint8_t* d_codes, const int32_t* d_lens, int32_t ld,
                                         int32_t n, int32_t maxlen, float* d_emb, void* stream);
/* Parameter gradient (d_grad, mss_prop_param_count() floats) of sum_i <d_demb[i], emb_i>. */
MSS_API mss_status mss_prop_grad_device(mss_prop* p, const uint8_t* d_codes, const int32_t* d_lens, int32_t ld,
                                        int32_t n, int32_t maxlen, const float* d_demb, float* d_grad, void* stream);
/* One training step: B read sequences (on their labelled strand) against C candidate
   fragment windows; label[i] = index of read i's best fragment among the candidates; loss =
   mean softmax cross-entropy of <e_read, e_cand> / temperature.  loss_out (host) optional.
   MSS_EINVAL unless B >= 1, 2 <= C <= 1024, lr > 0 and temperature > 0. */
MSS_API mss_status mss_prop_train_step(mss_prop* p, const uint8_t* d_rcodes, const int32_t* d_rlens, int32_t ld_r,
                                       int32_t B, int32_t maxlen_r, const uint8_t* d_ccodes, const int32_t* d_clens,
                                       int32_t ld_c, int32_t C, int32_t maxlen_c, const int32_t* d_labels, float lr,
                                       float temperature, float weight_decay, float* loss_out, void* stream);
/* Embed every fragment window [fF, fF + F + max_read_len - 1) of the context's genome.
   MSS_EREADLEN for max_read_len outside [1, the context's maximum]; MSS_EINVAL for a window
   above 65,536 bases. */
MSS_API mss_status mss_prop_build_index(mss_prop* p, mss_ctx* ctx, int32_t max_read_len, void* stream);
/* Proposal + exact rescoring: per read the top K fragments by embedding score (ties -> lower
   fragment), the exact scan of those K (both strands), and best / second among them; reads
   whose best proposal score is below tau are mapped by the exhaustive scan instead.  Optional
   outputs: d_cand [R][K] candidate fragments, d_top_score [R] best proposal score,
   *n_fallback (host) the number of fallback reads.  Synchronous.  MSS_ESTATE when no index
   was built for this context's genome or the fragment length changed since; MSS_EINVAL for
   K outside [1, 1024] or bad scores; MSS_EREADLEN for max_len outside [1, the context's
   maximum]. */
MSS_API mss_status mss_map_reads_proposed(mss_ctx* ctx, mss_prop* p, const char* d_reads, const int64_t* d_offsets,
                                          int32_t R, int32_t max_len, const mss_score_params* sp, int32_t K,
                                          float tau, mss_hit* d_out, int32_t* d_cand, float* d_top_score,
                                          int32_t* n_fallback, void* stream);
/* Checkpoint: master weights, Adam state and the pooling in a flat file with a header and a
   CRC-32 (files written before the pooling field existed load as max pooling).
   mss_prop_load rejects (MSS_EINVAL, model unchanged) a file with another header or size, a
   truncated file or a CRC mismatch. */
MSS_API mss_status mss_prop_save(const mss_prop* p, const char* path);
MSS_API mss_status mss_prop_load(mss_prop* p, const char* path);
MSS_API int64_t mss_prop_launch_count(const mss_prop* p);

/* ---- Base qualities ("Incorporating base qualities and position specific scoring matrix") ----
   A base of Phred quality Q (quality character Q + 33, '!'..'~') is right with probability
   x = 1 - 10^(-Q/10); matching it scores match * x and mismatching it mismatch * x / 3.  The
   scores are kept in fixed point: times scale (1..32), rounded to the nearest integer with
   halves away from zero, so results are in units of 1/scale.  A read N, or a genome N, scores
   the position's mismatch value.  d_quals: one quality character per read base, same offsets
   as d_reads (device memory).  The reverse strand's base k takes the quality of read base
   m - 1 - k. */
/* Phase one with those scores (int16 lanes; read step 1; default scan shape 8 lane pairs x 4
   query strands, other mss_tune shapes fail with MSS_EINVAL).  Errors as mss_map_reads_device,
   plus MSS_EINVAL for a null d_quals or a scale outside 1..32, MSS_EOVERFLOW when scale *
   match > 127, scale * mismatch < -384 (8-bit profile bytes) or max_len * round(scale * match)
   > 32767; a quality character outside '!'..'~' is reported by mss_sync (MSS_EINVAL). */
MSS_API mss_status mss_map_reads_quals_device(mss_ctx* ctx, const char* d_reads, const char* d_quals,
                                              const int64_t* d_offsets, int32_t R, int32_t max_len,
                                              const mss_score_params* sp, int32_t scale, mss_hit* d_out,
                                              void* stream);
/* Phase two with those scores: np->match / np->mismatch are weighted per read base, the gap
   costs multiplied by scale; the alignment score is in units of 1/scale.  Errors as
   nw_align_device, plus MSS_EINVAL for a null d_quals or a scale outside 1..32. */
MSS_API mss_status nw_align_quals_device(mss_ctx* ctx, const char* d_reads, const char* d_quals,
                                         const int64_t* d_offsets, int32_t R, int32_t max_len, const mss_hit* d_hits,
                                         const mss_nw_params* np, int32_t scale, mss_aln* d_out, char* d_cigars,
                                         int32_t cigar_stride, void* stream);

/* ---- SAM output ("Mapping qualities, read lengths, SAM output, and source code") ---- */
/* MAPQ of a phase-one result: -100 log2(second / best), the paper's probability of a wrong
   mapping being the ratio of the second-best to the best fragment score; rounded to the
   nearest integer, capped at 254; 254 when second_score == 0; 0 when best_score <= 0 or
   second_score >= best_score.  A read counts as mapped when MAPQ > 15.2, i.e. when the
   MSS_HIT_REPEAT flag is clear.  Pure function of its arguments. */
MSS_API int32_t mss_mapq(int32_t best_score, int32_t second_score);
/* SAM text (host memory only) for R reads: optional header (@HD, @SQ SN:ref_name LN:ref_len,
   @PG), then one line per read: QNAME r<index>, FLAG 0 / 16 (reverse strand) / 4 (unmapped:
   repeat-flagged in phase one or no in-band alignment in phase two), RNAME, POS =
   alns[r].gstart + 1, MAPQ (mss_mapq), CIGAR from cigars + r * cigar_stride (alns[r].cigar_len
   characters; '*' when cigars is NULL or the slot overflowed), RNEXT '*', PNEXT 0, TLEN 0,
   SEQ on the forward genome strand (reverse complement for strand 1, upper case), QUAL '*',
   tags AS:i (phase-two score, mapped reads), ZM:i (best fragment score), XS:i (second
   fragment score).  reads/offsets: the concatenated reads (offsets[R + 1]); hits/alns: the
   results of mss_map_reads / nw_align.  Returns the text length in bytes (without the NUL);
   the text and a NUL are written to out only when out != NULL and cap > length, so a call
   with out == NULL sizes the buffer.  Negative MSS_EINVAL for a null or empty ref_name (or
   one holding tabs, spaces or newlines), ref_len < 1, R < 0, missing arrays, a negative read
   length, or cigar_stride < 1 with cigars given.  Touches no GPU. */
MSS_API int64_t mss_format_sam(const char* ref_name, int64_t ref_len, const char* reads, const int64_t* offsets,
                               int32_t R, const mss_hit* hits, const mss_aln* alns, const char* cigars,
                               int32_t cigar_stride, int32_t header, char* out, int64_t cap);

MSS_API void mss_free(mss_ctx* ctx);
MSS_API const char* mss_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
