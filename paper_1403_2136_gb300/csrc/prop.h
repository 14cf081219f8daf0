// Host-side declarations of the learned-proposal kernels (prop.cu); not part of the ABI.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mss {

constexpr int kPropC = 128;    // channels and embedding width
constexpr int kPropTaps = 7;   // kernel width ("same" padding of 3)
constexpr int kPropLayers = 4;
// flat fp32 parameter vector: W1 [7][4][128], b1 [128], then for layers 2..4:
// W [7][128 ci][128 co], b [128]
constexpr int64_t kPropW1 = (int64_t)kPropTaps * 4 * kPropC;
constexpr int64_t kPropWl = (int64_t)kPropTaps * kPropC * kPropC;
constexpr int64_t kPropParams = kPropW1 + kPropC + 3 * (kPropWl + kPropC);
inline int64_t prop_off_b1() { return kPropW1; }
inline int64_t prop_off_w(int layer) { return kPropW1 + kPropC + (int64_t)(layer - 2) * (kPropWl + kPropC); }
inline int64_t prop_off_b(int layer) { return prop_off_w(layer) + kPropWl; }

// 2-D TMA tensor map over an activation buffer of nrows rows x 128 BF16 channels, boxes of
// box_ch channels x box_rows rows, 128-byte swizzle or none (conv_tc.cu).  cudaErrorInvalidValue
// for a base that is not 16-byte aligned or more than 2^31 - 1 rows.
cudaError_t prop_tensor_map_rows(CUtensorMap* map, const __nv_bfloat16* base, int64_t nrows, uint32_t box_ch,
                                 uint32_t box_rows, bool swizzle128);

// rows of an activation buffer for sequences of at most maxlen positions
inline int32_t prop_rows(int32_t maxlen) { return ((maxlen + 127) / 128) * 128 + 6; }

// zero the 3 halo rows on each side of every sequence of up to four activation buffers (null = skip)
cudaError_t prop_zero_halo(__nv_bfloat16* b0, __nv_bfloat16* b1, __nv_bfloat16* b2, __nv_bfloat16* b3, int32_t n,
                           int32_t rows, cudaStream_t s);
// first layer on the tensor cores (embed_tc.cu); err: device error word (bounded waits)
cudaError_t prop_embed_l1(const uint8_t* codes, const int32_t* lens, int32_t ld, int32_t n, const float* w1,
                          const float* b1, __nv_bfloat16* out, int32_t rows, int32_t* err, cudaStream_t s);
// 128 -> 128 conv on the tensor cores (conv_tc.cu).  wcanon: the layer's weights w[t][in][out]
// rearranged by prop_canon_weights (prop_canon_weight_bytes() bytes).  mode 0: out =
// relu(conv + bias) for p < len; mode 1 (backward data, flipped weights): out = conv where
// prev > 0.  err: device error word (a bounded wait that gives up sets ERR_TIMEOUT).
int64_t prop_canon_weight_bytes();
cudaError_t prop_canon_weights(const __nv_bfloat16* w, void* dst, cudaStream_t s);
cudaError_t prop_conv_tc(const __nv_bfloat16* in, const void* wcanon, const float* bias, const __nv_bfloat16* prev,
                         const int32_t* lens, __nv_bfloat16* out, int32_t n, int32_t rows, int mode, int32_t* err,
                         cudaStream_t s);
// Weight gradient of a 128 -> 128 layer, dw[t][ci][co] += sum over sequences and positions p
// of in[p + t - 3][ci] * g[p][co], and (db not null) its bias gradient db[co] += sum of
// g[p][co], on the fifth-generation tensor cores (wgrad_tc.cu); err: device error word (a
// bounded wait that gives up sets ERR_TIMEOUT).
cudaError_t prop_conv_wgrad_tc(const __nv_bfloat16* in, const __nv_bfloat16* g, const int32_t* lens, float* dw,
                               float* db, int32_t n, int32_t rows, int32_t* err, cudaStream_t s);
// first-layer weight and bias gradients on the tensor cores (wgrad_tc.cu); err: device error word
cudaError_t prop_l1_wgrad(const uint8_t* codes, const int32_t* lens, int32_t ld, const __nv_bfloat16* g, float* dw1,
                          float* db1, int32_t n, int32_t rows, int32_t* err, cudaStream_t s);
cudaError_t prop_pool_norm(const __nv_bfloat16* act, const int32_t* lens, int32_t n, int32_t rows, float* emb,
                           float* norms, int32_t* argmax, int32_t mean, cudaStream_t s);
cudaError_t prop_pool_norm_bwd(const float* emb, const float* demb, const float* norms, const int32_t* argmax,
                               const __nv_bfloat16* act, const int32_t* lens, int32_t n, int32_t rows,
                               __nv_bfloat16* g4, int32_t mean, cudaStream_t s);
cudaError_t prop_ce_loss(const float* r, const float* c, const int32_t* label, int32_t B, int32_t C, float inv_temp,
                         float* loss, float* dr, float* dc, float scale, cudaStream_t s);
cudaError_t prop_adamw(float* w, const float* g, float* m1, float* m2, __nv_bfloat16* wb, int64_t count, float lr,
                       float beta1, float beta2, float eps, float wd, float bc1, float bc2, cudaStream_t s);
cudaError_t prop_flip_weights(const __nv_bfloat16* w, __nv_bfloat16* wt, cudaStream_t s);
cudaError_t prop_scores(const float* er, int32_t R, const __nv_bfloat16* ef, int64_t NF, float* scores,
                        cudaStream_t s);
cudaError_t prop_topk(const float* scores, int32_t R, int64_t NF, int32_t K, int32_t* out_f, float* out_s,
                      cudaStream_t s);
// a9 on the tensor cores (score_tc.cu).  The fragment index is stored as BF16 tiles of 128
// fragments in the canonical K-major operand layout (tc.cuh); read embeddings are packed the
// same way in blocks of 128 sequences (forward, reverse complement of each read).
int64_t prop_index_bytes(int64_t NF);
int64_t prop_read_block_bytes(int32_t R);
cudaError_t prop_store_index(const float* emb, int64_t f0, int32_t nb, void* index, cudaStream_t s);
cudaError_t prop_pack_reads(const float* er, int32_t R, void* out, cudaStream_t s);
// fragment splits per block of 64 reads (at least one CTA per SM; S * K <= 256)
int32_t prop_score_splits(int32_t R, int64_t NF, int32_t K, int num_sms);
// per read the K <= 128 best fragments (score desc, fragment asc) into out_f / out_s [R][K];
// part_key / part_f: [S][R][K] workspace when S > 1
cudaError_t prop_score_topk(const void* breads, int32_t R, const void* index, int64_t NF, int32_t K, int32_t S,
                            int32_t* out_f, float* out_s, uint32_t* part_key, int32_t* part_f, int32_t* err,
                            cudaStream_t s);
// exact rescoring of K candidate fragments per read (rescore.cu): per-candidate maxima with the
// packed-lane scan, then the top-2 among the candidates and the best diagonal.  Reads longer
// than max_len set ERR_BAD_LEN in *err and are cut to max_len.
cudaError_t prop_rescore(const uint32_t* g2, const uint32_t* gm, int64_t F, const char* reads, const int64_t* offsets,
                         const int32_t* idx, int32_t R, int32_t max_len, const int32_t* cand, int32_t K,
                         int32_t match, int32_t mismatch, int32_t exclude_neighbors, void* hits,
                         int32_t* cand_scores, int32_t* err, int num_sms, cudaStream_t s);
// codes of reads (strand 0 forward, 1 reverse complement) and of genome windows
cudaError_t prop_read_codes(const char* reads, const int64_t* offsets, const int32_t* idx, const int8_t* strand,
                            int32_t n, int32_t ld, uint8_t* codes, int32_t* lens, cudaStream_t s);
cudaError_t prop_window_codes(const uint32_t* g2, const uint32_t* gm, const int64_t* starts, int32_t n, int32_t len,
                              int32_t ld, uint8_t* codes, int32_t* lens, cudaStream_t s);
cudaError_t prop_init_params(float* w, uint64_t seed, cudaStream_t s);
// fallback batch: reads sel[0..n) copied to out at new_off (n + 1 prefix offsets), and the
// batch's hits (mss_hit) written back to out[sel[j]]
cudaError_t prop_gather_reads(const char* reads, const int64_t* offsets, const int32_t* sel, int32_t n,
                              const int64_t* new_off, char* out, cudaStream_t s);
cudaError_t prop_scatter_hits(const void* sub, const int32_t* sel, int32_t n, void* out, cudaStream_t s);
cudaError_t prop_to_bf16(const float* w, __nv_bfloat16* wb, int64_t n, cudaStream_t s);

}  // namespace mss
