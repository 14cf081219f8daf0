// C ABI of the learned fragment proposal: model state, training step, fragment index,
// proposal-then-exact mapping with exhaustive fallback, checkpoints.  Argument checks and
// orchestration only; the compute is in prop.cu, rescore.cu and scan.cu.
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/maxss.h"
#include "internal.h"
#include "prop.h"

using namespace mss;

namespace {

struct Buf {  // a device buffer owned by its holder: freed by release() or when it goes out of scope
  void* p = nullptr;
  size_t cap = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { release(); }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max(bytes, (size_t)256));
    if (e == cudaSuccess) cap = std::max(bytes, (size_t)256);
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

#define PCK(expr, what)                                                  \
  do {                                                                   \
    cudaError_t _e = (expr);                                             \
    if (_e != cudaSuccess) return set_error(MSS_ECUDA, what);            \
  } while (0)

// activations of one forward pass (kept for the backward pass)
struct Acts {
  Buf act[4];  // bf16 [n][rows][128]
  Buf emb, norms, argmax;
  int32_t n = 0, rows = 0;
  cudaError_t ensure(int32_t nn, int32_t rr) {
    const size_t a = (size_t)nn * rr * kPropC * sizeof(__nv_bfloat16);
    for (auto& b : act) {
      cudaError_t e = b.ensure(a);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = emb.ensure((size_t)nn * kPropC * 4);
    if (e == cudaSuccess) e = norms.ensure((size_t)nn * 4);
    if (e == cudaSuccess) e = argmax.ensure((size_t)nn * kPropC * 4);
    n = nn;
    rows = rr;
    return e;
  }
};

}  // namespace

struct mss_prop {
  Buf w32, m1, m2, grad;            // fp32 master weights, Adam moments, gradient (flat)
  Buf wb[3], wflip[3];              // bf16 weights of layers 2..4 and their flipped copies
  Buf wct[3], wfct[3];              // the same as tensor-core B operands (conv_tc.cu layout)
  Buf err;                          // device error word of the proposal kernels
  Acts fa, fb;                      // forward activations (reads / candidates) for training
  Buf g[2];                         // gradient activations (ping-pong)
  Buf loss, de_r, de_c;
  Buf codes, lens, starts, idx, strand;
  Buf index;                        // bf16 [NF][128] fragment embeddings
  int64_t index_nf = 0, index_F = 0;
  int32_t index_window = 0;
  const void* index_genome = nullptr;
  Buf scores, cand, cand_s, cand_x, emb_reads, breads, part_key, part_f;
  int64_t step = 0;
  int64_t launches = 0;
  int32_t pooling = MSS_POOL_MAX;   // how a sequence's positions become one vector
};

namespace {

mss_status refresh_bf16(mss_prop* p, cudaStream_t s) {
  for (int l = 2; l <= 4; ++l) {
    PCK(prop_to_bf16(p->w32.as<float>() + prop_off_w(l), p->wb[l - 2].as<__nv_bfloat16>(), kPropWl, s), "bf16 copy");
    PCK(prop_flip_weights(p->wb[l - 2].as<__nv_bfloat16>(), p->wflip[l - 2].as<__nv_bfloat16>(), s), "flip");
    PCK(prop_canon_weights(p->wb[l - 2].as<__nv_bfloat16>(), p->wct[l - 2].p, s), "weight layout");
    PCK(prop_canon_weights(p->wflip[l - 2].as<__nv_bfloat16>(), p->wfct[l - 2].p, s), "weight layout");
    p->launches += 4;
  }
  return MSS_OK;
}

// forward pass of n sequences (codes [n][ld], lens[n]) into acts; embeddings in acts.emb
mss_status forward(mss_prop* p, const uint8_t* codes, const int32_t* lens, int32_t ld, int32_t n, int32_t maxlen,
                   Acts& a, cudaStream_t s) {
  const int32_t rows = prop_rows(maxlen);
  PCK(a.ensure(n, rows), "activation buffers");
  // every row but the halo is written by the layers below
  PCK(prop_zero_halo(a.act[0].as<__nv_bfloat16>(), a.act[1].as<__nv_bfloat16>(), a.act[2].as<__nv_bfloat16>(),
                     a.act[3].as<__nv_bfloat16>(), n, rows, s),
      "activation halo");
  const float* w = p->w32.as<float>();
  PCK(prop_embed_l1(codes, lens, ld, n, w, w + prop_off_b1(), a.act[0].as<__nv_bfloat16>(), rows,
                    p->err.as<int32_t>(), s),
      "layer 1");
  for (int l = 2; l <= 4; ++l)
    PCK(prop_conv_tc(a.act[l - 2].as<__nv_bfloat16>(), p->wct[l - 2].p, w + prop_off_b(l), nullptr, lens,
                     a.act[l - 1].as<__nv_bfloat16>(), n, rows, 0, p->err.as<int32_t>(), s),
        "conv layer");
  PCK(prop_pool_norm(a.act[3].as<__nv_bfloat16>(), lens, n, rows, a.emb.as<float>(), a.norms.as<float>(),
                     a.argmax.as<int32_t>(), p->pooling == MSS_POOL_MEAN, s),
      "pool");
  p->launches += 6;
  return MSS_OK;
}

// backward pass given d(emb) of the sequences of a; accumulates into p->grad
mss_status backward(mss_prop* p, const uint8_t* codes, const int32_t* lens, int32_t ld, Acts& a, const float* demb,
                    cudaStream_t s) {
  const int32_t n = a.n, rows = a.rows;
  const size_t abytes = (size_t)n * rows * kPropC * sizeof(__nv_bfloat16);
  PCK(p->g[0].ensure(abytes), "gradient buffers");
  PCK(p->g[1].ensure(abytes), "gradient buffers");
  PCK(cudaMemsetAsync(p->g[0].p, 0, abytes, s), "gradient clear");
  PCK(cudaMemsetAsync(p->g[1].p, 0, abytes, s), "gradient clear");
  float* gw = p->grad.as<float>();
  __nv_bfloat16* gcur = p->g[0].as<__nv_bfloat16>();
  __nv_bfloat16* gnext = p->g[1].as<__nv_bfloat16>();
  PCK(prop_pool_norm_bwd(a.emb.as<float>(), demb, a.norms.as<float>(), a.argmax.as<int32_t>(),
                         a.act[3].as<__nv_bfloat16>(), lens, n, rows, gcur, p->pooling == MSS_POOL_MEAN, s),
      "pool backward");
  p->launches += 1;
  for (int l = 4; l >= 2; --l) {
    // gcur = gradient of layer l's pre-activation; input activation of layer l is act[l - 2]
    PCK(prop_conv_wgrad_tc(a.act[l - 2].as<__nv_bfloat16>(), gcur, lens, gw + prop_off_w(l), gw + prop_off_b(l), n,
                           rows, p->err.as<int32_t>(), s),
        "weight and bias gradients");
    PCK(prop_conv_tc(gcur, p->wfct[l - 2].p, nullptr, a.act[l - 2].as<__nv_bfloat16>(), lens, gnext, n, rows, 1,
                     p->err.as<int32_t>(), s),
        "conv backward");
    std::swap(gcur, gnext);
    p->launches += 2;
  }
  PCK(prop_l1_wgrad(codes, lens, ld, gcur, gw, gw + prop_off_b1(), n, rows, p->err.as<int32_t>(), s), "layer 1 grad");
  p->launches += 1;
  return MSS_OK;
}

// Synchronize and read (then clear) the proposal kernels' error word.
mss_status read_prop_err(mss_prop* p, cudaStream_t s) {
  int32_t h = 0;
  PCK(cudaStreamSynchronize(s), "sync");
  PCK(cudaMemcpy(&h, p->err.p, sizeof(int32_t), cudaMemcpyDeviceToHost), "error word read");
  if (h == 0) return MSS_OK;
  PCK(cudaMemset(p->err.p, 0, sizeof(int32_t)), "error word clear");
  return set_error(MSS_ETIMEOUT, "a bounded wait of a tensor-core kernel gave up");
}

mss_status check_prop(const mss_prop* p) {
  if (!p) return set_error(MSS_EINVAL, "null proposal model");
  return MSS_OK;
}

// CRC-32 (IEEE polynomial, bitwise) of a byte range, for the checkpoint header
uint32_t crc32_bytes(const void* data, size_t n, uint32_t crc = 0xFFFFFFFFu) {
  const uint8_t* b = static_cast<const uint8_t*>(data);
  for (size_t i = 0; i < n; ++i) {
    crc ^= b[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return crc;
}

}  // namespace

extern "C" {

mss_status mss_prop_create(mss_prop** out, uint64_t seed, void* stream) {
  if (!out) return set_error(MSS_EINVAL, "null output");
  *out = nullptr;
  mss_prop* p = new (std::nothrow) mss_prop();
  if (!p) return set_error(MSS_ENOMEM, "proposal model");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t pb = (size_t)kPropParams * 4;
  cudaError_t e = p->w32.ensure(pb);
  if (e == cudaSuccess) e = p->m1.ensure(pb);
  if (e == cudaSuccess) e = p->m2.ensure(pb);
  if (e == cudaSuccess) e = p->grad.ensure(pb);
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = p->wb[l].ensure((size_t)kPropWl * 2);
    if (e == cudaSuccess) e = p->wflip[l].ensure((size_t)kPropWl * 2);
    if (e == cudaSuccess) e = p->wct[l].ensure((size_t)prop_canon_weight_bytes());
    if (e == cudaSuccess) e = p->wfct[l].ensure((size_t)prop_canon_weight_bytes());
  }
  if (e == cudaSuccess) e = p->err.ensure(sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(p->err.p, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->m1.p, 0, pb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->m2.p, 0, pb, s);
  if (e == cudaSuccess) e = prop_init_params(p->w32.as<float>(), seed, s);
  if (e != cudaSuccess) {
    mss_prop_free(p);
    return set_error(e == cudaErrorMemoryAllocation ? MSS_ENOMEM : MSS_ECUDA, cudaGetErrorString(e));
  }
  p->launches += 1;
  mss_status st = refresh_bf16(p, s);
  if (st) {
    mss_prop_free(p);
    return st;
  }
  *out = p;
  return MSS_OK;
}

void mss_prop_free(mss_prop* p) {
  if (!p) return;
  for (Buf* b : {&p->w32, &p->m1, &p->m2, &p->grad, &p->loss, &p->de_r, &p->de_c, &p->codes, &p->lens, &p->starts,
                 &p->idx, &p->strand, &p->index, &p->scores, &p->cand, &p->cand_s, &p->emb_reads, &p->g[0], &p->g[1],
                 &p->cand_x, &p->breads, &p->part_key, &p->part_f, &p->err})
    b->release();
  for (int l = 0; l < 3; ++l) {
    p->wb[l].release();
    p->wflip[l].release();
    p->wct[l].release();
    p->wfct[l].release();
  }
  for (Acts* a : {&p->fa, &p->fb}) {
    for (auto& b : a->act) b.release();
    a->emb.release();
    a->norms.release();
    a->argmax.release();
  }
  delete p;
}

mss_status mss_prop_get_params(const mss_prop* p, float* host, int64_t n) {
  if (check_prop(p) || !host) return set_error(MSS_EINVAL, "null argument");
  if (n != kPropParams) return set_error(MSS_EINVAL, "parameter count mismatch");
  PCK(cudaMemcpy(host, p->w32.p, (size_t)n * 4, cudaMemcpyDeviceToHost), "parameter read");
  return MSS_OK;
}

mss_status mss_prop_set_params(mss_prop* p, const float* host, int64_t n) {
  if (check_prop(p) || !host) return set_error(MSS_EINVAL, "null argument");
  if (n != kPropParams) return set_error(MSS_EINVAL, "parameter count mismatch");
  PCK(cudaMemcpy(p->w32.p, host, (size_t)n * 4, cudaMemcpyHostToDevice), "parameter write");
  return refresh_bf16(p, nullptr);
}

int64_t mss_prop_param_count(void) { return kPropParams; }

mss_status mss_prop_set_pooling(mss_prop* p, int32_t pooling) {
  if (check_prop(p)) return set_error(MSS_EINVAL, "null proposal model");
  if (pooling != MSS_POOL_MAX && pooling != MSS_POOL_MEAN) return set_error(MSS_EINVAL, "unknown pooling");
  p->pooling = pooling;
  return MSS_OK;
}

int32_t mss_prop_get_pooling(const mss_prop* p) { return p ? p->pooling : -1; }

mss_status mss_prop_embed_device(mss_prop* p, const uint8_t* d_codes, const int32_t* d_lens, int32_t ld, int32_t n,
                                 int32_t maxlen, float* d_emb, void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  if (n < 0 || ld < 1 || maxlen < 1 || maxlen > ld) return set_error(MSS_EINVAL, "bad sizes");
  if (n == 0) return MSS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  mss_status st = forward(p, d_codes, d_lens, ld, n, maxlen, p->fa, s);
  if (st) return st;
  PCK(cudaMemcpyAsync(d_emb, p->fa.emb.p, (size_t)n * kPropC * 4, cudaMemcpyDeviceToDevice, s), "embedding copy");
  return MSS_OK;
}

mss_status mss_prop_grad_device(mss_prop* p, const uint8_t* d_codes, const int32_t* d_lens, int32_t ld, int32_t n,
                                int32_t maxlen, const float* d_demb, float* d_grad, void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  if (n < 1 || ld < 1 || maxlen < 1 || maxlen > ld) return set_error(MSS_EINVAL, "bad sizes");
  cudaStream_t s = (cudaStream_t)stream;
  PCK(cudaMemsetAsync(p->grad.p, 0, (size_t)kPropParams * 4, s), "gradient clear");
  mss_status st = forward(p, d_codes, d_lens, ld, n, maxlen, p->fa, s);
  if (st) return st;
  st = backward(p, d_codes, d_lens, ld, p->fa, d_demb, s);
  if (st) return st;
  PCK(cudaMemcpyAsync(d_grad, p->grad.p, (size_t)kPropParams * 4, cudaMemcpyDeviceToDevice, s), "gradient copy");
  return MSS_OK;
}

mss_status mss_prop_train_step(mss_prop* p, const uint8_t* d_rcodes, const int32_t* d_rlens, int32_t ld_r, int32_t B,
                               int32_t maxlen_r, const uint8_t* d_ccodes, const int32_t* d_clens, int32_t ld_c,
                               int32_t C, int32_t maxlen_c, const int32_t* d_labels, float lr, float temperature,
                               float weight_decay, float* loss_out, void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  if (B < 1 || C < 2 || C > 1024 || maxlen_r < 1 || maxlen_c < 1 || maxlen_r > ld_r || maxlen_c > ld_c)
    return set_error(MSS_EINVAL, "bad batch sizes (B >= 1, 2 <= C <= 1024)");
  if (!(temperature > 0.f) || !(lr > 0.f)) return set_error(MSS_EINVAL, "temperature and lr must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  PCK(cudaMemsetAsync(p->grad.p, 0, (size_t)kPropParams * 4, s), "gradient clear");
  mss_status st = forward(p, d_rcodes, d_rlens, ld_r, B, maxlen_r, p->fa, s);
  if (!st) st = forward(p, d_ccodes, d_clens, ld_c, C, maxlen_c, p->fb, s);
  if (st) return st;
  PCK(p->loss.ensure((size_t)B * 4), "loss");
  PCK(p->de_r.ensure((size_t)B * kPropC * 4), "grad");
  PCK(p->de_c.ensure((size_t)C * kPropC * 4), "grad");
  PCK(cudaMemsetAsync(p->de_c.p, 0, (size_t)C * kPropC * 4, s), "grad clear");
  PCK(prop_ce_loss(p->fa.emb.as<float>(), p->fb.emb.as<float>(), d_labels, B, C, 1.f / temperature,
                   p->loss.as<float>(), p->de_r.as<float>(), p->de_c.as<float>(), 1.f / B, s),
      "loss");
  p->launches += 1;
  st = backward(p, d_rcodes, d_rlens, ld_r, p->fa, p->de_r.as<float>(), s);
  if (!st) st = backward(p, d_ccodes, d_clens, ld_c, p->fb, p->de_c.as<float>(), s);
  if (st) return st;
  p->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)p->step), bc2 = 1.f - powf(b2, (float)p->step);
  PCK(prop_adamw(p->w32.as<float>(), p->grad.as<float>(), p->m1.as<float>(), p->m2.as<float>(), nullptr, kPropParams,
                 lr, b1, b2, 1e-8f, weight_decay, bc1, bc2, s),
      "adamw");
  p->launches += 1;
  st = refresh_bf16(p, s);
  if (st) return st;
  if (loss_out) {
    std::vector<float> h(B);
    PCK(cudaMemcpyAsync(h.data(), p->loss.p, (size_t)B * 4, cudaMemcpyDeviceToHost, s), "loss read");
    st = read_prop_err(p, s);
    if (st) return st;
    double sum = 0;
    for (float v : h) sum += v;
    *loss_out = (float)(sum / B);
  }
  return MSS_OK;
}

mss_status mss_prop_build_index(mss_prop* p, mss_ctx* ctx, int32_t max_read_len, void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  CtxView v;
  if (!ctx_view(ctx, &v)) return set_error(MSS_EINVAL, "null context");
  mss_genome_info gi;
  if (mss_get_info(ctx, &gi)) return MSS_EINVAL;
  if (max_read_len < 1 || max_read_len > v.max_len) return set_error(MSS_EREADLEN, "max_read_len out of range");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t NF = gi.num_frags, F = gi.frag_len;
  const int32_t win = (int32_t)(F + max_read_len - 1);
  if (win > 65536) return set_error(MSS_EINVAL, "fragment window above 65536 bases");
  PCK(p->index.ensure((size_t)prop_index_bytes(NF)), "index");
  PCK(cudaMemsetAsync(p->index.p, 0, (size_t)prop_index_bytes(NF), s), "index clear");
  // batches of fragments bounded by ~1 GB of activations
  const int32_t rows = prop_rows(win);
  int32_t batch = (int32_t)std::max<int64_t>(1, (int64_t)(1u << 30) / ((int64_t)rows * kPropC * 2 * 4));
  batch = (int32_t)std::min<int64_t>(batch, NF);
  PCK(p->codes.ensure((size_t)batch * win), "codes");
  PCK(p->lens.ensure((size_t)batch * 4), "lens");
  PCK(p->starts.ensure((size_t)batch * 8), "starts");
  std::vector<int64_t> hs(batch);
  Buf tmp;
  PCK(tmp.ensure((size_t)batch * kPropC * 4), "tmp");
  for (int64_t f0 = 0; f0 < NF; f0 += batch) {
    const int32_t nb = (int32_t)std::min<int64_t>(batch, NF - f0);
    for (int32_t i = 0; i < nb; ++i) hs[i] = (f0 + i) * F;
    PCK(cudaMemcpyAsync(p->starts.p, hs.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, s), "starts");
    PCK(prop_window_codes(v.g2, v.gm, p->starts.as<int64_t>(), nb, win, win, p->codes.as<uint8_t>(),
                          p->lens.as<int32_t>(), s),
        "window codes");
    mss_status st = forward(p, p->codes.as<uint8_t>(), p->lens.as<int32_t>(), win, nb, win, p->fa, s);
    if (st) {
      tmp.release();
      return st;
    }
    PCK(prop_store_index(p->fa.emb.as<float>(), f0, nb, p->index.p, s), "index store");
    PCK(cudaStreamSynchronize(s), "sync");  // hs is reused
    p->launches += 2;
  }
  tmp.release();
  {
    mss_status est = read_prop_err(p, s);
    if (est) return est;
  }
  p->index_nf = NF;
  p->index_F = F;
  p->index_window = win;
  p->index_genome = v.g2;
  return MSS_OK;
}

mss_status mss_map_reads_proposed(mss_ctx* ctx, mss_prop* p, const char* d_reads, const int64_t* d_offsets, int32_t R,
                                  int32_t max_len, const mss_score_params* sp, int32_t K, float tau, mss_hit* d_out,
                                  int32_t* d_cand, float* d_top_score, int32_t* n_fallback, void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  CtxView v;
  if (!ctx_view(ctx, &v)) return set_error(MSS_EINVAL, "null context");
  if (!p->index.p || p->index_genome != v.g2) return set_error(MSS_ESTATE, "fragment index not built for this genome");
  mss_genome_info gi;
  if (mss_get_info(ctx, &gi)) return MSS_EINVAL;
  if (gi.frag_len != p->index_F) return set_error(MSS_ESTATE, "fragment length changed since the index was built");
  if (!sp || sp->match < 1 || sp->match > 127 || sp->mismatch < -128 || sp->mismatch > 0)
    return set_error(MSS_EINVAL, "bad score parameters");
  if (K < 1 || K > 1024) return set_error(MSS_EINVAL, "K outside [1, 1024]");
  if (max_len < 1 || max_len > v.max_len) return set_error(MSS_EREADLEN, "max_len out of range");
  if (R < 0) return set_error(MSS_EINVAL, "R < 0");
  if (n_fallback) *n_fallback = 0;
  if (R == 0) return MSS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t NF = p->index_nf;
  // read embeddings, both strands: sequence 2i = forward, 2i + 1 = reverse complement
  const int32_t nseq = 2 * R;
  PCK(p->codes.ensure((size_t)nseq * max_len), "codes");
  PCK(p->lens.ensure((size_t)nseq * 4), "lens");
  PCK(p->idx.ensure((size_t)nseq * 4), "idx");
  PCK(p->strand.ensure((size_t)nseq), "strand");
  {
    std::vector<int32_t> hi(nseq);
    std::vector<int8_t> hsg(nseq);
    for (int32_t i = 0; i < nseq; ++i) {
      hi[i] = i >> 1;
      hsg[i] = (int8_t)(i & 1);
    }
    PCK(cudaMemcpyAsync(p->idx.p, hi.data(), (size_t)nseq * 4, cudaMemcpyHostToDevice, s), "idx");
    PCK(cudaMemcpyAsync(p->strand.p, hsg.data(), (size_t)nseq, cudaMemcpyHostToDevice, s), "strand");
    PCK(prop_read_codes(d_reads, d_offsets, p->idx.as<int32_t>(), p->strand.as<int8_t>(), nseq, max_len,
                        p->codes.as<uint8_t>(), p->lens.as<int32_t>(), s),
        "read codes");
    PCK(cudaStreamSynchronize(s), "sync");
  }
  PCK(p->emb_reads.ensure((size_t)nseq * kPropC * 4), "embeddings");
  // embed in batches of at most 16384 sequences (about 1 GB per activation buffer at 250 bases)
  for (int32_t a = 0; a < nseq; a += 16384) {
    const int32_t nb = std::min(16384, nseq - a);
    mss_status st = forward(p, p->codes.as<uint8_t>() + (size_t)a * max_len, p->lens.as<int32_t>() + a, max_len, nb,
                            max_len, p->fa, s);
    if (st) return st;
    PCK(cudaMemcpyAsync(p->emb_reads.as<float>() + (size_t)a * kPropC, p->fa.emb.p, (size_t)nb * kPropC * 4,
                        cudaMemcpyDeviceToDevice, s),
        "embedding copy");
  }
  PCK(p->cand.ensure((size_t)R * K * 4), "candidates");
  PCK(p->cand_s.ensure((size_t)R * K * 4), "candidate scores");
  if (K <= 128) {
    // tensor cores: scores and the streaming top K fused, nothing of size R x NF stored
    PCK(p->breads.ensure((size_t)prop_read_block_bytes(R)), "read blocks");
    PCK(prop_pack_reads(p->emb_reads.as<float>(), R, p->breads.p, s), "read pack");
    const int32_t S = prop_score_splits(R, NF, K, v.num_sms);
    if (S > 1) {
      PCK(p->part_key.ensure((size_t)S * R * K * 4), "split lists");
      PCK(p->part_f.ensure((size_t)S * R * K * 4), "split lists");
    }
    PCK(prop_score_topk(p->breads.p, R, p->index.p, NF, K, S, p->cand.as<int32_t>(), p->cand_s.as<float>(),
                        p->part_key.as<uint32_t>(), p->part_f.as<int32_t>(), v.d_err, s),
        "scores and top K");
    p->launches += S > 1 ? 3 : 2;
  } else {
    // CUDA cores: scores in read batches bounded by ~2 GB, then a radix top K
    int32_t rb = (int32_t)std::max<int64_t>(1, std::min<int64_t>(R, (int64_t)(2ll << 30) / (NF * 4)));
    PCK(p->scores.ensure((size_t)rb * NF * 4), "scores");
    for (int32_t a = 0; a < R; a += rb) {
      const int32_t nb = std::min(rb, R - a);
      PCK(prop_scores(p->emb_reads.as<float>() + (size_t)a * 2 * kPropC, nb, p->index.as<__nv_bfloat16>(), NF,
                      p->scores.as<float>(), s),
          "scores");
      PCK(prop_topk(p->scores.as<float>(), nb, NF, K, p->cand.as<int32_t>() + (size_t)a * K,
                    p->cand_s.as<float>() + (size_t)a * K, s),
          "top K");
      p->launches += 2;
    }
  }
  // exact rescoring of the candidates
  PCK(p->cand_x.ensure((size_t)R * K * 4), "candidate maxima");
  PCK(prop_rescore(v.g2, v.gm, p->index_F, d_reads, d_offsets, nullptr, R, max_len, p->cand.as<int32_t>(), K,
                   sp->match, sp->mismatch, v.exclude_neighbors, d_out, p->cand_x.as<int32_t>(), v.d_err,
                   v.num_sms, s),
      "rescore");
  p->launches += 2;
  if (d_cand) PCK(cudaMemcpyAsync(d_cand, p->cand.p, (size_t)R * K * 4, cudaMemcpyDeviceToDevice, s), "cand copy");
  // fallback: reads whose best proposal score is below tau get the exhaustive scan
  std::vector<float> top((size_t)R * K);
  PCK(cudaMemcpyAsync(top.data(), p->cand_s.p, (size_t)R * K * 4, cudaMemcpyDeviceToHost, s), "scores read");
  {
    mss_status est = mss_sync(ctx, stream);  // synchronizes; reports bad characters / lengths
    if (!est) est = read_prop_err(p, s);
    if (est) return est;
  }
  if (d_top_score) {
    std::vector<float> t1(R);
    for (int32_t i = 0; i < R; ++i) t1[i] = top[(size_t)i * K];
    PCK(cudaMemcpyAsync(d_top_score, t1.data(), (size_t)R * 4, cudaMemcpyHostToDevice, s), "top score");
    PCK(cudaStreamSynchronize(s), "top score");   // t1 lives on this stack frame
  }
  std::vector<int32_t> fb;
  for (int32_t i = 0; i < R; ++i)
    if (top[(size_t)i * K] < tau) fb.push_back(i);
  if (n_fallback) *n_fallback = (int32_t)fb.size();
  if (fb.empty()) return MSS_OK;
  // gather the fallback reads into a compact batch, map them exhaustively, scatter the hits
  std::vector<int64_t> hoff(R + 1);
  PCK(cudaMemcpyAsync(hoff.data(), d_offsets, (size_t)(R + 1) * 8, cudaMemcpyDeviceToHost, s), "offsets read");
  PCK(cudaStreamSynchronize(s), "offsets read");
  std::vector<int64_t> noff(fb.size() + 1, 0);
  for (size_t j = 0; j < fb.size(); ++j) noff[j + 1] = noff[j] + (hoff[fb[j] + 1] - hoff[fb[j]]);
  const int32_t nfb = (int32_t)fb.size();
  Buf sub_reads, sub_off, sub_hits, sel;
  PCK(sub_reads.ensure((size_t)noff.back() + 16), "fallback reads");
  PCK(sub_off.ensure(noff.size() * 8), "fallback offsets");
  PCK(sub_hits.ensure(fb.size() * sizeof(mss_hit)), "fallback hits");
  PCK(sel.ensure(fb.size() * 4), "fallback reads");
  PCK(cudaMemcpyAsync(sub_off.p, noff.data(), noff.size() * 8, cudaMemcpyHostToDevice, s), "fallback offsets");
  PCK(cudaMemcpyAsync(sel.p, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice, s), "fallback reads");
  PCK(prop_gather_reads(d_reads, d_offsets, sel.as<int32_t>(), nfb, sub_off.as<int64_t>(), sub_reads.as<char>(), s),
      "gather");
  p->launches += 1;
  mss_status st = mss_map_reads_device(ctx, sub_reads.as<char>(), sub_off.as<int64_t>(), nfb, max_len, sp,
                                       sub_hits.as<mss_hit>(), stream);
  if (!st) st = mss_sync(ctx, stream);
  if (!st && prop_scatter_hits(sub_hits.p, sel.as<int32_t>(), nfb, d_out, s) != cudaSuccess)
    st = set_error(MSS_ECUDA, "scatter");
  if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = set_error(MSS_ECUDA, "sync");
  if (!st) p->launches += 1;
  sel.release();
  sub_reads.release();
  sub_off.release();
  sub_hits.release();
  return st;
}

mss_status mss_prop_read_codes(mss_prop* p, const char* d_reads, const int64_t* d_offsets, const int32_t* d_idx,
                               const int8_t* d_strand, int32_t n, int32_t ld, uint8_t* d_codes, int32_t* d_lens,
                               void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  if (n < 0 || ld < 1) return set_error(MSS_EINVAL, "bad sizes");
  PCK(prop_read_codes(d_reads, d_offsets, d_idx, d_strand, n, ld, d_codes, d_lens, (cudaStream_t)stream), "codes");
  p->launches += 1;
  return MSS_OK;
}

mss_status mss_prop_window_codes(mss_prop* p, const mss_ctx* ctx, const int64_t* d_starts, int32_t n, int32_t len,
                                 int32_t ld, uint8_t* d_codes, int32_t* d_lens, void* stream) {
  if (check_prop(p)) return MSS_EINVAL;
  CtxView v;
  if (!ctx_view(const_cast<mss_ctx*>(ctx), &v)) return set_error(MSS_EINVAL, "null context");
  if (n < 0 || len < 1 || len > ld) return set_error(MSS_EINVAL, "bad sizes");
  PCK(prop_window_codes(v.g2, v.gm, d_starts, n, len, ld, d_codes, d_lens, (cudaStream_t)stream), "codes");
  p->launches += 1;
  return MSS_OK;
}

int64_t mss_prop_launch_count(const mss_prop* p) { return p ? p->launches : -1; }

// checkpoint: "MSSPROP2", param count, step, pooling, then master weights, Adam moments;
// CRC-32 of all.  "MSSPROP1" files (no pooling field: max pooling) are still read.
mss_status mss_prop_save(const mss_prop* p, const char* path) {
  if (check_prop(p) || !path) return set_error(MSS_EINVAL, "null argument");
  std::vector<float> buf((size_t)kPropParams * 3);
  PCK(cudaMemcpy(buf.data(), p->w32.p, (size_t)kPropParams * 4, cudaMemcpyDeviceToHost), "read");
  PCK(cudaMemcpy(buf.data() + kPropParams, p->m1.p, (size_t)kPropParams * 4, cudaMemcpyDeviceToHost), "read");
  PCK(cudaMemcpy(buf.data() + 2 * kPropParams, p->m2.p, (size_t)kPropParams * 4, cudaMemcpyDeviceToHost), "read");
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(MSS_EINVAL, "cannot open checkpoint for writing");
  const char magic[8] = {'M', 'S', 'S', 'P', 'R', 'O', 'P', '2'};
  const int64_t hdr[3] = {kPropParams, p->step, (int64_t)p->pooling};
  uint32_t crc = crc32_bytes(hdr, sizeof(hdr));
  crc = crc32_bytes(buf.data(), buf.size() * 4, crc);
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(buf.data(), 4, buf.size(), f) == buf.size() && fwrite(&crc, 4, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok ? MSS_OK : set_error(MSS_EINVAL, "checkpoint write failed");
}

mss_status mss_prop_load(mss_prop* p, const char* path) {
  if (check_prop(p) || !path) return set_error(MSS_EINVAL, "null argument");
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(MSS_EINVAL, "cannot open checkpoint");
  char magic[8];
  int64_t hdr[3] = {0, 0, MSS_POOL_MAX};
  std::vector<float> buf((size_t)kPropParams * 3);
  uint32_t crc_file = 0;
  bool ok = fread(magic, 1, 8, f) == 8;
  const bool v1 = ok && memcmp(magic, "MSSPROP1", 8) == 0, v2 = ok && memcmp(magic, "MSSPROP2", 8) == 0;
  const size_t nh = v1 ? 2 : 3;
  ok = (v1 || v2) && fread(hdr, sizeof(int64_t), nh, f) == nh && hdr[0] == kPropParams &&
       (hdr[2] == MSS_POOL_MAX || hdr[2] == MSS_POOL_MEAN) && fread(buf.data(), 4, buf.size(), f) == buf.size() &&
       fread(&crc_file, 4, 1, f) == 1;
  fclose(f);
  if (!ok) return set_error(MSS_EINVAL, "not a proposal checkpoint (header, size or truncation)");
  uint32_t crc = crc32_bytes(hdr, nh * sizeof(int64_t));
  crc = crc32_bytes(buf.data(), buf.size() * 4, crc);
  if (crc != crc_file) return set_error(MSS_EINVAL, "checkpoint CRC mismatch");
  PCK(cudaMemcpy(p->w32.p, buf.data(), (size_t)kPropParams * 4, cudaMemcpyHostToDevice), "write");
  PCK(cudaMemcpy(p->m1.p, buf.data() + kPropParams, (size_t)kPropParams * 4, cudaMemcpyHostToDevice), "write");
  PCK(cudaMemcpy(p->m2.p, buf.data() + 2 * kPropParams, (size_t)kPropParams * 4, cudaMemcpyHostToDevice), "write");
  p->step = hdr[1];
  p->pooling = (int32_t)hdr[2];
  return refresh_bf16(p, nullptr);
}

}  // extern "C"
