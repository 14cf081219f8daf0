// Learned fragment proposal (a step added to the method, not in the paper): a small 1-D CNN
// embeds reads and genome fragments into 128-d unit vectors; the dot product ranks fragments
// per read so that the exact scan runs only on the top K.
//
// Network: one-hot bases (N = all zero) -> 4 x [conv1d k=7 "same", 128 channels, bias, ReLU]
// -> pool over positions (maximum, or mean as an option) -> L2 normalisation.  Weights BF16,
// accumulation FP32.
//
// Kernels here (the 128 -> 128 conv itself, forward and backward-data, runs on the
// fifth-generation tensor cores in conv_tc.cu, the weight and bias gradients of all layers in
// wgrad_tc.cu, the first layer in embed_tc.cu, the read x fragment score GEMM with its fused top K in score_tc.cu):
//   k_pool_norm     max (first argmax kept) or mean over positions, L2 norm
//   k_pool_norm_bwd gradient of the norm routed to the argmax positions (max) or spread
//                   over the positions with weight 1 / length (mean)
//   k_ce_loss       softmax cross-entropy of read-vs-candidate logits and its gradients
//   k_adamw         AdamW on FP32 master weights, refreshing the BF16 copies
//   k_scores        read x fragment scores (max over the read's two strands)
//   k_topk          per-read top K (ties -> lower fragment), by 4-round radix select
// (the exact rescoring of the candidates is in rescore.cu)
#include <cuda_bf16.h>

#include "../../include/maxss.h"
#include "common.cuh"
#include "internal.h"
#include "prop.h"
#include "tc.cuh"

namespace mss {

// zero the three halo rows on each side of every sequence of up to four activation buffers
// (the layers write every other row)
__global__ void k_zero_halo(__nv_bfloat16* b0, __nv_bfloat16* b1, __nv_bfloat16* b2, __nv_bfloat16* b3, int32_t n,
                            int32_t rows) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (sequence, halo row, 16-byte chunk)
  if (e >= (int64_t)n * 6 * 16) return;
  const int64_t seq = e / 96;
  const int r = (int)(e % 96) >> 4, c = (int)(e & 15);
  const int row = r < 3 ? r : rows - 6 + r;
  const int64_t off = (seq * rows + row) * kPropC + 8 * c;
  __nv_bfloat16* bs[4] = {b0, b1, b2, b3};
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (bs[i]) *reinterpret_cast<uint4*>(bs[i] + off) = make_uint4(0, 0, 0, 0);
}

// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// pool over the positions p < len of each channel, then the L2 norm.  CTA = one sequence,
// 256 threads = 16 position lanes x 16 groups of 8 channels.  Max: the lanes' maxima merge
// with ties going to the lower position, so the result is the first maximum.  Mean: the
// lanes' FP32 sums add in lane order and the total is divided by len.
__global__ void __launch_bounds__(256) k_pool_norm(const __nv_bfloat16* __restrict__ act,
                                                   const int32_t* __restrict__ lens, int32_t rows,
                                                   float* __restrict__ emb, float* __restrict__ norms,
                                                   int32_t* __restrict__ argmax, int32_t mean) {
  const int n = blockIdx.x, tid = threadIdx.x;
  const int g = tid & 15, pl = tid >> 4;
  const int len = lens[n];
  float best[8];
  int bi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) best[j] = mean ? 0.f : -1.f, bi[j] = 0;
  const __nv_bfloat16* an = act + ((int64_t)n * rows + 3) * kPropC + 8 * g;
  if (mean) {
#pragma unroll 4
    for (int p = pl; p < len; p += 16) {
      const uint4 u = *reinterpret_cast<const uint4*>(an + (int64_t)p * kPropC);
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[j]);
        best[2 * j] += __bfloat162float(h.x);
        best[2 * j + 1] += __bfloat162float(h.y);
      }
    }
  } else {
#pragma unroll 4
    for (int p = pl; p < len; p += 16) {
      const uint4 u = *reinterpret_cast<const uint4*>(an + (int64_t)p * kPropC);
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[j]);
        const float v0 = __bfloat162float(h.x), v1 = __bfloat162float(h.y);
        if (v0 > best[2 * j]) best[2 * j] = v0, bi[2 * j] = p;
        if (v1 > best[2 * j + 1]) best[2 * j + 1] = v1, bi[2 * j + 1] = p;
      }
    }
  }
  __shared__ float s_best[16][kPropC];
  __shared__ int s_bi[16][kPropC];
#pragma unroll
  for (int j = 0; j < 8; ++j) s_best[pl][8 * g + j] = best[j], s_bi[pl][8 * g + j] = bi[j];
  __syncthreads();
  if (tid >= kPropC) return;
  const int co = tid;
  float b = -1.f;
  int bp = 0;
  if (mean) {
    b = 0.f;
    for (int l = 0; l < 16; ++l) b += s_best[l][co];
    if (len > 0) b /= (float)len;
  } else {
    for (int l = 0; l < 16; ++l) {
      const float v = s_best[l][co];
      const int q = s_bi[l][co];
      if (v > b || (v == b && v >= 0.f && q < bp)) b = v, bp = q;
    }
  }
  if (len <= 0) b = 0.f, bp = 0;
  __shared__ float red[4];
  float sq = b * b;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s);
  if ((co & 31) == 0) red[co >> 5] = sq;
  asm volatile("bar.sync 1, 128;" ::: "memory");
  const float nrm = sqrtf(red[0] + red[1] + red[2] + red[3]) + 1e-6f;
  emb[n * kPropC + co] = b / nrm;
  if (argmax) argmax[n * kPropC + co] = bp;
  if (norms && co == 0) norms[n] = nrm;
}

// gradient through the L2 norm and the pool, masked by the last ReLU (g4 holds zeros on
// entry): max, g4[n][argmax + 3][co] = de_raw where act > 0; mean, g4[n][p + 3][co] =
// de_raw / len at every p < len where act > 0
__global__ void k_pool_norm_bwd(const float* __restrict__ emb, const float* __restrict__ demb,
                                const float* __restrict__ norms, const int32_t* __restrict__ argmax,
                                const __nv_bfloat16* __restrict__ act, const int32_t* __restrict__ lens, int32_t rows,
                                __nv_bfloat16* __restrict__ g4, int32_t mean) {
  const int n = blockIdx.x, co = threadIdx.x;
  __shared__ float red[4];
  const float e = emb[n * kPropC + co], de = demb[n * kPropC + co];
  float dot = e * de;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, s);
  if ((co & 31) == 0) red[co >> 5] = dot;
  __syncthreads();
  dot = red[0] + red[1] + red[2] + red[3];
  const float draw = (de - e * dot) / norms[n];
  const int len = lens[n];
  if (len <= 0) return;
  if (mean) {
    const __nv_bfloat16 gv = __float2bfloat16(draw / (float)len);
    for (int p = 0; p < len; ++p) {
      const int64_t o = ((int64_t)n * rows + p + 3) * kPropC + co;
      if (__bfloat162float(act[o]) > 0.f) g4[o] = gv;
    }
    return;
  }
  const int p = argmax[n * kPropC + co];
  const int64_t o = ((int64_t)n * rows + p + 3) * kPropC + co;
  if (__bfloat162float(act[o]) > 0.f) g4[o] = __float2bfloat16(draw);
}

// ------------------------------------------------------------------------------------------
// softmax cross-entropy: logits[i][j] = <r_i, c_j> / temp over the C candidates, label[i];
// loss[i], dr[i] = sum_j (p_ij - y_ij) c_j / temp, dc[j] += (p_ij - y_ij) r_i / temp.
// One CTA (128 threads) per read; C <= 1024.
__global__ void k_ce_loss(const float* __restrict__ r, const float* __restrict__ c, const int32_t* __restrict__ label,
                          int32_t C, float inv_temp, float* __restrict__ loss, float* __restrict__ dr,
                          float* __restrict__ dc, float scale) {
  __shared__ float s_r[kPropC];
  __shared__ float s_p[1024];
  __shared__ float red[4];
  const int i = blockIdx.x, tid = threadIdx.x;
  s_r[tid] = r[i * kPropC + tid];
  __syncthreads();
  for (int j = tid; j < C; j += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < kPropC; ++k) s += s_r[k] * c[j * kPropC + k];
    s_p[j] = s * inv_temp;
  }
  __syncthreads();
  float mx = -1e30f;
  for (int j = tid; j < C; j += blockDim.x) mx = fmaxf(mx, s_p[j]);
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
  __syncthreads();
  float se = 0.f;
  for (int j = tid; j < C; j += blockDim.x) {
    const float ex = __expf(s_p[j] - mx);
    s_p[j] = ex;
    se += ex;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) se += __shfl_xor_sync(0xffffffffu, se, s);
  if ((tid & 31) == 0) red[tid >> 5] = se;
  __syncthreads();
  se = red[0] + red[1] + red[2] + red[3];
  const int lab = label[i];
  const bool lab_ok = lab >= 0 && lab < C;  // an out-of-range label yields NaN loss, no gradient term
  for (int j = tid; j < C; j += blockDim.x) s_p[j] = s_p[j] / se - (j == lab ? 1.f : 0.f);
  __syncthreads();
  if (tid == 0) loss[i] = lab_ok ? -logf(fmaxf((s_p[lab] + 1.f), 1e-30f)) : __int_as_float(0x7fc00000);
  // dr
  float acc = 0.f;
  for (int j = 0; j < C; ++j) acc += s_p[j] * c[j * kPropC + tid];
  dr[i * kPropC + tid] = acc * inv_temp * scale;
  for (int j = 0; j < C; ++j) atomicAdd(dc + j * kPropC + tid, s_p[j] * s_r[tid] * inv_temp * scale);
}

// AdamW step on fp32 master weights; refreshes the bf16 copy when given
__global__ void k_adamw(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                        float* __restrict__ m2, __nv_bfloat16* __restrict__ wb, int64_t count, float lr, float beta1,
                        float beta2, float eps, float wd, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float a = beta1 * m1[i] + (1.f - beta1) * gi;
  const float b = beta2 * m2[i] + (1.f - beta2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  float wi = w[i] * (1.f - lr * wd);
  wi -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16(wi);
}

// flipped, transposed copy for the backward-data pass: wt[t][co][ci] = w[6 - t][ci][co]
__global__ void k_flip_weights(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt) {
  const int t = blockIdx.x, ci = threadIdx.x;
  for (int co = 0; co < kPropC; ++co)
    wt[((int64_t)t * kPropC + co) * kPropC + ci] = w[((int64_t)(kPropTaps - 1 - t) * kPropC + ci) * kPropC + co];
}

// ------------------------------------------------------------------------------------------
// scores[i][f] = max(<e_fwd_i, e_f>, <e_rev_i, e_f>); a CTA takes 8 reads x 128 fragments
// (CUDA cores, FP32 read embeddings; used for K above the tensor-core path's 128)
__global__ void k_scores(const float* __restrict__ er, int32_t R, const __nv_bfloat16* __restrict__ ef, int64_t NF,
                         float* __restrict__ scores) {
  __shared__ float s_e[16][kPropC];
  const int r0 = blockIdx.y * 8;
  for (int e = threadIdx.x; e < 16 * kPropC; e += blockDim.x) {
    const int q = e / kPropC, k = e % kPropC;
    const int read = r0 + (q >> 1);
    s_e[q][k] = read < R ? er[((int64_t)read * 2 + (q & 1)) * kPropC + k] : 0.f;
  }
  __syncthreads();
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= NF) return;
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  // the index is stored as canonical tensor-core tiles of 128 fragments (tc.cuh)
  const uint8_t* ft = reinterpret_cast<const uint8_t*>(ef) + (f >> 7) * (int64_t)(128 * kPropC * 2);
  for (int k2 = 0; k2 < kPropC / 2; ++k2) {
    const float2 v = __bfloat1622float2(
        *reinterpret_cast<const __nv_bfloat162*>(ft + canon_offset((uint32_t)(f & 127), (uint32_t)(2 * k2))));
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] += s_e[q][2 * k2] * v.x + s_e[q][2 * k2 + 1] * v.y;
  }
#pragma unroll
  for (int q = 0; q < 16; q += 2) {
    const int read = r0 + (q >> 1);
    if (read < R) scores[(int64_t)read * NF + f] = fmaxf(acc[q], acc[q + 1]);
  }
}

// order-preserving key of a float
__device__ __forceinline__ uint32_t fkey(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// per-read top K of scores[i][0..NF) (largest first; ties -> lower fragment); one CTA per read:
// 4-round radix select of the K-th largest key, then the elements above it plus the lowest-
// indexed elements equal to it, sorted.
__global__ void k_topk(const float* __restrict__ scores, int64_t NF, int32_t K, int32_t* __restrict__ out_f,
                       float* __restrict__ out_s) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_mask, s_need;
  __shared__ int32_t s_cnt_gt, s_cnt_eq;
  __shared__ uint32_t s_key[1024];
  __shared__ int32_t s_idx[1024];
  const int i = blockIdx.x, tid = threadIdx.x;
  const float* sc = scores + (int64_t)i * NF;
  const int32_t Kc = (int32_t)(NF < (int64_t)K ? NF : K);
  if (tid == 0) {
    s_prefix = 0;
    s_mask = 0;
    s_need = (uint32_t)Kc;
  }
  __syncthreads();
  for (int round = 0; round < 4; ++round) {
    const int shift = 24 - 8 * round;
    for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t pre = s_prefix, msk = s_mask;
    for (int64_t f = tid; f < NF; f += blockDim.x) {
      const uint32_t k = fkey(sc[f]);
      if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {  // walk buckets from the top until the K-th element is reached
      uint32_t need = s_need, b = 255;
      for (;; --b) {
        if (hist[b] >= need || b == 0) break;
        need -= hist[b];
      }
      s_prefix = pre | (b << shift);
      s_mask = msk | (255u << shift);
      s_need = need;
    }
    __syncthreads();
  }
  const uint32_t kth = s_prefix;  // key of the K-th largest element
  if (tid == 0) {
    s_cnt_gt = 0;
    s_cnt_eq = 0;
  }
  __syncthreads();
  // elements strictly above the K-th key (fewer than K), then ties in fragment order
  for (int64_t f = tid; f < NF; f += blockDim.x) {
    const uint32_t k = fkey(sc[f]);
    if (k > kth) {
      const int slot = atomicAdd(&s_cnt_gt, 1);
      if (slot < 1024) {
        s_key[slot] = k;
        s_idx[slot] = (int32_t)f;
      }
    }
  }
  __syncthreads();
  const int ngt = s_cnt_gt;
  const int need_eq = Kc - ngt;
  // lowest-indexed ties: collect the equal keys in parallel (usually a handful), keep the
  // need_eq smallest indices; with very many ties fall back to an ordered scan
  __shared__ int32_t s_tie[1024];
  __shared__ int32_t s_ntie;
  if (tid == 0) s_ntie = 0;
  __syncthreads();
  for (int64_t f = tid; f < NF; f += blockDim.x)
    if (fkey(sc[f]) == kth) {
      const int slot = atomicAdd(&s_ntie, 1);
      if (slot < 1024) s_tie[slot] = (int32_t)f;
    }
  __syncthreads();
  const int ntie = s_ntie;
  if (ntie <= 1024) {
    for (int a = tid; a < ntie; a += blockDim.x) {
      int rank = 0;
      for (int b = 0; b < ntie; ++b) rank += s_tie[b] < s_tie[a];
      if (rank < need_eq) {
        s_key[ngt + rank] = kth;
        s_idx[ngt + rank] = s_tie[a];
      }
    }
    if (tid == 0) s_cnt_eq = ntie < need_eq ? ntie : need_eq;
  } else if (tid == 0) {
    int taken = 0;
    for (int64_t f = 0; f < NF && taken < need_eq; ++f)
      if (fkey(sc[f]) == kth) {
        s_key[ngt + taken] = kth;
        s_idx[ngt + taken] = (int32_t)f;
        ++taken;
      }
    s_cnt_eq = taken;
  }
  __syncthreads();
  const int tot = ngt + s_cnt_eq;
  // sort (key desc, index asc) by rank counting (tot <= K <= 1024)
  for (int a = tid; a < tot; a += blockDim.x) {
    int rank = 0;
    for (int b = 0; b < tot; ++b)
      rank += (s_key[b] > s_key[a]) || (s_key[b] == s_key[a] && s_idx[b] < s_idx[a]);
    out_f[(int64_t)i * K + rank] = s_idx[a];
    if (out_s) out_s[(int64_t)i * K + rank] = sc[s_idx[a]];
  }
  for (int a = tot + tid; a < K; a += blockDim.x) {
    out_f[(int64_t)i * K + a] = -1;
    if (out_s) out_s[(int64_t)i * K + a] = -1e30f;
  }
}

// ------------------------------------------------------------------------------------------
// host launchers
cudaError_t prop_zero_halo(__nv_bfloat16* b0, __nv_bfloat16* b1, __nv_bfloat16* b2, __nv_bfloat16* b3, int32_t n,
                           int32_t rows, cudaStream_t s) {
  const int64_t work = (int64_t)n * 96;
  if (work <= 0) return cudaSuccess;
  k_zero_halo<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(b0, b1, b2, b3, n, rows);
  return cudaGetLastError();
}


cudaError_t prop_pool_norm(const __nv_bfloat16* act, const int32_t* lens, int32_t n, int32_t rows, float* emb,
                           float* norms, int32_t* argmax, int32_t mean, cudaStream_t s) {
  k_pool_norm<<<n, 256, 0, s>>>(act, lens, rows, emb, norms, argmax, mean);
  return cudaGetLastError();
}

cudaError_t prop_pool_norm_bwd(const float* emb, const float* demb, const float* norms, const int32_t* argmax,
                               const __nv_bfloat16* act, const int32_t* lens, int32_t n, int32_t rows,
                               __nv_bfloat16* g4, int32_t mean, cudaStream_t s) {
  k_pool_norm_bwd<<<n, kPropC, 0, s>>>(emb, demb, norms, argmax, act, lens, rows, g4, mean);
  return cudaGetLastError();
}

cudaError_t prop_ce_loss(const float* r, const float* c, const int32_t* label, int32_t B, int32_t C, float inv_temp,
                         float* loss, float* dr, float* dc, float scale, cudaStream_t s) {
  if (C > 1024) return cudaErrorInvalidValue;
  k_ce_loss<<<B, kPropC, 0, s>>>(r, c, label, C, inv_temp, loss, dr, dc, scale);
  return cudaGetLastError();
}

cudaError_t prop_adamw(float* w, const float* g, float* m1, float* m2, __nv_bfloat16* wb, int64_t count, float lr,
                       float beta1, float beta2, float eps, float wd, float bc1, float bc2, cudaStream_t s) {
  k_adamw<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(w, g, m1, m2, wb, count, lr, beta1, beta2, eps, wd, bc1,
                                                          bc2);
  return cudaGetLastError();
}

cudaError_t prop_flip_weights(const __nv_bfloat16* w, __nv_bfloat16* wt, cudaStream_t s) {
  k_flip_weights<<<kPropTaps, kPropC, 0, s>>>(w, wt);
  return cudaGetLastError();
}

cudaError_t prop_scores(const float* er, int32_t R, const __nv_bfloat16* ef, int64_t NF, float* scores,
                        cudaStream_t s) {
  dim3 grid((unsigned)((NF + 127) / 128), (unsigned)((R + 7) / 8));
  k_scores<<<grid, 128, 0, s>>>(er, R, ef, NF, scores);
  return cudaGetLastError();
}

cudaError_t prop_topk(const float* scores, int32_t R, int64_t NF, int32_t K, int32_t* out_f, float* out_s,
                      cudaStream_t s) {
  if (K > 1024) return cudaErrorInvalidValue;
  k_topk<<<R, 256, 0, s>>>(scores, NF, K, out_f, out_s);
  return cudaGetLastError();
}


}  // namespace mss

namespace mss {

// ------------------------------------------------------------------------------------------
// input codes: reads (forward or reverse complement) and genome windows (N beyond the genome)
__global__ void k_read_codes(const char* __restrict__ reads, const int64_t* __restrict__ offsets,
                             const int32_t* __restrict__ idx, const int8_t* __restrict__ strand, int32_t n, int32_t ld,
                             uint8_t* __restrict__ codes, int32_t* __restrict__ lens) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int r = idx ? idx[i] : i;
  const int64_t off = offsets[r];
  int64_t l = offsets[r + 1] - off;
  const int32_t m = (int32_t)(l < 0 ? 0 : (l > ld ? ld : l));
  const bool rc = strand && strand[i];
  for (int k = threadIdx.x; k < ld; k += blockDim.x) {
    uint32_t c = 4;
    if (k < m) {
      c = ascii_code((uint8_t)reads[off + (rc ? (m - 1 - k) : k)]);
      if (c > 4) c = 4;
      if (rc && c < 4) c = 3 - c;
    }
    codes[(int64_t)i * ld + k] = (uint8_t)c;
  }
  if (threadIdx.x == 0) lens[i] = m;
}

__global__ void k_window_codes(const uint32_t* __restrict__ g2, const uint32_t* __restrict__ gm,
                               const int64_t* __restrict__ starts, int32_t n, int32_t len, int32_t ld,
                               uint8_t* __restrict__ codes, int32_t* __restrict__ lens) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int64_t s = starts[i];
  for (int k = threadIdx.x; k < ld; k += blockDim.x)
    codes[(int64_t)i * ld + k] = (uint8_t)(k < len ? genome_code(g2, gm, s + k) : 4u);
  if (threadIdx.x == 0) lens[i] = len;
}

// fallback reads: gather the selected reads into a compact batch (one warp per read) and
// scatter their hits back to the reads' places
__global__ void k_gather_reads(const char* __restrict__ reads, const int64_t* __restrict__ offsets,
                               const int32_t* __restrict__ sel, int32_t n, const int64_t* __restrict__ new_off,
                               char* __restrict__ out) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (w >= n) return;
  const int64_t src = offsets[sel[w]], len = new_off[w + 1] - new_off[w];
  for (int64_t k = lane; k < len; k += 32) out[new_off[w] + k] = reads[src + k];
}

__global__ void k_scatter_hits(const mss_hit* __restrict__ sub, const int32_t* __restrict__ sel, int32_t n,
                               mss_hit* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[sel[j]] = sub[j];
}

// deterministic initialisation: uniform(-a, a) with a = sqrt(6 / fan_in), biases 0.01; the
// uniform draw is a SplitMix64-style hash of (seed, index)
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((z >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
}

__global__ void k_init_params(float* w, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kPropParams) return;
  float v;
  if (i < kPropW1) {
    v = hash_uniform(seed, i) * sqrtf(6.f / (4 * kPropTaps));
  } else if (i < kPropW1 + kPropC) {
    v = 0.01f;
  } else {
    const int64_t j = (i - kPropW1 - kPropC) % (kPropWl + kPropC);
    v = j < kPropWl ? hash_uniform(seed, i) * sqrtf(6.f / (kPropC * kPropTaps)) : 0.01f;
  }
  w[i] = v;
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

cudaError_t prop_read_codes(const char* reads, const int64_t* offsets, const int32_t* idx, const int8_t* strand,
                            int32_t n, int32_t ld, uint8_t* codes, int32_t* lens, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_read_codes<<<n, 128, 0, s>>>(reads, offsets, idx, strand, n, ld, codes, lens);
  return cudaGetLastError();
}

cudaError_t prop_window_codes(const uint32_t* g2, const uint32_t* gm, const int64_t* starts, int32_t n, int32_t len,
                              int32_t ld, uint8_t* codes, int32_t* lens, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_window_codes<<<n, 256, 0, s>>>(g2, gm, starts, n, len, ld, codes, lens);
  return cudaGetLastError();
}

cudaError_t prop_gather_reads(const char* reads, const int64_t* offsets, const int32_t* sel, int32_t n,
                              const int64_t* new_off, char* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_reads<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(reads, offsets, sel, n, new_off, out);
  return cudaGetLastError();
}

cudaError_t prop_scatter_hits(const void* sub, const int32_t* sel, int32_t n, void* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scatter_hits<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(static_cast<const mss_hit*>(sub), sel, n,
                                                             static_cast<mss_hit*>(out));
  return cudaGetLastError();
}

cudaError_t prop_init_params(float* w, uint64_t seed, cudaStream_t s) {
  k_init_params<<<(unsigned)((kPropParams + 255) / 256), 256, 0, s>>>(w, seed);
  return cudaGetLastError();
}

cudaError_t prop_to_bf16(const float* w, __nv_bfloat16* wb, int64_t n, cudaStream_t s) {
  k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, wb, n);
  return cudaGetLastError();
}

}  // namespace mss
