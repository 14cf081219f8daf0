// a1: genome packing (ASCII -> 2-bit codes + valid bits) and a2: read ordering.
//
// The paper packs the genome as int4 characters and transposes it so that fragment-parallel
// threads read consecutive bytes ("Byte packing", "Coalescent global memory access").  Here
// the genome is kept in genome order at 2 bits per base plus one valid bit (N and padding are
// invalid): 3/8 byte per base, read by the scan through bulk (TMA) copies of whole tiles, so
// no transposed copy is needed in global memory.
#include "common.cuh"
#include "internal.h"

namespace mss {

__global__ void k_pack_genome(const char* __restrict__ seq, int64_t G, uint32_t* __restrict__ g2,
                              uint32_t* __restrict__ gm, int32_t* err) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one valid-bit word = 32 bases
  int64_t p0 = w * 32;
  if (p0 >= G) return;
  uint8_t ch[32];
  if (p0 + 32 <= G && ((reinterpret_cast<uintptr_t>(seq + p0) & 15u) == 0)) {
    const uint4* src = reinterpret_cast<const uint4*>(seq + p0);  // 16-byte aligned (checked)
    uint4 a = src[0], b = src[1];
    *reinterpret_cast<uint4*>(ch) = a;
    *reinterpret_cast<uint4*>(ch + 16) = b;
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) ch[i] = (p0 + i < G) ? (uint8_t)seq[p0 + i] : (uint8_t)'N';
  }
  uint32_t lo = 0, hi = 0, mask = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    uint32_t c = ascii_code(ch[i]);
    bad |= (c == 5);
    if (c < 4) {
      mask |= 1u << i;
      if (i < 16)
        lo |= c << (2 * i);
      else
        hi |= c << (2 * (i - 16));
    }
  }
  g2[2 * w] = lo;
  g2[2 * w + 1] = hi;
  gm[w] = mask;
  if (bad) atomicOr(err, ERR_BAD_CHAR);
}

cudaError_t launch_pack_genome(const char* d_seq, int64_t G, PackedGenome* pg, int32_t* err, cudaStream_t s) {
  int64_t words = (G + 31) / 32;
  int threads = 256;
  int64_t blocks = (words + threads - 1) / threads;
  k_pack_genome<<<(unsigned)blocks, threads, 0, s>>>(d_seq, G, pg->g2, pg->gm, err);
  return cudaGetLastError();
}

__global__ void k_decode_genome(const uint32_t* __restrict__ g2, const uint32_t* __restrict__ gm, int64_t start,
                                int64_t n, uint8_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint8_t)genome_code(g2, gm, start + i);
}

cudaError_t launch_decode_genome(const PackedGenome* pg, int64_t start, int64_t n, uint8_t* d_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int threads = 256;
  k_decode_genome<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(pg->g2, pg->gm, start, n, d_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- read order (a2)
// Reads are processed in groups that share one padded length, so they are ordered by length,
// longest first (longest work first also balances the persistent scan).  Counting sort over
// lengths 0..max_len; the order inside one length is arbitrary (each read's result depends on
// that read alone).

__device__ __forceinline__ int32_t clamp_len(int64_t len, int32_t max_len) {
  return len < 0 ? 0 : (len > max_len ? max_len : (int32_t)len);
}

__global__ void k_len_hist(const int64_t* __restrict__ off, int32_t R, int32_t max_len, int32_t* hist,
                           int32_t* err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R) return;
  int64_t len = off[i + 1] - off[i];
  if (len < 1 || len > max_len) atomicOr(err, ERR_BAD_LEN);
  atomicAdd(&hist[clamp_len(len, max_len)], 1);
}

__global__ void k_hist_scan(int32_t* hist, int32_t max_len) {
  // exclusive prefix over lengths in descending order: cursor[L] = #reads longer than L
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t run = 0;
  for (int32_t L = max_len; L >= 0; --L) {
    int32_t c = hist[L];
    hist[L] = run;
    run += c;
  }
}

__global__ void k_scatter(const int64_t* __restrict__ off, int32_t R, int32_t max_len, int32_t* hist,
                          int32_t* __restrict__ order) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R) return;
  int32_t L = clamp_len(off[i + 1] - off[i], max_len);
  int32_t pos = atomicAdd(&hist[L], 1);
  order[pos] = i;
}

cudaError_t launch_sort_reads(const int64_t* d_off, int32_t R, int32_t max_len, int32_t* hist, int32_t* order,
                              int32_t* err, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)(max_len + 2), s);
  if (e != cudaSuccess) return e;
  int threads = 256;
  unsigned blocks = (unsigned)((R + threads - 1) / threads);
  k_len_hist<<<blocks, threads, 0, s>>>(d_off, R, max_len, hist, err);
  k_hist_scan<<<1, 32, 0, s>>>(hist, max_len);
  k_scatter<<<blocks, threads, 0, s>>>(d_off, R, max_len, hist, order);
  return cudaGetLastError();
}

}  // namespace mss
