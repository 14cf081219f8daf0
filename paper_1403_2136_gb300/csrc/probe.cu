// Throughput probe of the two packed 16-bit pipes the scan relies on: the integer/DPX pipe
// (packed int16 add-max) and the FMA pipe (packed f16 fused multiply-add with relu).  Each
// thread runs 16 independent dependency chains so that issue, not latency, is measured.
// The measured warp-instructions per SM clock set the denominator of the scan's roofline.
#include "common.cuh"
#include "internal.h"

namespace mss {

template <int MODE>
__global__ void k_probe(uint32_t* out, int iters, uint32_t seed) {
  constexpr int C = 16;
  uint32_t h[C], m[C];
  const uint32_t t = threadIdx.x + blockIdx.x * blockDim.x;
#pragma unroll
  for (int i = 0; i < C; ++i) {
    h[i] = (t * 2654435761u + i * 40503u + seed) & 0x03ff03ffu;
    m[i] = (h[i] * 7u) & 0x00ff00ffu;
  }
  const uint32_t one = 0x3C003C00u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < C; ++i) {
      if (MODE == 0) {  // two packed int16 DPX add-max per chain step
        h[i] = __viaddmax_s16x2(h[i], m[i], 0u);
        m[i] = __viaddmax_s16x2(m[i], h[i], 0u);
      } else if (MODE == 1) {  // two packed f16 FMA-relu per chain step
        h[i] = hfma2_relu(h[i], one, m[i]);
        m[i] = hfma2_relu(m[i], one, h[i]);
      } else {  // one of each: both pipes busy
        h[i] = __viaddmax_s16x2(h[i], m[i], 0u);
        m[i] = hfma2_relu(m[i], one, h[i]);
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < C; ++i) acc ^= h[i] ^ m[i];
  out[t] = acc;
}

template <int MODE>
static cudaError_t time_probe(int sms, uint32_t* buf, int blocks, int threads, int iters, double* rate) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) return e;
  k_probe<MODE><<<blocks, threads>>>(buf, 16, 1u);
  cudaEventRecord(a);
  k_probe<MODE><<<blocks, threads>>>(buf, iters, 2u);
  cudaEventRecord(b);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  // clock: cycles counted through the SM clock the device reports now
  int dev = 0, clk_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const double warp_instr = (double)blocks * threads / 32.0 * iters * 32.0;
  *rate = warp_instr / (ms * 1e-3) / sms / (clk_khz * 1e3);
  return cudaGetLastError();
}

cudaError_t probe_pipes(double* rates3, double* clk_mhz) {
  int dev = 0, sms = 0, clk_khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int threads = 256, blocks = sms * 8, iters = 4096;
  uint32_t* buf = nullptr;
  e = cudaMalloc(&buf, sizeof(uint32_t) * blocks * threads);
  if (e != cudaSuccess) return e;
  e = time_probe<0>(sms, buf, blocks, threads, iters, &rates3[0]);
  if (e == cudaSuccess) e = time_probe<1>(sms, buf, blocks, threads, iters, &rates3[1]);
  if (e == cudaSuccess) e = time_probe<2>(sms, buf, blocks, threads, iters, &rates3[2]);
  cudaFree(buf);
  *clk_mhz = clk_khz / 1000.0;
  return e;
}

// Self-check of the bounded-wait error path: one thread waits, with the given limit, on an
// mbarrier phase that nothing completes (no copy armed, no arrival), then reports the time-out
// through the context's error word exactly as the scan does, and returns.
__global__ void k_wait_selfcheck(int32_t* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(&bar, 0u, limit_ns)) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_wait_selfcheck(int32_t* err, uint64_t limit_ns, cudaStream_t s) {
  k_wait_selfcheck<<<1, 32, 0, s>>>(err, limit_ns);
  return cudaGetLastError();
}

}  // namespace mss
