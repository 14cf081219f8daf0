// Throughput probes of the packed 16-bit instructions the scan is built from, in
// warp-instructions per SM clock.  Each thread runs 16 independent dependency chains so that
// issue and pipe occupancy, not latency, are measured.
//   0  packed int16 DPX add-max alone (integer/DPX pipe)
//   1  packed f16 FMA with relu alone (FMA pipe)
//   2  PRMT and f16 FMA-relu interleaved: both 16-lane pipes busy (the two-pipe peak)
//   3  PRMT alone
//   4  three-input packed int16 max alone
//   5  the scan's own mix per chain step: 2 PRMT + 2 f16 FMA-relu + 1 three-input max
//   6  DPX add-max and f16 FMA-relu interleaved (these two share issue capacity)
// The rates set the denominators of the scan's roofline.
#include "common.cuh"
#include "internal.h"

namespace mss {

constexpr int kProbeModes = 7;

template <int MODE>
__global__ void k_probe(uint32_t* out, int iters, uint32_t seed) {
  constexpr int C = 16;
  uint32_t h[C], m[C], z[C];
  const uint32_t t = threadIdx.x + blockIdx.x * blockDim.x;
#pragma unroll
  for (int i = 0; i < C; ++i) {
    h[i] = (t * 2654435761u + i * 40503u + seed) & 0x03ff03ffu;
    m[i] = (h[i] * 7u) & 0x00ff00ffu;
    z[i] = h[i] ^ 0x00510040u;
  }
  const uint32_t one = 0x3C003C00u, mmw = 0xC400u ^ (seed >> 30), sel = 0x7150u ^ (seed >> 29);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < C; ++i) {
      if (MODE == 0) {
        h[i] = __viaddmax_s16x2(h[i], m[i], 0u);
        m[i] = __viaddmax_s16x2(m[i], h[i], 0u);
      } else if (MODE == 1) {
        h[i] = hfma2_relu(h[i], one, m[i]);
        m[i] = hfma2_relu(m[i], one, h[i]);
      } else if (MODE == 2) {  // independent streams, shared operands: PRMT on one, FMA-relu on the other
        h[i] = prmt(h[i], mmw, sel);
        m[i] = hfma2_relu(m[i], one, mmw);
      } else if (MODE == 3) {
        h[i] = prmt(h[i], mmw, z[i]);
        m[i] = prmt(m[i], mmw, z[i]);
      } else if (MODE == 4) {
        h[i] = __vimax3_s16x2(h[i], m[i], z[i]);
        m[i] = __vimax3_s16x2(m[i], h[i], z[i]);
      } else if (MODE == 5) {  // two lane pairs of the scan's inner loop (score, H, running max)
        const uint32_t s1 = prmt(z[i], mmw, m[i]);
        const uint32_t a = hfma2_relu(h[i], one, s1);
        const uint32_t s2 = prmt(z[i], mmw, sel);
        const uint32_t b = hfma2_relu(a, one, s2);
        z[i] = __vimax3_s16x2(z[i], a, b);
        h[i] = b;
      } else {
        h[i] = __viaddmax_s16x2(h[i], z[i], 0u);
        m[i] = hfma2_relu(m[i], one, z[i]);
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < C; ++i) acc ^= h[i] ^ m[i] ^ z[i];
  out[t] = acc;
}

template <int MODE>
static cudaError_t time_probe(int sms, uint32_t* buf, int blocks, int threads, int iters, double* rate) {
  constexpr double kInstrPerStep = MODE == 5 ? 5.0 : 2.0;  // warp-instructions per chain step
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
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
  // clock: cycles counted through the SM clock the device reports (its maximum)
  int dev = 0, clk_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const double warp_instr = (double)blocks * threads / 32.0 * iters * 16.0 * kInstrPerStep;
  *rate = warp_instr / (ms * 1e-3) / sms / (clk_khz * 1e3);
  return cudaGetLastError();
}

cudaError_t probe_pipes(double* rates, int n, double* clk_mhz) {
  int dev = 0, sms = 0, clk_khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int threads = 256, blocks = sms * 8, iters = 4096;
  uint32_t* buf = nullptr;
  e = cudaMalloc(&buf, sizeof(uint32_t) * blocks * threads);
  if (e != cudaSuccess) return e;
  double r[kProbeModes] = {0, 0, 0, 0, 0, 0, 0};
  e = time_probe<0>(sms, buf, blocks, threads, iters, &r[0]);
  if (e == cudaSuccess) e = time_probe<1>(sms, buf, blocks, threads, iters, &r[1]);
  if (e == cudaSuccess) e = time_probe<2>(sms, buf, blocks, threads, iters, &r[2]);
  if (e == cudaSuccess) e = time_probe<3>(sms, buf, blocks, threads, iters, &r[3]);
  if (e == cudaSuccess) e = time_probe<4>(sms, buf, blocks, threads, iters, &r[4]);
  if (e == cudaSuccess) e = time_probe<5>(sms, buf, blocks, threads, iters, &r[5]);
  if (e == cudaSuccess) e = time_probe<6>(sms, buf, blocks, threads, iters, &r[6]);
  cudaFree(buf);
  for (int i = 0; i < n && i < kProbeModes; ++i) rates[i] = r[i];
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
