// Phase two for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: code that runs while a CUDA stream is being
// captured into a graph (an allocation there breaks or invalidates the capture), latency-
// critical serving loops where an allocation can stall on a device-wide synchronisation, and
// hosts whose device memory is owned by a pool or a framework allocator that would not see a
// private cudaMalloc.  For them nw_align_device_noalloc runs the same banded NW kernel as
// nw_align_device, but its per-warp traceback scratch is a fixed array that lives in this
// library's device image instead of a buffer the context grows on demand.
//
// The array is kNoAllocScratchBytes (4 MiB); every GPU that loads the library keeps it until
// the process exits.  Its device address is looked up once per device, on that device's first
// call (so make the first call on each device outside any stream capture).  All calls share
// the one array: calls that can run at the same time on the GPU (different streams, or
// different host threads with one device) race on it and must be ordered by the caller.
// Nothing in it needs to start at zero: every direction byte is written before it is read.
#include <mutex>

#include "../../include/maxss.h"
#include "internal.h"

namespace mss {

constexpr int64_t kNoAllocScratchBytes = int64_t(4) << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) uint8_t g_nw_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_nw_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace mss

using namespace mss;

extern "C" mss_status nw_align_device_noalloc(mss_ctx* ctx, const char* d_reads, const int64_t* d_offsets,
                                              int32_t R, int32_t max_len, const mss_hit* d_hits,
                                              const mss_nw_params* np, mss_aln* d_out, char* d_cigar_buf,
                                              int32_t cigar_stride, void* stream) {
  CtxView v;
  if (!ctx_view(ctx, &v)) return set_error(MSS_EINVAL, "null context");
  if (!np) return set_error(MSS_EINVAL, "null NW parameters");
  if (np->reserved != 0) return set_error(MSS_EINVAL, "mss_nw_params.reserved must be 0");
  if (np->band < 0 || np->band > 63) return set_error(MSS_EINVAL, "band outside [0, 63]");
  if (!(np->gap_open <= np->gap_extend && np->gap_extend <= 0))
    return set_error(MSS_EINVAL, "gap costs must satisfy gap_open <= gap_extend <= 0");
  if (np->match < -1000 || np->match > 1000 || np->mismatch < -1000 || np->mismatch > 1000 || np->gap_open < -1000)
    return set_error(MSS_EINVAL, "NW scores must lie in [-1000, 1000]");
  if (cigar_stride < 1) return set_error(MSS_EINVAL, "cigar_stride < 1");
  if (R < 0) return set_error(MSS_EINVAL, "R < 0");
  if (max_len < 1 || max_len > v.max_len) return set_error(MSS_EREADLEN, "max_len outside [1, context maximum]");
  const int64_t per_warp = nw_scratch_per_warp(max_len, np->band);
  if (per_warp > kNoAllocScratchBytes)
    return set_error(MSS_EINVAL, "one traceback slot needs more than the 4 MiB static scratch");
  if (R == 0) return MSS_OK;
  if (!d_reads || !d_offsets || !d_hits || !d_out || !d_cigar_buf) return set_error(MSS_EINVAL, "null buffer");
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return set_error(MSS_ECUDA, cudaGetErrorString(e));
  // as many concurrent traceback slots as the array holds, at most one warp per read
  int64_t slots = kNoAllocScratchBytes / per_warp;
  slots = slots < (int64_t)v.num_sms * 32 ? slots : (int64_t)v.num_sms * 32;
  slots = slots < (int64_t)R ? slots : (int64_t)R;
  NwArgs a{};
  a.g2 = v.g2;
  a.gm = v.gm;
  a.G = v.G;
  a.reads = d_reads;
  a.offsets = d_offsets;
  a.R = R;
  a.max_len = max_len;
  a.hits = d_hits;
  a.match = np->match;
  a.mismatch = np->mismatch;
  a.gap_open = np->gap_open;
  a.gap_extend = np->gap_extend;
  a.band = np->band;
  a.alns = d_out;
  a.cigars = d_cigar_buf;
  a.cigar_stride = cigar_stride;
  a.scratch = static_cast<uint8_t*>(scratch);
  a.scratch_per_warp = per_warp;
  a.n_warps = (int32_t)slots;
  a.err = v.d_err;
  e = launch_nw(a, (int)slots, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(MSS_ECUDA, cudaGetErrorString(e));
  ++*v.launches;
  return MSS_OK;
}
