// C ABI of libmaxss: context, validation, workspaces, stream/graph orchestration, autotuner.
// Every compute step runs in the kernels of pack.cu, scan.cu and nw.cu; this file only
// checks arguments, sizes buffers and enqueues work.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/maxss.h"
#include "internal.h"

using namespace mss;

namespace {

thread_local std::string g_last_error;

mss_status fail(mss_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

mss_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(MSS_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(MSS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                              \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

constexpr int64_t kMaxFrag = int64_t(1) << 20;

// Device buffer that grows on demand (never shrinks while the context lives).
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max(bytes, (size_t)256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct GraphKey {
  const void* reads;
  const void* offsets;
  const void* out;
  int32_t R, max_len, match, mismatch;
  int64_t F;
  ScanConfig cfg;
  int grid;
  int64_t chunk_len;
  cudaStream_t stream;
  const void* ws[4];  // workspace pointers baked into the graph
  int32_t exclude;    // second-fragment rule baked into the finalize node
  const void* quals;  // base qualities of the call (null: plain scores)
  const void* qtab;
  int32_t scale;
  bool timing;        // event nodes around the scan
  bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

}  // namespace

struct mss_ctx {
  int device = 0;
  int num_sms = 0;
  PackedGenome pg;
  int64_t G = 0, F = 2048, NF = 0, Gp = 0;
  int32_t max_len = MSS_MAX_READ_LEN;
  int32_t* d_err = nullptr;
  int64_t launches = 0;
  mss_tune tune{-1, 0, 0, 0, 0, 0};  // automatic
  int32_t read_step = 1;              // 2: "MaxSSmap_fast" (every other read base)
  int32_t exclude_neighbors = 0;      // 1: the second fragment is not adjacent to the best
  // position-specific scores from base qualities: the qualities and fixed-point scale of the
  // mapping call in progress (null between calls), and the device tables of phase one / two
  const char* call_quals = nullptr;
  int32_t call_scale = 0;
  DevBuf qtab_scan, qtab_nw;
  int32_t qtab_scan_key[3] = {0, 0, 0}, qtab_nw_key[3] = {0, 0, 0};
  DevBuf hist, order, partial, queue, nw_scratch;
  DevBuf h_reads, h_offsets, h_hits, h_alns, h_cigars;  // staging for the host-pointer calls
  cudaGraphExec_t graph = nullptr;
  GraphKey gkey;
  bool have_graph = false;
  cudaEvent_t ev_scan[2] = {nullptr, nullptr};  // optional events around the scan kernel
  bool timing = false;

  void set_frag(int64_t f) {
    F = f;
    NF = (G + F - 1) / F;
    Gp = NF * F;
  }
};

namespace {

mss_status check_ctx(const mss_ctx* c) {
  if (!c) return fail(MSS_EINVAL, "null context");
  return MSS_OK;
}

mss_status make_ctx(mss_ctx** out, int64_t len, const mss_genome_params* p) {
  if (!out) return fail(MSS_EINVAL, "null output pointer");
  *out = nullptr;
  if (len < 1) return fail(MSS_EINVAL, "genome length %lld < 1", (long long)len);
  int64_t F = p && p->frag_len ? p->frag_len : 2048;
  int32_t ml = p && p->max_read_len ? p->max_read_len : MSS_MAX_READ_LEN;
  if (p && p->reserved != 0) return fail(MSS_EINVAL, "mss_genome_params.reserved must be 0");
  if (F < 16 || F > kMaxFrag) return fail(MSS_EINVAL, "frag_len %lld outside [16, %lld]", (long long)F, (long long)kMaxFrag);
  if (ml < 1 || ml > MSS_MAX_READ_LEN) return fail(MSS_EREADLEN, "max_read_len %d outside [1, %d]", ml, MSS_MAX_READ_LEN);
  mss_ctx* c = new (std::nothrow) mss_ctx();
  if (!c) return fail(MSS_ENOMEM, "context allocation");
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "device query");
  }
  c->G = len;
  c->max_len = ml;
  c->set_frag(F);
  // cover every tile the scan may stage for any allowed F
  int64_t pos = ((len + kMaxFrag + kGenomeTailPad) + 1023) / 1024 * 1024;
  c->pg.G = len;
  c->pg.alloc_pos = pos;
  e = cudaMalloc(&c->pg.g2, (size_t)(pos / 4));
  if (e == cudaSuccess) e = cudaMalloc(&c->pg.gm, (size_t)(pos / 8));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int32_t));
  if (e != cudaSuccess) {
    mss_free(c);
    return cuda_fail(e, "genome allocation");
  }
  *out = c;
  return MSS_OK;
}

mss_status pack_into(mss_ctx* c, const char* d_seq, cudaStream_t s) {
  CK(cudaMemsetAsync(c->pg.g2, 0, (size_t)(c->pg.alloc_pos / 4), s), "genome clear");
  CK(cudaMemsetAsync(c->pg.gm, 0, (size_t)(c->pg.alloc_pos / 8), s), "genome clear");
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s), "error word clear");
  CK(launch_pack_genome(d_seq, c->G, &c->pg, c->d_err, s), "pack kernel");
  c->launches += 1;
  return MSS_OK;
}

mss_status read_err(mss_ctx* c, cudaStream_t s) {
  int32_t h = 0;
  CK(cudaStreamSynchronize(s), "stream synchronize");
  CK(cudaMemcpy(&h, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost), "error word read");
  if (h) CK(cudaMemset(c->d_err, 0, sizeof(int32_t)), "error word clear");
  if (h & ERR_BAD_CHAR) return fail(MSS_EINVAL, "invalid base character (allowed: ACGTN, either case)");
  if (h & ERR_BAD_LEN) return fail(MSS_EREADLEN, "read length 0 or above the declared maximum");
  if (h & ERR_TIMEOUT) return fail(MSS_ETIMEOUT, "a bounded device wait gave up");
  if (h & ERR_SELFCHECK) return fail(MSS_ESTATE, "best-fragment rescan disagreed with the scan");
  if (h & ERR_BAD_QUAL) return fail(MSS_EINVAL, "base quality character outside '!'..'~'");
  return MSS_OK;
}

mss_status resolve_config(const mss_ctx* c, int32_t max_len, const mss_score_params* sp, ScanConfig* cfg,
                          int* grid, int64_t* chunk_len, int32_t R, int32_t* n_chunks, size_t* smem, int* slots) {
  const mss_tune& t = c->tune;
  const bool pssm = c->call_quals != nullptr;
  bool exact16 = !pssm && f16_path_exact(max_len, sp->match, sp->mismatch);
  int variant = t.variant;
  if (variant < 0) variant = exact16 ? 1 : 0;
  if (variant == 1 && !exact16)
    return fail(MSS_EINVAL, "f16 scan variant is not exact for these scores / read lengths (or base qualities)");
  cfg->variant = variant;
  cfg->pairs = t.pairs ? t.pairs : 8;
  cfg->queries = t.queries ? t.queries : (cfg->pairs == 8 ? 4 : 8);
  cfg->threads = t.threads ? t.threads : 256;
  cfg->max_len = max_len;
  cfg->step = c->read_step;
  cfg->pssm = pssm;
  if (cfg->step == 2 && (cfg->pairs != 8 || cfg->queries != 4))
    return fail(MSS_EINVAL, "read step 2 is built for 8 lane pairs x 4 query strands only");
  if (pssm && (cfg->pairs != 8 || cfg->queries != 4 || cfg->step != 1))
    return fail(MSS_EINVAL, "base qualities are built for read step 1 and 8 lane pairs x 4 query strands only");
  if (cfg->threads == 128 && (cfg->pairs != 8 || cfg->queries != 4 || cfg->step != 1 || pssm))
    return fail(MSS_EINVAL, "128 threads per CTA are built for 8 lane pairs x 4 query strands at read step 1 only");
  *slots = scan_ring_slots(*cfg, c->F);
  *smem = scan_smem_bytes(*cfg, max_len, *slots);
  if (*smem == 0)
    return fail(MSS_EINVAL, "unsupported scan configuration (pairs %d, queries %d, max_len %d)", cfg->pairs,
                cfg->queries, max_len);
  int per_sm = 0;
  CK(scan_max_ctas_per_sm(*cfg, *smem, &per_sm), "scan occupancy");
  if (per_sm < 1) return fail(MSS_EINVAL, "scan configuration does not fit on an SM");
  if (t.ctas_per_sm > 0) per_sm = std::min(per_sm, t.ctas_per_sm);
  *grid = c->num_sms * per_sm;
  const int64_t tile = scan_tile_diags(*cfg);
  const int64_t ntiles = (c->Gp + tile - 1) / tile;
  const int RG = cfg->queries / 2;
  const int64_t n_groups = (R + RG - 1) / RG;
  const int64_t want_items = (int64_t)(*grid) * (t.min_items_per_cta > 0 ? t.min_items_per_cta : 4);
  int64_t nch = n_groups > 0 ? (want_items + n_groups - 1) / n_groups : 1;
  nch = std::max<int64_t>(1, std::min(nch, ntiles));
  int64_t tiles_per_chunk = (ntiles + nch - 1) / nch;
  *chunk_len = tiles_per_chunk * tile;
  *n_chunks = (int32_t)((c->Gp + *chunk_len - 1) / *chunk_len);
  return MSS_OK;
}

mss_status check_scores(const mss_ctx* c, int32_t max_len, const mss_score_params* sp) {
  if (!sp) return fail(MSS_EINVAL, "null score parameters");
  if (sp->match < 1 || sp->match > 127) return fail(MSS_EINVAL, "match %d outside [1, 127]", sp->match);
  if (sp->mismatch < -128 || sp->mismatch > 0) return fail(MSS_EINVAL, "mismatch %d outside [-128, 0]", sp->mismatch);
  if (max_len < 1 || max_len > c->max_len)
    return fail(MSS_EREADLEN, "max_len %d outside [1, %d]", max_len, c->max_len);
  if ((int64_t)max_len * sp->match > 32767)
    return fail(MSS_EOVERFLOW, "max_len * match = %lld exceeds the 16-bit lanes", (long long)max_len * sp->match);
  return MSS_OK;
}

// Enqueue phase one.  All buffers are device pointers.
mss_status enqueue_map(mss_ctx* c, const char* d_reads, const int64_t* d_offsets, int32_t R, int32_t max_len,
                       const mss_score_params* sp, mss_hit* d_out, cudaStream_t s, const ScanConfig& cfg, int grid,
                       int64_t chunk_len, int32_t n_chunks, size_t smem, int slots) {
  const int RG = cfg.queries / 2;
  const int32_t n_groups = (R + RG - 1) / RG;
  CK(launch_sort_reads(d_offsets, R, max_len, (int32_t*)c->hist.p, (int32_t*)c->order.p, c->d_err, s), "read sort");
  CK(cudaMemsetAsync(c->queue.p, 0, sizeof(int32_t), s), "queue reset");
  ScanArgs a{};
  a.g2 = c->pg.g2;
  a.gm = c->pg.gm;
  a.Gp = c->Gp;
  a.F = c->F;
  a.reads = d_reads;
  a.offsets = d_offsets;
  a.order = (const int32_t*)c->order.p;
  a.R = R;
  a.n_groups = n_groups;
  a.n_chunks = n_chunks;
  a.n_items = n_groups * n_chunks;
  a.chunk_len = chunk_len;
  a.queue = (int32_t*)c->queue.p;
  a.partial = (int4*)c->partial.p;
  a.err = c->d_err;
  a.max_len = max_len;
  a.ring_slots = slots;
  if (cfg.variant == 1) {
    a.prof_match = (int_to_f16_bits(sp->match) >> 8) & 0xFFu;
    a.prof_mismatch = (int_to_f16_bits(sp->mismatch) >> 8) & 0xFFu;
    a.mm_word = a.prof_mismatch << 8;  // byte 4 = 0x00 (low byte), byte 5 = mismatch high byte
  } else {
    a.prof_match = (uint32_t)sp->match & 0xFFu;
    a.prof_mismatch = (uint32_t)sp->mismatch & 0xFFu;
    a.mm_word = a.prof_mismatch * 0x01010101u;
  }
  a.quals = c->call_quals;
  a.qtab = c->call_quals ? (const int16_t*)c->qtab_scan.p : nullptr;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(grid, a.n_items));
  // inside a stream capture the events become external event nodes of the graph; outside one
  // they are recorded plainly
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (c->timing) CK(cudaStreamIsCapturing(s, &cap), "capture status");
  const bool capturing = cap == cudaStreamCaptureStatusActive;
  if (c->timing)
    CK(capturing ? cudaEventRecordWithFlags(c->ev_scan[0], s, cudaEventRecordExternal) : cudaEventRecord(c->ev_scan[0], s),
       "timing event");
  CK(launch_scan(cfg, a, g, smem, s), "scan kernel");
  if (c->timing)
    CK(capturing ? cudaEventRecordWithFlags(c->ev_scan[1], s, cudaEventRecordExternal) : cudaEventRecord(c->ev_scan[1], s),
       "timing event");
  FinalArgs f{};
  f.g2 = c->pg.g2;
  f.gm = c->pg.gm;
  f.F = c->F;
  f.NF = c->NF;
  f.reads = d_reads;
  f.offsets = d_offsets;
  f.order = (const int32_t*)c->order.p;
  f.R = R;
  f.n_chunks = n_chunks;
  f.reads_per_group = RG;
  f.partial = (const int4*)c->partial.p;
  f.match = sp->match;
  f.mismatch = sp->mismatch;
  f.step = cfg.step;
  f.exclude_neighbors = c->exclude_neighbors;
  f.quals = a.quals;
  f.qtab = a.qtab;
  f.hits = d_out;
  f.err = c->d_err;
  CK(launch_finalize(f, s), "finalize kernel");
  c->launches += 5;  // length histogram, scan of the histogram, scatter, scan, finalize
  return MSS_OK;
}

mss_status map_device(mss_ctx* c, const char* d_reads, const int64_t* d_offsets, int32_t R, int32_t max_len,
                      const mss_score_params* sp, mss_hit* d_out, cudaStream_t s, bool use_graph) {
  mss_status st = check_scores(c, max_len, sp);
  if (st) return st;
  if (R < 0) return fail(MSS_EINVAL, "R < 0");
  if (R == 0) return MSS_OK;
  if (!d_reads || !d_offsets || !d_out) return fail(MSS_EINVAL, "null buffer");
  ScanConfig cfg;
  int grid = 0, slots = 0;
  int64_t chunk_len = 0;
  int32_t n_chunks = 0;
  size_t smem = 0;
  st = resolve_config(c, max_len, sp, &cfg, &grid, &chunk_len, R, &n_chunks, &smem, &slots);
  if (st) return st;
  const int RG = cfg.queries / 2;
  const int64_t n_groups = (R + RG - 1) / RG;
  CK(c->hist.ensure(sizeof(int32_t) * (size_t)(max_len + 2)), "workspace");
  CK(c->order.ensure(sizeof(int32_t) * (size_t)R), "workspace");
  CK(c->partial.ensure(2 * sizeof(int4) * (size_t)(n_groups * RG * n_chunks)), "workspace");
  CK(c->queue.ensure(sizeof(int32_t)), "workspace");

  if (!use_graph || s == nullptr) {
    return enqueue_map(c, d_reads, d_offsets, R, max_len, sp, d_out, s, cfg, grid, chunk_len, n_chunks, smem, slots);
  }
  GraphKey key;
  memset(&key, 0, sizeof(key));
  key.reads = d_reads;
  key.offsets = d_offsets;
  key.out = d_out;
  key.R = R;
  key.max_len = max_len;
  key.match = sp->match;
  key.mismatch = sp->mismatch;
  key.F = c->F;
  key.cfg = cfg;
  key.grid = grid;
  key.chunk_len = chunk_len;
  key.stream = s;
  key.ws[0] = c->hist.p;
  key.ws[1] = c->order.p;
  key.ws[2] = c->partial.p;
  key.ws[3] = c->queue.p;
  key.exclude = c->exclude_neighbors;
  key.quals = c->call_quals;
  key.qtab = c->call_quals ? c->qtab_scan.p : nullptr;
  key.scale = c->call_quals ? c->call_scale : 0;
  key.timing = c->timing;
  if (!(c->have_graph && c->gkey == key)) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    c->have_graph = false;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    int64_t before = c->launches;
    mss_status est = enqueue_map(c, d_reads, d_offsets, R, max_len, sp, d_out, s, cfg, grid, chunk_len, n_chunks,
                                 smem, slots);
    c->launches = before;  // counted when the graph runs
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (est) {
      if (g) cudaGraphDestroy(g);
      return est;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture end");
    ce = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
    c->gkey = key;
    c->have_graph = true;
  }
  CK(cudaGraphLaunch(c->graph, s), "graph launch");
  c->launches += 5;
  return MSS_OK;
}

mss_status check_nw(const mss_nw_params* np, int32_t cigar_stride) {
  if (!np) return fail(MSS_EINVAL, "null NW parameters");
  if (np->reserved != 0) return fail(MSS_EINVAL, "mss_nw_params.reserved must be 0");
  if (np->band < 0 || np->band > 63) return fail(MSS_EINVAL, "band %d outside [0, 63]", np->band);
  if (!(np->gap_open <= np->gap_extend && np->gap_extend <= 0))
    return fail(MSS_EINVAL, "gap costs must satisfy gap_open <= gap_extend <= 0");
  if (np->match < -1000 || np->match > 1000 || np->mismatch < -1000 || np->mismatch > 1000 || np->gap_open < -1000)
    return fail(MSS_EINVAL, "NW scores must lie in [-1000, 1000]");
  if (cigar_stride < 1) return fail(MSS_EINVAL, "cigar_stride < 1");
  return MSS_OK;
}

mss_status nw_device(mss_ctx* c, const char* d_reads, const int64_t* d_offsets, int32_t R, int32_t max_len,
                     const mss_hit* d_hits, const mss_nw_params* np, mss_aln* d_out, char* d_cig, int32_t stride,
                     cudaStream_t s, const char* d_quals = nullptr, int32_t scale = 1) {
  mss_status st = check_nw(np, stride);
  if (st) return st;
  if (R < 0) return fail(MSS_EINVAL, "R < 0");
  if (R == 0) return MSS_OK;
  if (max_len < 1 || max_len > c->max_len) return fail(MSS_EREADLEN, "max_len %d outside [1, %d]", max_len, c->max_len);
  if (!d_reads || !d_offsets || !d_hits || !d_out || !d_cig) return fail(MSS_EINVAL, "null buffer");
  const int n_warps = std::max(1, std::min<int>(R, c->num_sms * 32));
  const int64_t per_warp = nw_scratch_per_warp(max_len, np->band);
  CK(c->nw_scratch.ensure((size_t)(per_warp * n_warps)), "NW scratch");
  NwArgs a{};
  a.g2 = c->pg.g2;
  a.gm = c->pg.gm;
  a.G = c->G;
  a.reads = d_reads;
  a.offsets = d_offsets;
  a.R = R;
  a.max_len = max_len;
  a.hits = d_hits;
  a.match = np->match;
  a.mismatch = np->mismatch;
  a.gap_open = np->gap_open * (d_quals ? scale : 1);   // gaps in the fixed point of the table
  a.gap_extend = np->gap_extend * (d_quals ? scale : 1);
  a.band = np->band;
  a.quals = d_quals;
  a.qtab = d_quals ? (const int16_t*)c->qtab_nw.p : nullptr;
  a.alns = d_out;
  a.cigars = d_cig;
  a.cigar_stride = stride;
  a.scratch = (uint8_t*)c->nw_scratch.p;
  a.scratch_per_warp = per_warp;
  a.n_warps = n_warps;
  a.err = c->d_err;
  CK(launch_nw(a, n_warps, s), "NW kernel");
  c->launches += 1;
  return MSS_OK;
}

// host-pointer calls: validate lengths on the host and stage reads/offsets on the device
mss_status stage_reads(mss_ctx* c, const char* reads, const int64_t* offsets, int32_t R, int32_t* max_len,
                       cudaStream_t s) {
  if (R < 0) return fail(MSS_EINVAL, "R < 0");
  if (R > 0 && (!reads || !offsets)) return fail(MSS_EINVAL, "null buffer");
  if (R > 0 && offsets[0] != 0) return fail(MSS_EINVAL, "offsets[0] must be 0");
  int32_t ml = 0;
  for (int32_t i = 0; i < R; ++i) {
    int64_t l = offsets[i + 1] - offsets[i];
    if (l < 1 || l > c->max_len)
      return fail(MSS_EREADLEN, "read %d has length %lld (allowed 1..%d)", i, (long long)l, c->max_len);
    ml = std::max<int32_t>(ml, (int32_t)l);
  }
  *max_len = ml;
  if (R == 0) return MSS_OK;
  const size_t nb = (size_t)offsets[R];
  CK(c->h_reads.ensure(nb + 16), "staging");
  CK(c->h_offsets.ensure(sizeof(int64_t) * (size_t)(R + 1)), "staging");
  CK(cudaMemcpyAsync(c->h_reads.p, reads, nb, cudaMemcpyHostToDevice, s), "reads upload");
  CK(cudaMemcpyAsync(c->h_offsets.p, offsets, sizeof(int64_t) * (size_t)(R + 1), cudaMemcpyHostToDevice, s),
     "offsets upload");
  return MSS_OK;
}

}  // namespace

namespace mss {

// f16 bit pattern of a small integer (|x| <= 2048), built from the IEEE half layout.
uint32_t int_to_f16_bits(int32_t x) {
  if (x == 0) return 0;
  uint32_t sign = x < 0 ? 0x8000u : 0u;
  uint32_t v = (uint32_t)(x < 0 ? -x : x);
  int e = 31 - __builtin_clz(v);  // v = 1.f * 2^e
  uint32_t mant = (e >= 10) ? ((v >> (e - 10)) & 0x3FFu) : ((v << (10 - e)) & 0x3FFu);
  return sign | ((uint32_t)(e + 15) << 10) | mant;
}

bool f16_path_exact(int32_t max_len, int32_t match, int32_t mismatch) {
  if ((int64_t)max_len * match > 2048) return false;  // every partial sum is an integer <= 2048
  if (match > 2048 || mismatch < -2048) return false;
  return (int_to_f16_bits(match) & 0xFFu) == 0 && (int_to_f16_bits(mismatch) & 0xFFu) == 0;
}


bool ctx_view(mss_ctx* c, CtxView* v) {
  if (!c || !v) return false;
  v->g2 = c->pg.g2;
  v->gm = c->pg.gm;
  v->G = c->G;
  v->max_len = c->max_len;
  v->num_sms = c->num_sms;
  v->d_err = c->d_err;
  v->launches = &c->launches;
  v->exclude_neighbors = c->exclude_neighbors;
  return true;
}

int32_t set_error(int32_t st, const char* msg) { return fail(st, "%s", msg); }

}  // namespace mss

extern "C" {

mss_status mss_load_genome(mss_ctx** out, const char* seq, int64_t len, const mss_genome_params* p, void* stream) {
  if (!seq) return fail(MSS_EINVAL, "null genome");
  mss_status st = make_ctx(out, len, p);
  if (st) return st;
  mss_ctx* c = *out;
  cudaStream_t s = (cudaStream_t)stream;
  char* d = nullptr;
  cudaError_t e = cudaMalloc(&d, (size_t)len + 64);
  if (e != cudaSuccess) {
    mss_free(c);
    *out = nullptr;
    return cuda_fail(e, "genome staging");
  }
  e = cudaMemcpyAsync(d, seq, (size_t)len, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) st = pack_into(c, d, s);
  if (e == cudaSuccess && st == MSS_OK) st = read_err(c, s);
  cudaFree(d);
  if (e != cudaSuccess) st = cuda_fail(e, "genome upload");
  if (st) {
    mss_free(c);
    *out = nullptr;
  }
  return st;
}

mss_status mss_load_genome_device(mss_ctx** out, const char* d_seq, int64_t len, const mss_genome_params* p,
                                  void* stream) {
  if (!d_seq) return fail(MSS_EINVAL, "null genome");
  mss_status st = make_ctx(out, len, p);
  if (st) return st;
  st = pack_into(*out, d_seq, (cudaStream_t)stream);
  if (st == MSS_OK) st = read_err(*out, (cudaStream_t)stream);
  if (st) {
    mss_free(*out);
    *out = nullptr;
  }
  return st;
}

mss_status mss_get_info(const mss_ctx* c, mss_genome_info* info) {
  if (check_ctx(c) || !info) return fail(MSS_EINVAL, "null argument");
  info->genome_len = c->G;
  info->frag_len = c->F;
  info->num_frags = c->NF;
  info->padded_len = c->Gp;
  info->max_read_len = c->max_len;
  info->num_sms = c->num_sms;
  return MSS_OK;
}

mss_status mss_set_frag_len(mss_ctx* c, int64_t F) {
  if (check_ctx(c)) return MSS_EINVAL;
  if (F < 16 || F > kMaxFrag) return fail(MSS_EINVAL, "frag_len %lld outside [16, %lld]", (long long)F, (long long)kMaxFrag);
  c->set_frag(F);
  return MSS_OK;
}

mss_status mss_set_read_step(mss_ctx* c, int32_t step) {
  if (check_ctx(c)) return MSS_EINVAL;
  if (step != 1 && step != 2) return fail(MSS_EINVAL, "read step %d: 1 (every base) or 2 (every other base)", step);
  c->read_step = step;
  return MSS_OK;
}

int32_t mss_get_read_step(const mss_ctx* c) { return c ? c->read_step : -1; }

mss_status mss_set_second_rule(mss_ctx* c, int32_t exclude_neighbors) {
  if (check_ctx(c)) return MSS_EINVAL;
  if (exclude_neighbors != 0 && exclude_neighbors != 1) return fail(MSS_EINVAL, "second rule must be 0 or 1");
  c->exclude_neighbors = exclude_neighbors;
  return MSS_OK;
}

mss_status mss_set_tune(mss_ctx* c, const mss_tune* t) {
  if (check_ctx(c) || !t) return fail(MSS_EINVAL, "null argument");
  if (t->variant < -1 || t->variant > 1) return fail(MSS_EINVAL, "variant must be -1, 0 or 1");
  if (t->pairs != 0 && t->pairs != 4 && t->pairs != 8) return fail(MSS_EINVAL, "pairs must be 4 or 8");
  if (t->queries != 0 && t->queries != 4 && t->queries != 8) return fail(MSS_EINVAL, "queries must be 4 or 8");
  if (t->threads != 0 && t->threads != 128 && t->threads != 256) return fail(MSS_EINVAL, "threads must be 128 or 256");
  if ((t->pairs == 8 ? 8 : 4) == 8 && t->queries == 8) return fail(MSS_EINVAL, "pairs 8 with queries 8 is not built");
  if (t->pairs == 8 && t->queries == 0) {
    mss_tune u = *t;
    u.queries = 4;
    c->tune = u;
    return MSS_OK;
  }
  c->tune = *t;
  return MSS_OK;
}

mss_status mss_get_tune(const mss_ctx* c, mss_tune* t) {
  if (check_ctx(c) || !t) return fail(MSS_EINVAL, "null argument");
  *t = c->tune;
  return MSS_OK;
}

namespace {

// Position-specific scores of base qualities ("Incorporating base qualities and position
// specific scoring matrix"): a base of Phred quality Q is right with probability
// x = 1 - 10^(-Q/10); a match scores match * x, a mismatch mismatch * x / 3; both in fixed point
// (times scale), rounded to the nearest integer with halves away from zero.
void pssm_table(int32_t match, int32_t mismatch, int32_t scale, int16_t* tab) {
  for (int Q = 0; Q < kQualLevels; ++Q) {
    const double x = 1.0 - pow(10.0, -Q / 10.0);
    tab[2 * Q] = (int16_t)lround((double)scale * match * x);
    tab[2 * Q + 1] = (int16_t)lround((double)scale * mismatch * x / 3.0);
  }
}

mss_status ensure_qtab(DevBuf& buf, int32_t* key, int32_t match, int32_t mismatch, int32_t scale) {
  if (buf.p && key[0] == match && key[1] == mismatch && key[2] == scale) return MSS_OK;
  int16_t tab[2 * kQualLevels];
  pssm_table(match, mismatch, scale, tab);
  CK(buf.ensure(sizeof(tab)), "quality table");
  CK(cudaMemcpy(buf.p, tab, sizeof(tab), cudaMemcpyHostToDevice), "quality table upload");
  key[0] = match;
  key[1] = mismatch;
  key[2] = scale;
  return MSS_OK;
}

}  // namespace

mss_status mss_map_reads_quals_device(mss_ctx* c, const char* d_reads, const char* d_quals, const int64_t* d_offsets,
                                      int32_t R, int32_t max_len, const mss_score_params* sp, int32_t scale,
                                      mss_hit* d_out, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  mss_status st = check_scores(c, max_len, sp);
  if (st) return st;
  if (!d_quals) return fail(MSS_EINVAL, "null base qualities");
  if (scale < 1 || scale > 32) return fail(MSS_EINVAL, "scale %d outside [1, 32]", scale);
  if ((int64_t)scale * sp->match > 127 || (int64_t)scale * sp->mismatch < -3 * 128)
    return fail(MSS_EOVERFLOW, "scale * match above 127 or scale * mismatch / 3 below -128 (8-bit profile bytes)");
  if ((int64_t)max_len * (int64_t)lround((double)scale * sp->match) > 32767)
    return fail(MSS_EOVERFLOW, "max_len * scale * match exceeds the 16-bit lanes");
  st = ensure_qtab(c->qtab_scan, c->qtab_scan_key, sp->match, sp->mismatch, scale);
  if (st) return st;
  c->call_quals = d_quals;
  c->call_scale = scale;
  st = map_device(c, d_reads, d_offsets, R, max_len, sp, d_out, (cudaStream_t)stream, true);
  c->call_quals = nullptr;
  c->call_scale = 0;
  return st;
}

mss_status nw_align_quals_device(mss_ctx* c, const char* d_reads, const char* d_quals, const int64_t* d_offsets,
                                 int32_t R, int32_t max_len, const mss_hit* d_hits, const mss_nw_params* np,
                                 int32_t scale, mss_aln* d_out, char* d_cig, int32_t stride, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  mss_status st = check_nw(np, stride);
  if (st) return st;
  if (!d_quals) return fail(MSS_EINVAL, "null base qualities");
  if (scale < 1 || scale > 32) return fail(MSS_EINVAL, "scale %d outside [1, 32]", scale);
  st = ensure_qtab(c->qtab_nw, c->qtab_nw_key, np->match, np->mismatch, scale);
  if (st) return st;
  return nw_device(c, d_reads, d_offsets, R, max_len, d_hits, np, d_out, d_cig, stride, (cudaStream_t)stream, d_quals,
                   scale);
}

mss_status mss_map_reads_device(mss_ctx* c, const char* d_reads, const int64_t* d_offsets, int32_t R,
                                int32_t max_len, const mss_score_params* sp, mss_hit* d_out, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  return map_device(c, d_reads, d_offsets, R, max_len, sp, d_out, (cudaStream_t)stream, true);
}

mss_status mss_map_reads(mss_ctx* c, const char* reads, const int64_t* offsets, int32_t R,
                         const mss_score_params* sp, mss_hit* out, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t ml = 0;
  mss_status st = stage_reads(c, reads, offsets, R, &ml, s);
  if (st || R == 0) return st;
  if (!out) return fail(MSS_EINVAL, "null output");
  CK(c->h_hits.ensure(sizeof(mss_hit) * (size_t)R), "staging");
  st = map_device(c, (const char*)c->h_reads.p, (const int64_t*)c->h_offsets.p, R, ml, sp, (mss_hit*)c->h_hits.p, s,
                  true);
  if (st) return st;
  CK(cudaMemcpyAsync(out, c->h_hits.p, sizeof(mss_hit) * (size_t)R, cudaMemcpyDeviceToHost, s), "hits download");
  return read_err(c, s);
}

mss_status nw_align_device(mss_ctx* c, const char* d_reads, const int64_t* d_offsets, int32_t R, int32_t max_len,
                           const mss_hit* d_hits, const mss_nw_params* np, mss_aln* d_out, char* d_cig,
                           int32_t stride, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  return nw_device(c, d_reads, d_offsets, R, max_len, d_hits, np, d_out, d_cig, stride, (cudaStream_t)stream);
}

mss_status nw_align(mss_ctx* c, const char* reads, const int64_t* offsets, int32_t R, const mss_hit* hits,
                    const mss_nw_params* np, mss_aln* out, char* cig, int32_t stride, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  mss_status st = check_nw(np, stride);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t ml = 0;
  st = stage_reads(c, reads, offsets, R, &ml, s);
  if (st || R == 0) return st;
  if (!hits || !out || !cig) return fail(MSS_EINVAL, "null buffer");
  for (int32_t i = 0; i < R; ++i)
    if (hits[i].offset < 0 || hits[i].strand < 0 || hits[i].strand > 1)
      return fail(MSS_EINVAL, "hit %d has offset %lld / strand %d", i, (long long)hits[i].offset, hits[i].strand);
  CK(c->h_hits.ensure(sizeof(mss_hit) * (size_t)R), "staging");
  CK(c->h_alns.ensure(sizeof(mss_aln) * (size_t)R), "staging");
  CK(c->h_cigars.ensure((size_t)R * (size_t)stride), "staging");
  CK(cudaMemcpyAsync(c->h_hits.p, hits, sizeof(mss_hit) * (size_t)R, cudaMemcpyHostToDevice, s), "hits upload");
  st = nw_device(c, (const char*)c->h_reads.p, (const int64_t*)c->h_offsets.p, R, ml, (const mss_hit*)c->h_hits.p, np,
                 (mss_aln*)c->h_alns.p, (char*)c->h_cigars.p, stride, s);
  if (st) return st;
  CK(cudaMemcpyAsync(out, c->h_alns.p, sizeof(mss_aln) * (size_t)R, cudaMemcpyDeviceToHost, s), "alns download");
  CK(cudaMemcpyAsync(cig, c->h_cigars.p, (size_t)R * (size_t)stride, cudaMemcpyDeviceToHost, s), "cigar download");
  return read_err(c, s);
}

mss_status mss_map_align(mss_ctx* c, const char* reads, const int64_t* offsets, int32_t R,
                         const mss_score_params* sp, const mss_nw_params* np, mss_hit* hits, mss_aln* alns, char* cig,
                         int32_t stride, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  mss_status st = check_nw(np, stride);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t ml = 0;
  st = stage_reads(c, reads, offsets, R, &ml, s);
  if (st || R == 0) return st;
  if (!hits || !alns || !cig) return fail(MSS_EINVAL, "null buffer");
  CK(c->h_hits.ensure(sizeof(mss_hit) * (size_t)R), "staging");
  CK(c->h_alns.ensure(sizeof(mss_aln) * (size_t)R), "staging");
  CK(c->h_cigars.ensure((size_t)R * (size_t)stride), "staging");
  st = map_device(c, (const char*)c->h_reads.p, (const int64_t*)c->h_offsets.p, R, ml, sp, (mss_hit*)c->h_hits.p, s,
                  true);
  if (st) return st;
  st = nw_device(c, (const char*)c->h_reads.p, (const int64_t*)c->h_offsets.p, R, ml, (const mss_hit*)c->h_hits.p, np,
                 (mss_aln*)c->h_alns.p, (char*)c->h_cigars.p, stride, s);
  if (st) return st;
  CK(cudaMemcpyAsync(hits, c->h_hits.p, sizeof(mss_hit) * (size_t)R, cudaMemcpyDeviceToHost, s), "hits download");
  CK(cudaMemcpyAsync(alns, c->h_alns.p, sizeof(mss_aln) * (size_t)R, cudaMemcpyDeviceToHost, s), "alns download");
  CK(cudaMemcpyAsync(cig, c->h_cigars.p, (size_t)R * (size_t)stride, cudaMemcpyDeviceToHost, s), "cigar download");
  return read_err(c, s);
}

mss_status mss_sync(mss_ctx* c, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  return read_err(c, (cudaStream_t)stream);
}

mss_status mss_autotune(mss_ctx* c, const char* d_reads, const int64_t* d_offsets, int32_t R, int32_t max_len,
                        const mss_score_params* sp, int32_t allow_frag_len, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  mss_status st = check_scores(c, max_len, sp);
  if (st) return st;
  if (R < 1) return fail(MSS_EINVAL, "autotune needs at least one read");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf hits;
  CK(hits.ensure(sizeof(mss_hit) * (size_t)R), "autotune buffer");
  const bool exact16 = f16_path_exact(max_len, sp->match, sp->mismatch);
  std::vector<mss_tune> cands;
  for (int v = exact16 ? 1 : 0; v >= 0; --v)
    for (int pq = 0; pq < 3; ++pq)
      for (int cps : {0, 1}) {
        const int pairs = pq == 1 ? 8 : 4, queries = pq == 1 ? 4 : (pq == 2 ? 4 : 8);
        mss_tune t{v, pairs, queries, cps, 0, 0};
        cands.push_back(t);
        if (pq == 1 && c->read_step == 1 && !c->call_quals) {  // the 128-thread shape
          t.threads = 128;
          cands.push_back(t);
        }
      }
  std::vector<int64_t> frags = {c->F};
  if (allow_frag_len) frags = {1024, 2048, 4096, 8192};
  const mss_tune saved = c->tune;
  const int64_t savedF = c->F;
  float best_ms = 1e30f;
  mss_tune best = saved;
  int64_t bestF = savedF;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  int timed = 0;
  std::string last_failure;
  for (int64_t F : frags) {
    c->set_frag(F);
    for (const mss_tune& t : cands) {
      c->tune = t;
      st = map_device(c, d_reads, d_offsets, R, max_len, sp, (mss_hit*)hits.p, s, false);  // warm-up
      if (st) {
        last_failure = g_last_error;
        continue;
      }
      cudaEventRecord(e0, s);
      st = map_device(c, d_reads, d_offsets, R, max_len, sp, (mss_hit*)hits.p, s, false);
      cudaEventRecord(e1, s);
      if (st) continue;
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ++timed;
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
        bestF = F;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tune = best;
  c->set_frag(bestF);
  hits.release();
  if (timed == 0) return fail(MSS_ECUDA, "autotune: no candidate ran (%s)", last_failure.c_str());
  g_last_error.clear();
  return read_err(c, s);
}

mss_status mss_scan_timing(mss_ctx* c, int32_t enable) {
  if (check_ctx(c)) return MSS_EINVAL;
  if (enable && !c->ev_scan[0]) {
    CK(cudaEventCreate(&c->ev_scan[0]), "event create");
    CK(cudaEventCreate(&c->ev_scan[1]), "event create");
  }
  c->timing = enable != 0;
  return MSS_OK;
}

mss_status mss_scan_time_ms(mss_ctx* c, float* ms) {
  if (check_ctx(c) || !ms) return fail(MSS_EINVAL, "null argument");
  if (!c->ev_scan[0]) return fail(MSS_ESTATE, "scan timing was never enabled");
  CK(cudaEventSynchronize(c->ev_scan[1]), "event synchronize");
  CK(cudaEventElapsedTime(ms, c->ev_scan[0], c->ev_scan[1]), "event elapsed time");
  return MSS_OK;
}

int64_t mss_launch_count(const mss_ctx* c) { return c ? c->launches : -1; }

mss_status mss_genome_codes(const mss_ctx* c, int64_t start, int64_t n, uint8_t* out) {
  if (check_ctx(c) || !out) return fail(MSS_EINVAL, "null argument");
  if (start < 0 || n < 0 || start + n > c->pg.alloc_pos) return fail(MSS_EINVAL, "range outside the packed genome");
  if (n == 0) return MSS_OK;
  uint8_t* d = nullptr;
  CK(cudaMalloc(&d, (size_t)n), "decode buffer");
  cudaError_t e = launch_decode_genome(&c->pg, start, n, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "genome decode");
  const_cast<mss_ctx*>(c)->launches += 1;
  return MSS_OK;
}

mss_status mss_probe_pipes(double* rates, int32_t n_rates, double* clk_mhz) {
  if (!rates || !clk_mhz || n_rates < 1) return fail(MSS_EINVAL, "null argument or no rate slots");
  CK(probe_pipes(rates, n_rates, clk_mhz), "pipe probe");
  return MSS_OK;
}

mss_status mss_check_wait_timeout(mss_ctx* c, uint32_t limit_us, void* stream) {
  if (check_ctx(c)) return MSS_EINVAL;
  if (limit_us < 1 || limit_us > 1000000) return fail(MSS_EINVAL, "wait limit must be 1 us .. 1 s");
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_wait_selfcheck(c->d_err, (uint64_t)limit_us * 1000ull, s), "wait self-check kernel");
  c->launches += 1;
  return read_err(c, s);
}

void mss_free(mss_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (cudaEvent_t e : c->ev_scan)
    if (e) cudaEventDestroy(e);
  if (c->pg.g2) cudaFree(c->pg.g2);
  if (c->pg.gm) cudaFree(c->pg.gm);
  if (c->d_err) cudaFree(c->d_err);
  for (DevBuf* b : {&c->hist, &c->order, &c->partial, &c->queue, &c->nw_scratch, &c->h_reads, &c->h_offsets,
                    &c->h_hits, &c->h_alns, &c->h_cigars})
    b->release();
  delete c;
}

const char* mss_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
