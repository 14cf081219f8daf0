// Host-side declarations shared by the libmaxss translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mss {

// Device error bits (OR-ed into the context's error word; read back by mss_sync).
enum : int32_t {
  ERR_BAD_CHAR = 1,     // a read character outside ACGTN (either case)
  ERR_BAD_LEN = 2,      // a read of length 0 or above the declared maximum
  ERR_TIMEOUT = 4,      // a bounded mbarrier wait gave up
  ERR_SELFCHECK = 8,    // the best-fragment rescan disagreed with the scan
  ERR_BAD_QUAL = 16,    // a base-quality character outside '!'..'~'
};
// Position-specific scores of base qualities: entry 2Q, 2Q + 1 = (match, mismatch) of a base of
// Phred quality Q = 0..93, in fixed point (built on the host, see pssm_table in api.cu).
constexpr int kQualLevels = 94;

// Genome tiles: the largest tile a scan variant uses and the extra positions past the last
// fragment that a tile may read; the packed genome is allocated (zero = N) to cover them.
constexpr int64_t kMaxTileDiags = 4096;  // largest NT * 2D of any scan variant
constexpr int64_t kGenomeTailPad = kMaxTileDiags + 2432 + 512;

struct PackedGenome {
  uint32_t* g2 = nullptr;  // 2-bit codes
  uint32_t* gm = nullptr;  // valid bits
  int64_t G = 0;
  int64_t alloc_pos = 0;   // positions covered by the allocation
};

// a1: ASCII (device) -> packed genome.  err: device error word.
cudaError_t launch_pack_genome(const char* d_seq, int64_t G, PackedGenome* pg, int32_t* err, cudaStream_t s);
cudaError_t launch_decode_genome(const PackedGenome* pg, int64_t start, int64_t n, uint8_t* d_out, cudaStream_t s);

// a2: read lengths, validation and the length-descending order.
//   hist: int32[max_len + 2] scratch, order: int32[R] out.
cudaError_t launch_sort_reads(const int64_t* d_off, int32_t R, int32_t max_len, int32_t* hist, int32_t* order,
                              int32_t* err, cudaStream_t s);

struct ScanConfig {
  int variant;  // 0 int16 DPX, 1 f16 FMA + DPX max
  int pairs;    // D
  int queries;  // RQ
  int threads;  // NT
  int max_len;  // longest read of the call (selects the selector-row size)
  int step;     // read step: 1 every base, 2 every other base ("MaxSSmap_fast")
  bool pssm;    // position-specific scores from base qualities (int16 lanes only)
};

struct ScanArgs {
  const uint32_t* g2;
  const uint32_t* gm;
  int64_t Gp;
  int64_t F;
  const char* reads;
  const int64_t* offsets;
  const int32_t* order;
  int32_t R;
  int32_t n_groups;
  int32_t n_chunks;
  int32_t n_items;
  int64_t chunk_len;
  int32_t* queue;
  int4* partial;           // per (read, chunk): top-4 summary, two int4
  int32_t* err;
  int32_t max_len;
  int32_t ring_slots;
  uint32_t prof_match;     // byte encodings used to build the query profile
  uint32_t prof_mismatch;
  uint32_t mm_word;        // second PRMT operand (genome N -> mismatch)
  const char* quals;       // base qualities (Phred+33, same offsets as the reads) or null
  const int16_t* qtab;     // [kQualLevels][2] position-specific scores when quals is set
};

// Smallest tile (diagonals) of a configuration; chunk lengths are multiples of it.
int64_t scan_tile_diags(const ScanConfig& c);
size_t scan_smem_bytes(const ScanConfig& c, int32_t max_len, int32_t ring_slots);
int scan_ring_slots(const ScanConfig& c, int64_t F);
cudaError_t scan_max_ctas_per_sm(const ScanConfig& c, size_t smem, int* out);
cudaError_t launch_scan(const ScanConfig& c, const ScanArgs& a, int grid, size_t smem, cudaStream_t s);
bool scan_supported(const ScanConfig& c);

struct FinalArgs {
  const uint32_t* g2;
  const uint32_t* gm;
  int64_t F;
  int64_t NF;
  const char* reads;
  const int64_t* offsets;
  const int32_t* order;
  int32_t R;
  int32_t n_chunks;
  int32_t reads_per_group;
  const int4* partial;      // per (read, chunk): the top-4 as two int4 (score, fragment) pairs
  int32_t exclude_neighbors;  // second = best fragment not adjacent to the best
  int32_t match, mismatch;
  int32_t step;  // read step of the scan (the rescan samples the read the same way)
  const char* quals;    // base qualities or null (as ScanArgs)
  const int16_t* qtab;
  void* hits;  // mss_hit[R], input order
  int32_t* err;
};
cudaError_t launch_finalize(const FinalArgs& a, cudaStream_t s);

struct NwArgs {
  const uint32_t* g2;
  const uint32_t* gm;
  int64_t G;
  const char* reads;
  const int64_t* offsets;
  int32_t R;
  int32_t max_len;
  const void* hits;  // mss_hit[R]
  int32_t match, mismatch, gap_open, gap_extend, band;
  const char* quals;     // base qualities or null: per read base (match, mismatch) from qtab
  const int16_t* qtab;
  void* alns;        // mss_aln[R]
  char* cigars;
  int32_t cigar_stride;
  uint8_t* scratch;  // per-warp traceback: n_warps * scratch_per_warp bytes
  int64_t scratch_per_warp;
  int32_t n_warps;
  int32_t* err;
};
int64_t nw_scratch_per_warp(int32_t max_len, int32_t band);
cudaError_t launch_nw(const NwArgs& a, int grid_warps, cudaStream_t s);

cudaError_t probe_pipes(double* rates, int n, double* clk_mhz);
cudaError_t launch_wait_selfcheck(int32_t* err, uint64_t limit_ns, cudaStream_t s);
// f16 bit pattern of a small integer; whether the f16 lanes are exact for these scores
uint32_t int_to_f16_bits(int32_t x);
bool f16_path_exact(int32_t max_len, int32_t match, int32_t mismatch);

}  // namespace mss

typedef struct mss_ctx mss_ctx;

namespace mss {

// Read-only view of a context for entry points defined outside api.cu.
struct CtxView {
  const uint32_t* g2;
  const uint32_t* gm;
  int64_t G;
  int32_t max_len;
  int32_t num_sms;
  int32_t* d_err;
  int64_t* launches;
  int32_t exclude_neighbors;  // second-fragment rule of the context
};
bool ctx_view(mss_ctx* c, CtxView* v);
// Record the thread-local message returned by mss_last_error() and return st.
int32_t set_error(int32_t st, const char* msg);

}  // namespace mss
