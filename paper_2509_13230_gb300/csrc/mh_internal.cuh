// Internal declarations of the GB300 maximum-entropy sampler library.
//
// Device-wide conventions
//  * Node ranks follow the sort of Sec. 2.4 step (i) / Algorithm 1: rank 0 has
//    the largest key (x for UBCM, a = x*y for UECM).
//  * FP64 expressions that decide sampled bits are written in one fixed order;
//    the library is compiled with --fmad=false so none of them is contracted
//    into an FMA.  Explicit fma() calls are used only where a rounding error is
//    being measured, never in a decision.
//  * Device status bits are OR-ed into Ctrl::status and mapped to MH_ERR_* on
//    the host after the final read-back; no kernel traps or asserts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/maxent_mh.h"

namespace mh {

// ---- status bits ----------------------------------------------------------
constexpr unsigned kStDomain = 1u;    // bad x / y value
constexpr unsigned kStSegments = 2u;  // segment table larger than its capacity
constexpr unsigned kStCapacity = 4u;  // output or staging shorter than the sample
constexpr unsigned kStOverflow = 8u;  // weight above INT32_MAX
constexpr unsigned kStTimeout = 16u;  // bounded device wait gave up
constexpr unsigned kStInternal = 32u; // an internal consistency check failed
constexpr unsigned kStNotPrepared = 64u;  // batch workspace prepared for other networks
constexpr unsigned kStWaveItems = 128u;   // a wave holds more work items than its buffers

// ---- control block (first bytes of the workspace) ---------------------------
struct Ctrl {
  unsigned int status;
  unsigned int pad0;
  unsigned long long key_or;    // OR of all sort keys (constant-digit detection)
  unsigned long long key_and;   // AND of all sort keys
  long long num_segments;       // rows of the segment table (S)
  unsigned long long ticket;    // walk work-queue ticket
  unsigned long long stage_used;      // staging entries handed out
  unsigned long long overflow_count;  // items re-walked by the overflow kernel
  long long out_base;           // edges emitted by earlier sample chunks
  long long out_end;            // edges emitted including the current chunk
  unsigned long long stats[MH_NUM_STATS];  // MH_STAT_* counters
  unsigned long long ticket2;   // batched waves: work-queue ticket of the UECM walk
  long long wave_items;         // batched waves: work items of the wave
  long long model_items[2];     // batched waves: work items of the UBCM / UECM queues
  long long sym_len;            // symmetric CSR: edges of the chunk that fit the capacity
  long long sym_base;           // symmetric CSR: first index entry of the chunk (2 x its first edge)
};

// ---- tuning constants --------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortThreads * kSortIPT;  // keys per sort tile
constexpr int kMergeMaxTiles = 32;                  // tile sorts + merge up to this many tiles
// Node sets sorted by tile sorts + merge, which also leave the suffix top-2 of y.
__host__ __device__ inline bool merge_sorted(int64_t n) { return (n + kSortTile - 1) / kSortTile <= kMergeMaxTiles; }
constexpr int kScanThreads = 256;
constexpr int kScanIPT = 8;
constexpr int kScanTile = kScanThreads * kScanIPT;
constexpr int kWalkWarps = 8;                    // warps per walk block
constexpr int kSlot = 48;                        // edges a lane buffers in shared memory
constexpr int kSlotStride = kSlot + 1;           // padded to spread banks
constexpr int kFlushMin = 8;                     // walk: finished runs a warp gathers before it flushes them
constexpr int kMaxWalkWarps = 8192;              // cap on resident walk warps (staging slack)
constexpr int kStageChunk = 1024;                // staging entries a warp reserves at a time
constexpr int kEmitWarps = 8;                   // emit: warps per block
constexpr int kEmitGroup = 32;                  // emit: work items a warp takes at a time (one per lane)
constexpr long long kItemChunk = 1ll << 22;      // work items per sample chunk
constexpr int kDefaultSegTarget = 32;

// ---- workspace layout --------------------------------------------------------
struct Layout {
  int64_t n = 0, rows = 0, tiles = 0, max_segments = 0, spc = 0, items_max = 0, capacity = 0;
  bool bip = false;
  // bipartite rows (the + set): arrays of the sorted rows, scratch for the
  // row set's own cost prefix and bounds (unused), the directed exclusions
  size_t perm_r = 0, rank_r = 0, xs_r = 0, ys_r = 0, as_r = 0, xdf_r = 0, adf_r = 0, ydf_r = 0, lny_r = 0,
         Q_r = 0, top_r = 0, excl = 0;
  size_t ctrl = 0, keys0 = 0, keys1 = 0, vals0 = 0, vals1 = 0, hist = 0, perm = 0, rank = 0, xs = 0, ys = 0,
         as = 0, top1 = 0, Q = 0, rowoff = 0, seg = 0, item_cnt = 0, item_base = 0,
         item_off = 0, sample_counts = 0, staging = 0, xdf = 0, adf = 0, ydf = 0, lny = 0,
         seg_c = 0, seg_cf = 0, ghist = 0, sort_state = 0, sort_counters = 0, scan_flags = 0,
         scan_values = 0, scan_counters = 0, zero_begin = 0, zero_end = 0, tsuf = 0, tsuf2 = 0, total = 0;
  // symmetric CSR scratch (MH_CSR_SYMMETRIC): (sample, rank) keys and
  // positions of the chunk's edges, their sources and weights in output
  // order, per-(sample, rank) counts of edges arriving at a node, and the
  // histograms of the key sort
  size_t sym_k0 = 0, sym_k1 = 0, sym_v0 = 0, sym_v1 = 0, sym_src = 0, sym_w = 0, sym_rev = 0, sym_hist = 0;
  // CSR-only output of a one-set network: work items numbered (sample, node
  // id, segment) through these maps (0 when not allocated)
  size_t rowoff_node = 0, seg_slot = 0, slot_ik = 0;
  int64_t sym_tiles = 0;
  int64_t scan_tiles = 0;
  int64_t staging_entries = 0;
};

Layout make_layout(int model, int64_t n, const mh_params& p, int64_t capacity);
// Bipartite: rows = the + set (n_plus), candidates = the - set (n_minus).
Layout make_layout_bip(int model, int64_t n_plus, int64_t n_minus, const mh_params& p, int64_t capacity);

struct Top2 {
  double a, b;  // largest and second largest
};
struct LnEntry;  // logarithm table entry (walk_math.cuh)

// Device views of the workspace.
struct Net {
  int model;
  uint32_t flags;
  int64_t n;
  const double* x;  // original order
  const double* y;
  int32_t* perm;    // rank -> id
  int32_t* rank;    // id -> rank
  double* xs;
  double* ys;
  double* as;
  Top2* top;        // [n+1]: two largest y among ranks >= i (top[i].a = suffix max)
  unsigned long long* Q;  // [n+1] proxy prefix sums
  long long* rowoff;      // [n+1] first segment of each row; rowoff[n] = S
  int4* seg;              // {row, k, a, b}
  double* seg_c;          // UECM: bound constant c of each segment
  float4* seg_cf;         // UECM: (1/(1-c) hi, lo, 1-c, 0) of each segment
  float2* xdf;            // x_s as double-float (hi, lo)
  float2* adf;            // a_s = x_s y_s as double-float (UECM)
  float2* ydf;            // y_s as double-float (UECM)
  float2* lny;            // ln y_s as double-float (UECM weights)
  LnEntry* lntab;         // logarithm table (kLnTable entries, one per device)
  int64_t max_segments;
  int seg_target;
  // Rows.  One node set: the same nodes and arrays as the candidates, row i
  // walking candidates [i+1, n).  Bipartite (Sec. 2.6): the + set, in its own
  // rank order, each row walking all candidates [0, n) of the - set.
  int64_t rows;
  bool bip;
  const double* x_r;      // row parameters in original order
  const double* y_r;
  int32_t* excl;          // directed: the candidate rank row i skips (its own in-copy), else NULL
  int32_t* perm_r;        // row rank -> row id
  int32_t* rank_r;        // row id -> row rank
  double* xs_r;
  double* ys_r;
  double* as_r;
  float2* xdf_r;
  float2* adf_r;
  float2* ydf_r;
  float2* lny_r;
};

// First candidate of row i.
__host__ __device__ inline int64_t row_start(const Net& g, int64_t i) { return g.bip ? 0 : i + 1; }

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned long long p0 = static_cast<unsigned long long>(0xD2511F53u) * c.x;  // one wide multiply
    const unsigned long long p1 = static_cast<unsigned long long>(0xCD9E8D57u) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0, static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1, static_cast<uint32_t>(p0));
  }
  return c;
}

// Round keys of Philox4x32-10 (k_r = k + r W, mod 2^32, r = 0..9), set once
// per launch so that a round reads its key as a kernel parameter.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
inline PhiloxKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys r;
  for (int i = 0; i < 10; ++i) {
    r.k0[i] = k0 + static_cast<uint32_t>(i) * 0x9E3779B9u;
    r.k1[i] = k1 + static_cast<uint32_t>(i) * 0xBB67AE85u;
  }
  return r;
}
// philox4x32_10 with the round keys of word 0 precomputed, and of word 1
// too (kK1 = true) or from a per-lane key k1 (batched networks).
template <bool kK1>
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const PhiloxKeys& rk, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (!kK1 && round) k1 += 0xBB67AE85u;
    const uint32_t kr1 = kK1 ? rk.k1[round] : k1;
    const unsigned long long p0 = static_cast<unsigned long long>(0xD2511F53u) * c.x;
    const unsigned long long p1 = static_cast<unsigned long long>(0xCD9E8D57u) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ rk.k0[round], static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ kr1, static_cast<uint32_t>(p0));
  }
  return c;
}

// 53 bits -> (0, 1] (logarithm inputs) and [0, 1) (acceptance draws).
__device__ __forceinline__ unsigned long long top53(uint32_t hi, uint32_t lo) {
  return ((static_cast<unsigned long long>(hi) << 32) | lo) >> 11;
}
__device__ __forceinline__ double unit_open0(uint32_t hi, uint32_t lo) {
  return static_cast<double>(top53(hi, lo) + 1ull) * 0x1p-53;
}
__device__ __forceinline__ double unit_open1(uint32_t hi, uint32_t lo) {
  return static_cast<double>(top53(hi, lo)) * 0x1p-53;
}

// Fixed-point scale of the segment-cost prefix sums: n * min(vmax, 2^20) * 2^F < 2^62.
__host__ __device__ inline int proxy_scale(double vmax, int64_t n) {
  if (vmax > 0x1p20) vmax = 0x1p20;
  unsigned long long bits;
  memcpy(&bits, &vmax, sizeof(bits));
  int E = static_cast<int>((bits >> 52) & 0x7FF) - 1022;
  if (E < 1) E = 1;
  int len = 0;
  for (unsigned long long v = static_cast<unsigned long long>(n); v; v >>= 1) ++len;
  int F = 62 - len - E;
  return F < 0 ? 0 : F;
}

// ---- host helpers ------------------------------------------------------------------
void set_error(const char* fmt, ...);
void note_launches(int count);  // counts kernels launched by the current call
inline unsigned grid_for(int64_t work, int per_block, unsigned cap = 1u << 30) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<unsigned>(g);
}
int sm_count();

// Launchers (return cudaError_t of the launch).
cudaError_t launch_validate_keys(const Net& g, unsigned long long* keys, int32_t* vals, unsigned* ghist, Ctrl* ctrl,
                                 cudaStream_t s);
cudaError_t launch_sort(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_gather(const Net& g, const int32_t* sorted_vals, Ctrl* ctrl, cudaStream_t s);
// Sets of at most kMergeMaxTiles tiles: validation, tile sorts, then merge by
// rank and gather (two launches); also clears the single-pass scan states.
cudaError_t launch_sort_merge(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s);
cudaError_t sort_kernel_attributes(int dev);  // before any capture
// Device copy of the logarithm table of the current device, built on first
// use (a launch and a synchronisation: never while a stream is captured);
// NULL if it could not be built.
LnEntry* ln_table_ptr(cudaStream_t s = nullptr);  // per-device table, built on first use
cudaError_t launch_first_level_probe(const unsigned long long* N, const double* z, const int32_t* room, long long n,
                                     float* E_out, float* lam_out, int32_t* fl_out, cudaStream_t s);
// Stable LSD sort of `len` (key, value) pairs on the 8-bit digits at the
// given shifts, `*dev_len` of them (at most host_len) present; the result
// is in buffer 0 or 1 as returned through *out_buf.  `st` is the scan state.
cudaError_t launch_pair_sort(unsigned long long* keys[2], int32_t* vals[2], int64_t host_len,
                             const long long* dev_len, const int* shifts, int passes, unsigned* hist,
                             const void* scan_state, Ctrl* ctrl, int* out_buf, cudaStream_t s);
cudaError_t launch_bounds_and_partition(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s);
struct ScanState;
// Node-id order of a one-set network's work items (CSR-only output): the
// exclusive scan over node ids of each row's segment count (rows + 1
// entries), each table row's slot and each slot's (row rank, segment index).
cudaError_t launch_node_order(const Net& g, Ctrl* ctrl, long long* rowoff_node, int32_t* seg_slot, int2* slot_ik,
                              const ScanState& st, cudaStream_t s);
cudaError_t launch_exclusions(const Net& g, cudaStream_t s);  // directed: excl[i] = rank of row i's own node

// Device scratch of the symmetric CSR layout (all NULL when it is off).
struct SymArgs {
  unsigned long long* keys[2];  // (sample in chunk << 32) | rank of the lower-ranked endpoint
  int32_t* vals[2];             // the edge's position within the chunk
  int32_t* src;                 // by position: the higher-ranked endpoint's id
  int32_t* w;                   // by position: the weight (1 for UBCM)
  long long* rev;               // [chunk samples][n + 1]: edges arriving at each rank, then its exclusive scan
  unsigned* hist;               // radix histograms, 256 x tiles
  int64_t tiles;                // key-sort tiles for capacity_edges keys
};

struct ChunkArgs {
  int64_t chunk_first;  // index of the chunk's first sample within the call
  int64_t chunk_samples;
  uint32_t sample0;     // global sample id of the chunk's first sample
  uint32_t key0, key1;
  int32_t* item_cnt;     // edges of each work item (< 2^31: a run fits int32 staging positions)
  long long* item_base;
  long long* item_off;
  int32_t* staging;
  long long* sample_counts;
  void* scan_state;  // ScanState of the single-pass scans
  int64_t staging_cap;
  int64_t items_max;
  // node-order CSR: each table row's slot, each slot's (row rank, segment
  // index), and the exclusive scan over node ids of each row's segment count
  // (all NULL: items in (sample, rank, segment) order)
  const int32_t* seg_slot = nullptr;
  const int2* slot_ik = nullptr;
  const long long* rowoff_node = nullptr;
  int walk_ctas_per_sm;  // 0: as many walk blocks per SM as fit
  SymArgs sym{};         // symmetric CSR scratch, when requested
};
struct Outputs {
  int32_t* src;
  int32_t* dst;
  int32_t* w;
  long long* csr_off;
  int32_t* csr_idx;
  int32_t* csr_w;
  int64_t capacity;
};
cudaError_t launch_walk(const Net& g, const ChunkArgs& c, Ctrl* ctrl, cudaStream_t s);

// ---- batched ensembles (batch.cu) ------------------------------------------------
// Static data of one network of a batch.  Its per-node arrays are slices of
// concatenated arrays: ranks of network t occupy [node_base, node_base + n)
// of xs, as, ys, xdf, adf, ydf, lny, perm (local ids) and rank (local ranks);
// its (n+1)-long arrays (top, Q, rowoff) start at node1_base and its segment
// table rows (local coordinates) at seg_base.
struct BatchNet {
  long long node_base;
  long long node1_base;
  long long seg_base;
  long long max_segments;
  int n;
  int model;
};
// One network's share of a wave: host part first, then what the plan kernel
// derives from the prepared segment counts.
struct WaveNet {
  long long pair_base;   // index of the network's first pair within the wave
  long long csr_base;    // first CSR offset entry of that pair
  uint32_t sample_lo;    // sample id of that pair
  uint32_t sample_cnt;   // pairs of this network in the wave (0: none)
  uint32_t key1;         // Philox key word 1
  uint32_t pad;
  long long S;           // segment-table rows (device)
  long long item_begin;  // first work item of the network in the wave (device)
};
// What a batched walk launch reads besides the concatenated arrays.
struct BatchQueue {
  const BatchNet* nets;
  const WaveNet* wave;
  const int32_t* order;   // networks of the launch's model, ascending
  const long long* mb;    // [n_order + 1]: first queue position of each
  int n_order;
  unsigned long long* ticket;
  const long long* total;  // queue length
  // CSR waves: the slot of each segment-table row among its network's rows
  // in node-id order (work items numbered (sample, node id, segment)); NULL
  // numbers them (sample, rank, segment)
  const int32_t* seg_slot;
};
cudaError_t launch_walk_batched(const Net& g, const ChunkArgs& c, const BatchQueue& q, Ctrl* ctrl, int model,
                                cudaStream_t s);
cudaError_t prepare_kernel_attributes(int model);  // before any capture
cudaError_t launch_emit(const Net& g, const ChunkArgs& c, const Outputs& o, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_export_table(const Net& g, const Ctrl* ctrl, int32_t* row, int32_t* k, int64_t* a, int64_t* b,
                                int64_t cap, cudaStream_t s);

// Existing sampling steps, reachable from the fixed-scratch entry point.
int check_sample_params(int model, int64_t n, const mh_params* p);
int64_t take_launch_count();                          // kernels launched since the last call (and resets)
void record_call_info(const mh_call_info& info);      // what mh_last_call_info returns
Net net_view(int model, const mh_params& p, const double* x, const double* y, int64_t n, const Layout& L,
             char* ws);
int enqueue_sample_direct(const Net& g, const Layout& L, char* ws, const mh_params* p, const Outputs& o, char* hbuf,
                          cudaStream_t s);
int status_code(unsigned status, long long num_segments, int64_t max_segments);

// Rows [row_begin, row_begin + rows) of the expected sums (outputs indexed from
// row_begin); rows >= 1 and row_begin + rows <= n.
cudaError_t launch_expected_fwd(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                int64_t rows, double* k, double* s, cudaStream_t st);
cudaError_t launch_expected_bwd(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                int64_t rows, const double* gk, const double* gs, double* gx, double* gy,
                                cudaStream_t st);
// Symmetric pair sums (pairsym.cu): kind 0 the expected sums, 1 the Jacobian
// diagonal, 2 the gradient; outputs as the row kernels' whole-range calls.
size_t expected_sym_workspace_bytes(int model, int64_t n);
cudaError_t launch_expected_sym(int kind, int model, const double* x, const double* y, const double* gk,
                                const double* gs, int64_t n, void* workspace, double* o0, double* o1, double* o2,
                                double* o3, cudaStream_t st);

}  // namespace mh
