// C ABI entry points (include/maxent_mh.h).
//
// A sampling call runs, in stream order and without a host round trip until
// the end:  validate + sort keys and copy the parameters into rank order
// (sort.cu) -> bound prep + segment table (partition.cu) -> per sample chunk:
// walk (walk.cu) -> item scan + emit (emit.cu).  It then copies the status
// word, the counters and the per-sample edge counts to a pinned host buffer,
// synchronises the stream and maps the status to a code.  A call repeated
// with the same arguments replays a captured CUDA graph.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mh_internal.cuh"
#include "scan.cuh"

namespace mh {
// Diagonal of the Jacobian of the expected sums, rows [row_begin, row_begin +
// rows) (pairwise.cu); used by this file only.
cudaError_t launch_expected_jacobian_diag(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                          int64_t rows, double* dk_dx, double* dk_dy, double* ds_dx, double* ds_dy,
                                          cudaStream_t st);
}  // namespace mh

namespace mh {

namespace {

thread_local char g_detail[512] = "";
thread_local mh_call_info g_info = {0, 0, 0, 0.0, 0.0, 0.0, 0.0};
thread_local int64_t g_launches = 0;

// CUDA events of a timed call: start, after prepare, then (before walk,
// after walk, after emit) per chunk.  Created on first use, per thread.
constexpr int64_t kTimedChunks = 1024;  // MH_TIMING covers calls of at most this many sample chunks

struct CallTimer {
  static constexpr int kMax = 2 + 3 * kTimedChunks;
  cudaEvent_t ev[kMax] = {};
  bool ready = false;
  int used = 0;
  bool on = false;
  cudaError_t create() {  // outside any capture
    if (!ready) {
      for (int t = 0; t < kMax; ++t) {
        cudaError_t e = cudaEventCreate(&ev[t]);
        if (e != cudaSuccess) return e;
      }
      ready = true;
    }
    return cudaSuccess;
  }
  cudaError_t start(bool enable, cudaStream_t s) {
    on = enable;
    used = 0;
    if (!on) return cudaSuccess;
    cudaError_t e = create();
    if (e != cudaSuccess) return e;
    return mark(s);
  }
  cudaError_t mark(cudaStream_t s) {
    if (!on || used >= kMax) return cudaSuccess;
    // inside a capture the record must become a graph node of its own
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &st);
    if (e != cudaSuccess) return e;
    if (st == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev[used++], s, cudaEventRecordExternal);
    return cudaEventRecord(ev[used++], s);
  }
  float between(int a, int b) const {
    float ms = 0.f;
    if (a < used && b < used) cudaEventElapsedTime(&ms, ev[a], ev[b]);
    return ms;
  }
};
thread_local CallTimer g_timer;

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

struct PinnedBuffer {
  void* ptr = nullptr;
  size_t bytes = 0;
  ~PinnedBuffer() {
    if (ptr) cudaFreeHost(ptr);
  }
  cudaError_t reserve(size_t want) {
    if (want <= bytes) return cudaSuccess;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaHostAlloc(&ptr, want, cudaHostAllocDefault);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
};
thread_local PinnedBuffer g_pinned;

constexpr uint32_t kKnownFlags =
    MH_OUT_COO | MH_OUT_CSR | MH_BOUND_PAPER | MH_INIT_PREV | MH_DIRECTED | MH_CSR_SYMMETRIC | MH_FP64_ONLY |
    MH_TIMING | MH_TEST_WAIT_TIMEOUT | MH_CHUNG_LU;

}  // namespace

void note_launches(int count) { g_launches += count; }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}

static int64_t default_max_segments(int64_t n) { return 4 * n + 1024; }

// Rows and candidates: one node set (rows = n, bip = false) or a bipartite
// network (rows = the + set, candidates = the - set).
static Layout make_layout_impl(int model, int64_t rows, int64_t n, bool bip, const mh_params& p, int64_t capacity) {
  (void)model;
  Layout L;
  L.n = n;
  L.rows = rows;
  L.bip = bip;
  const int64_t nmax = rows > n ? rows : n;
  L.tiles = (nmax + kSortTile - 1) / kSortTile;
  L.max_segments = p.max_segments > 0 ? p.max_segments : default_max_segments(rows);
  int64_t spc = kItemChunk / L.max_segments;
  if (spc < 1) spc = 1;
  if (spc > static_cast<int64_t>(p.num_samples)) spc = p.num_samples;
  L.spc = spc;
  L.items_max = spc * L.max_segments;
  L.capacity = capacity;
  int64_t scan_len = 256 * L.tiles;
  if (n + 1 > scan_len) scan_len = n + 1;
  if (rows + 1 > scan_len) scan_len = rows + 1;
  if (L.items_max + 1 > scan_len) scan_len = L.items_max + 1;
  if (spc * (rows + 1) > scan_len) scan_len = spc * (rows + 1);
  const bool sym = (p.flags & MH_CSR_SYMMETRIC) != 0 && !bip;
  if (sym) {
    L.sym_tiles = (capacity + kSortTile - 1) / kSortTile > 0 ? (capacity + kSortTile - 1) / kSortTile : 1;
    if (256 * L.sym_tiles > scan_len) scan_len = 256 * L.sym_tiles;
  }
  const size_t n1 = static_cast<size_t>(n) + 1, r1 = static_cast<size_t>(rows) + 1, nm = static_cast<size_t>(nmax);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  L.ctrl = take(sizeof(Ctrl));
  L.keys0 = take(8 * nm);
  L.keys1 = take(8 * nm);
  L.vals0 = take(4 * nm);
  L.vals1 = take(4 * nm);
  L.tsuf = take(sizeof(Top2) * nm);
  L.tsuf2 = take(sizeof(Top2) * nm);
  L.hist = take(4 * 256 * static_cast<size_t>(L.tiles));
  L.perm = take(4 * static_cast<size_t>(n));
  L.rank = take(4 * static_cast<size_t>(n));
  L.xs = take(8 * static_cast<size_t>(n));
  L.ys = take(8 * static_cast<size_t>(n));
  L.as = take(8 * static_cast<size_t>(n));
  L.top1 = take(sizeof(Top2) * n1);
  L.Q = take(8 * n1);
  L.rowoff = take(8 * r1);
  L.seg = take(sizeof(int4) * static_cast<size_t>(L.max_segments));
  L.item_cnt = take(4 * static_cast<size_t>(L.items_max));
  L.item_base = take(8 * static_cast<size_t>(L.items_max));
  L.item_off = take(8 * (static_cast<size_t>(L.items_max) + 1));
  L.sample_counts = take(8 * static_cast<size_t>(p.num_samples));
  // Warps reserve staging in chunks of kStageChunk entries; a chunk switch
  // leaves fewer than kSlot entries behind and a warp's last chunk may be
  // partly unused, so staging holds capacity + capacity / 16 + the chunks.
  L.staging_entries = capacity + capacity / 16 + static_cast<int64_t>(kMaxWalkWarps) * (kStageChunk + kSlot);
  L.staging = take(4 * static_cast<size_t>(L.staging_entries));
  L.xdf = take(8 * static_cast<size_t>(n));
  L.adf = take(8 * static_cast<size_t>(n));
  L.ydf = take(8 * static_cast<size_t>(n));
  L.lny = take(8 * static_cast<size_t>(n));
  L.seg_c = take(8 * static_cast<size_t>(L.max_segments));
  L.seg_cf = take(16 * static_cast<size_t>(L.max_segments));
  // CSR-only output of a one-set network numbers its work items by node id
  // (the item scan then gives every edge its CSR position)
  if ((p.flags & MH_OUT_CSR) && !(p.flags & MH_OUT_COO) && !sym && !bip) {
    L.rowoff_node = take(8 * r1);
    L.seg_slot = take(4 * static_cast<size_t>(L.max_segments));
    L.slot_ik = take(8 * static_cast<size_t>(L.max_segments));
  }
  if (bip) {
    const size_t r = static_cast<size_t>(rows);
    L.perm_r = take(4 * r);
    L.rank_r = take(4 * r);
    L.xs_r = take(8 * r);
    L.ys_r = take(8 * r);
    L.as_r = take(8 * r);
    L.xdf_r = take(8 * r);
    L.adf_r = take(8 * r);
    L.ydf_r = take(8 * r);
    L.lny_r = take(8 * r);
    L.Q_r = take(8 * r1);
    L.top_r = take(sizeof(Top2) * r1);
    L.excl = take(4 * r);
  }
  if (sym) {
    const size_t c = static_cast<size_t>(capacity > 0 ? capacity : 1);
    L.sym_k0 = take(8 * c);
    L.sym_k1 = take(8 * c);
    L.sym_v0 = take(4 * c);
    L.sym_v1 = take(4 * c);
    L.sym_src = take(4 * c);
    L.sym_w = take(4 * c);
    L.sym_rev = take(8 * static_cast<size_t>(spc) * r1);
    L.sym_hist = take(4 * 256 * static_cast<size_t>(L.sym_tiles));
  }
  // states of the single-pass scans and of the one-sweep sort, cleared by one
  // memset per sort (the kernels leave them cleared)
  L.scan_tiles = scan_len / kScanTile + 2;
  L.zero_begin = off;
  L.ghist = take(4 * 8 * 256);
  L.sort_counters = take(16);
  L.sort_state = take(2 * 8 * 256 * static_cast<size_t>(L.tiles > 0 ? L.tiles : 1));
  L.scan_counters = take(16);
  L.scan_flags = take(4 * static_cast<size_t>(L.scan_tiles));
  L.zero_end = off;
  L.scan_values = take(2 * sizeof(Top2) * static_cast<size_t>(L.scan_tiles));
  L.total = off;
  return L;
}

Layout make_layout(int model, int64_t n, const mh_params& p, int64_t capacity) {
  return make_layout_impl(model, n, n, false, p, capacity);
}

Layout make_layout_bip(int model, int64_t n_plus, int64_t n_minus, const mh_params& p, int64_t capacity) {
  return make_layout_impl(model, n_plus, n_minus, true, p, capacity);
}

static Net make_net(int model, const mh_params& p, const double* x, const double* y, int64_t n, const Layout& L,
                    char* ws) {
  Net g;
  g.model = model;
  g.flags = p.flags;
  g.n = n;
  g.x = x;
  g.y = y;
  g.perm = reinterpret_cast<int32_t*>(ws + L.perm);
  g.rank = reinterpret_cast<int32_t*>(ws + L.rank);
  g.xs = reinterpret_cast<double*>(ws + L.xs);
  g.ys = reinterpret_cast<double*>(ws + L.ys);
  g.as = (model == MH_UECM) ? reinterpret_cast<double*>(ws + L.as) : g.xs;
  g.top = reinterpret_cast<Top2*>(ws + L.top1);
  g.Q = reinterpret_cast<unsigned long long*>(ws + L.Q);
  g.rowoff = reinterpret_cast<long long*>(ws + L.rowoff);
  g.seg = reinterpret_cast<int4*>(ws + L.seg);
  g.seg_c = reinterpret_cast<double*>(ws + L.seg_c);
  g.seg_cf = reinterpret_cast<float4*>(ws + L.seg_cf);
  g.xdf = reinterpret_cast<float2*>(ws + L.xdf);
  g.adf = (model == MH_UECM) ? reinterpret_cast<float2*>(ws + L.adf) : g.xdf;
  g.ydf = reinterpret_cast<float2*>(ws + L.ydf);
  g.lny = reinterpret_cast<float2*>(ws + L.lny);
  g.lntab = ln_table_ptr();
  g.max_segments = L.max_segments;
  g.seg_target = p.seg_target ? static_cast<int>(p.seg_target) : kDefaultSegTarget;
  g.rows = L.rows;
  g.bip = L.bip;
  g.excl = nullptr;
  if (!L.bip) {
    g.x_r = g.x;
    g.y_r = g.y;
    g.perm_r = g.perm;
    g.rank_r = g.rank;
    g.xs_r = g.xs;
    g.ys_r = g.ys;
    g.as_r = g.as;
    g.xdf_r = g.xdf;
    g.adf_r = g.adf;
    g.ydf_r = g.ydf;
    g.lny_r = g.lny;
  } else {
    g.perm_r = reinterpret_cast<int32_t*>(ws + L.perm_r);
    g.rank_r = reinterpret_cast<int32_t*>(ws + L.rank_r);
    g.xs_r = reinterpret_cast<double*>(ws + L.xs_r);
    g.ys_r = reinterpret_cast<double*>(ws + L.ys_r);
    g.as_r = (model == MH_UECM) ? reinterpret_cast<double*>(ws + L.as_r) : g.xs_r;
    g.xdf_r = reinterpret_cast<float2*>(ws + L.xdf_r);
    g.adf_r = (model == MH_UECM) ? reinterpret_cast<float2*>(ws + L.adf_r) : g.xdf_r;
    g.ydf_r = reinterpret_cast<float2*>(ws + L.ydf_r);
    g.lny_r = reinterpret_cast<float2*>(ws + L.lny_r);
    if (p.flags & MH_DIRECTED) g.excl = reinterpret_cast<int32_t*>(ws + L.excl);
  }
  return g;
}

// The rows of a bipartite network as a one-set view, for their sort and gather.
static Net row_view(const Net& g, const Layout& L, char* ws) {
  Net r = g;
  r.n = g.rows;
  r.x = g.x_r;
  r.y = g.y_r;
  r.perm = g.perm_r;
  r.rank = g.rank_r;
  r.xs = g.xs_r;
  r.ys = g.ys_r;
  r.as = g.as_r;
  r.xdf = g.xdf_r;
  r.adf = g.adf_r;
  r.ydf = g.ydf_r;
  r.lny = g.lny_r;
  r.Q = reinterpret_cast<unsigned long long*>(ws + L.Q_r);
  r.top = reinterpret_cast<Top2*>(ws + L.top_r);
  r.bip = false;
  r.rows = g.rows;
  return r;
}

static int check_params_impl(int model, int64_t rows, int64_t n, bool bip, const mh_params* p) {
  if (model != MH_UBCM && model != MH_UECM) {
    set_error("model must be MH_UBCM or MH_UECM (got %d)", model);
    return MH_ERR_ARG;
  }
  if (!p) {
    set_error("params is NULL");
    return MH_ERR_ARG;
  }
  if (n < 1 || n > 0x7FFFFFFEll || rows < 1 || rows > 0x7FFFFFFEll) {
    set_error("node counts must be in [1, 2^31 - 2] (got %lld and %lld)", static_cast<long long>(rows),
              static_cast<long long>(n));
    return MH_ERR_ARG;
  }
  if (p->num_samples < 1) {
    set_error("num_samples must be >= 1");
    return MH_ERR_ARG;
  }
  if (static_cast<uint64_t>(p->sample_begin) + p->num_samples > 0xFFFFFFFFull) {
    set_error("sample_begin + num_samples exceeds 2^32 - 1");
    return MH_ERR_ARG;
  }
  if (p->seg_target == 1 || p->seg_target > (1u << 30)) {
    set_error("seg_target must be 0 (default) or in [2, 2^30] (got %u)", p->seg_target);
    return MH_ERR_ARG;
  }
  if (p->flags & ~kKnownFlags) {
    set_error("unknown flag bits 0x%x", p->flags & ~kKnownFlags);
    return MH_ERR_ARG;
  }
  if (!bip && (p->flags & MH_DIRECTED)) {
    set_error("MH_DIRECTED applies to mh_sample_bipartite only");
    return MH_ERR_ARG;
  }
  if ((p->flags & MH_CSR_SYMMETRIC) && (bip || !(p->flags & MH_OUT_CSR))) {
    set_error("MH_CSR_SYMMETRIC needs MH_OUT_CSR and one node set (mh_sample_ubcm / mh_sample_weighted)");
    return MH_ERR_ARG;
  }
  if ((p->flags & MH_CHUNG_LU) && (model != MH_UBCM || bip)) {
    set_error("MH_CHUNG_LU applies to one-set MH_UBCM calls only");
    return MH_ERR_ARG;
  }
  if (bip && (p->flags & (MH_BOUND_PAPER | MH_INIT_PREV))) {
    set_error("MH_BOUND_PAPER and MH_INIT_PREV do not apply to bipartite networks");
    return MH_ERR_ARG;
  }
  if (bip && (p->flags & MH_DIRECTED) && rows != n) {
    set_error("a directed network needs n_plus == n_minus (got %lld and %lld)", static_cast<long long>(rows),
              static_cast<long long>(n));
    return MH_ERR_ARG;
  }
  if (p->walk_ctas_per_sm > 64 || p->max_segments < 0) {
    set_error("walk_ctas_per_sm must be at most 64 and max_segments >= 0");
    return MH_ERR_ARG;
  }
  const int64_t least = bip ? rows : n - 1;  // every row with candidates has a segment
  if (p->max_segments > 0 && p->max_segments < least) {
    set_error("max_segments must be 0 or >= %lld", static_cast<long long>(least));
    return MH_ERR_ARG;
  }
  if (p->max_segments >= (1ll << 31) || (p->max_segments == 0 && default_max_segments(rows) >= (1ll << 31))) {
    set_error("the segment table would exceed 2^31 rows");
    return MH_ERR_ARG;
  }
  return MH_OK;
}

static int check_params(int model, int64_t n, const mh_params* p) { return check_params_impl(model, n, n, false, p); }

#define MH_CUDA(expr)                                                             \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error("%s failed: %s", #expr, cudaGetErrorString(e_));                  \
      return MH_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)

// Sort, gather, bound prep and segment table into the workspace.
// Validation, sort and gather of one node set (g.n nodes).
static int sort_set(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  if (merge_sorted(g.n)) {
    MH_CUDA(launch_sort_merge(g, L, ws, ctrl, s));
    return MH_OK;
  }
  MH_CUDA(cudaMemsetAsync(&ctrl->key_or, 0, sizeof(ctrl->key_or), s));
  MH_CUDA(cudaMemsetAsync(&ctrl->key_and, 0xFF, sizeof(ctrl->key_and), s));
  MH_CUDA(cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_end - L.zero_begin, s));
  Layout Ls = L;  // the sort's tiles follow this set's size
  Ls.tiles = (g.n + kSortTile - 1) / kSortTile;
  auto* keys0 = reinterpret_cast<unsigned long long*>(ws + L.keys0);
  auto* vals0 = reinterpret_cast<int32_t*>(ws + L.vals0);
  MH_CUDA(launch_validate_keys(g, keys0, vals0, reinterpret_cast<unsigned*>(ws + L.ghist), ctrl, s));
  MH_CUDA(launch_sort(g, Ls, ws, ctrl, s));
  MH_CUDA(launch_gather(g, vals0, ctrl, s));
  return MH_OK;
}

static int prepare(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  MH_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
  int rc = sort_set(g, L, ws, ctrl, s);  // the candidates (the - set when bipartite)
  if (rc != MH_OK) return rc;
  if (g.bip) {
    rc = sort_set(row_view(g, L, ws), L, ws, ctrl, s);  // the rows (the + set)
    if (rc != MH_OK) return rc;
    if (g.excl) MH_CUDA(launch_exclusions(g, s));
  }
  MH_CUDA(launch_bounds_and_partition(g, L, ws, ctrl, s));
  return MH_OK;
}

static int status_to_code(unsigned status, long long num_segments, int64_t max_segments) {
  if (status & kStDomain) {
    set_error("x must be finite, >= 0 and <= 1e150; y must be in [0, 1)");
    return MH_ERR_DOMAIN;
  }
  if (status & kStSegments) {
    set_error("segment table needs %lld rows, max_segments is %lld", num_segments,
              static_cast<long long>(max_segments));
    return MH_ERR_WORKSPACE;
  }
  if (status & kStInternal) {
    set_error("internal consistency check failed on the device");
    return MH_ERR_CUDA;
  }
  if (status & kStTimeout) {
    set_error("a bounded device wait gave up");
    return MH_ERR_DEVICE_TIMEOUT;
  }
  if (status & kStOverflow) {
    set_error("a sampled weight exceeds INT32_MAX");
    return MH_ERR_OVERFLOW;
  }
  return MH_OK;
}

// A range [begin, end) of segment-table rows that a call walks (end < 0: all).
struct SegRange {
  int64_t begin = 0, end = -1;
  bool all() const { return end < 0; }
};

// Narrows the walked table to rows [a, b) of the one the partition wrote:
// the walk and the emit then see a table of b - a rows starting at row a
// (their table pointers are offset by a on the host).  A truncated table
// (more rows than max_segments) is left as it is, so the call fails as usual.
__global__ void seg_range_kernel(Ctrl* ctrl, long long a, long long b, long long max_segments) {
  const long long S = ctrl->num_segments;
  if (S > max_segments) return;
  const long long lo = a < S ? a : S, hi = b < S ? b : S;
  ctrl->num_segments = hi > lo ? hi - lo : 0;
}

// Everything a sampling call enqueues: prepare, then walk + emit per sample
// chunk, then the read-back of the control block and the per-sample counts
// into the pinned buffer `hbuf`.
static int enqueue_sample(const Net& g_full, const Layout& L, char* ws, const mh_params* p, const Outputs& o,
                          bool timed, char* hbuf, cudaStream_t s, SegRange range = SegRange{}) {
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  MH_CUDA(g_timer.start(timed, s));
  int rc = prepare(g_full, L, ws, ctrl, s);
  if (rc != MH_OK) return rc;
  Net g = g_full;
  if (!range.all()) {
    const int64_t a = range.begin < L.max_segments ? range.begin : L.max_segments;
    seg_range_kernel<<<1, 1, 0, s>>>(ctrl, a, range.end, L.max_segments);
    note_launches(1);
    MH_CUDA(cudaGetLastError());
    g.seg += a;
    if (g.seg_c) g.seg_c += a;
    if (g.seg_cf) g.seg_cf += a;
  }
  MH_CUDA(g_timer.mark(s));

  Outputs out = o;
  if (!(p->flags & MH_OUT_COO)) out.src = out.dst = out.w = nullptr;
  if (!(p->flags & MH_OUT_CSR)) out.csr_off = nullptr, out.csr_idx = nullptr, out.csr_w = nullptr;
  if (g.model == MH_UBCM) out.w = out.csr_w = nullptr;

  ChunkArgs c;
  c.key0 = static_cast<uint32_t>(p->seed);
  c.key1 = static_cast<uint32_t>(p->seed >> 32) + p->network_id;
  c.item_cnt = reinterpret_cast<int32_t*>(ws + L.item_cnt);
  c.item_base = reinterpret_cast<long long*>(ws + L.item_base);
  c.item_off = reinterpret_cast<long long*>(ws + L.item_off);
  c.staging = reinterpret_cast<int32_t*>(ws + L.staging);
  c.sample_counts = reinterpret_cast<long long*>(ws + L.sample_counts);
  const ScanState scan_state{reinterpret_cast<unsigned*>(ws + L.scan_flags), ws + L.scan_values,
                             reinterpret_cast<unsigned*>(ws + L.scan_counters), ctrl, L.scan_tiles,
                             (p->flags & MH_TEST_WAIT_TIMEOUT) ? kTestStuckPolls : 0u};
  c.scan_state = const_cast<ScanState*>(&scan_state);
  c.staging_cap = L.staging_entries;
  c.items_max = L.items_max;
  c.walk_ctas_per_sm = static_cast<int>(p->walk_ctas_per_sm);
  if (L.rowoff_node && range.all()) {
    long long* rn = reinterpret_cast<long long*>(ws + L.rowoff_node);
    int32_t* ss = reinterpret_cast<int32_t*>(ws + L.seg_slot);
    int2* ik = reinterpret_cast<int2*>(ws + L.slot_ik);
    MH_CUDA(launch_node_order(g, ctrl, rn, ss, ik, scan_state, s));
    c.seg_slot = ss;
    c.slot_ik = ik;
    c.rowoff_node = rn;
  }
  if (L.sym_rev) {
    c.sym.keys[0] = reinterpret_cast<unsigned long long*>(ws + L.sym_k0);
    c.sym.keys[1] = reinterpret_cast<unsigned long long*>(ws + L.sym_k1);
    c.sym.vals[0] = reinterpret_cast<int32_t*>(ws + L.sym_v0);
    c.sym.vals[1] = reinterpret_cast<int32_t*>(ws + L.sym_v1);
    c.sym.src = reinterpret_cast<int32_t*>(ws + L.sym_src);
    c.sym.w = reinterpret_cast<int32_t*>(ws + L.sym_w);
    c.sym.rev = reinterpret_cast<long long*>(ws + L.sym_rev);
    c.sym.hist = reinterpret_cast<unsigned*>(ws + L.sym_hist);
    c.sym.tiles = L.sym_tiles;
  }
  for (int64_t first = 0; first < static_cast<int64_t>(p->num_samples); first += L.spc) {
    const int64_t left = static_cast<int64_t>(p->num_samples) - first;
    c.chunk_first = first;
    c.chunk_samples = left < L.spc ? left : L.spc;
    c.sample0 = p->sample_begin + static_cast<uint32_t>(first);
    MH_CUDA(cudaMemsetAsync(&ctrl->ticket, 0, 3 * sizeof(unsigned long long), s));
    MH_CUDA(g_timer.mark(s));
    MH_CUDA(launch_walk(g, c, ctrl, s));
    MH_CUDA(g_timer.mark(s));
    MH_CUDA(launch_emit(g, c, out, ctrl, s));
    MH_CUDA(g_timer.mark(s));
  }
  const size_t counts_bytes = 8 * static_cast<size_t>(p->num_samples);
  MH_CUDA(cudaMemcpyAsync(hbuf, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  MH_CUDA(cudaMemcpyAsync(hbuf + sizeof(Ctrl), c.sample_counts, counts_bytes, cudaMemcpyDeviceToHost, s));
  return MH_OK;
}

// ---- graph cache --------------------------------------------------------------
// A call's kernel sequence depends only on its arguments, so a repeated call
// is captured into a CUDA graph (on a library-owned stream: the legacy
// default stream cannot be captured) and replayed on the caller's stream.
struct CallKey {
  int model, device;
  int64_t n, capacity, rows;
  const void *x, *y, *xr, *yr, *ws, *src, *dst, *w, *csr_off, *csr_idx, *csr_w, *hbuf;
  size_t ws_bytes;
  mh_params params;
  int64_t seg_begin, seg_end;
};
struct CachedGraph {
  CallKey key;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0, chunks = 0, timer_marks = 0;
  uint64_t last_use = 0;
};
constexpr int kGraphCache = 8;
constexpr int kSeenKeys = 16;
struct GraphCache {
  CachedGraph entries[kGraphCache];
  uint64_t clock = 0;
  cudaStream_t capture_stream[64] = {};
  unsigned long long seen[kSeenKeys] = {};
  int seen_next = 0;
  // A call is captured the second time its key is seen; one-off calls
  // launch directly, which costs less than a capture.
  bool seen_before(const CallKey& k) {
    unsigned long long h = 0xcbf29ce484222325ull;
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&k);
    for (size_t i = 0; i < sizeof(CallKey); ++i) {
      h ^= b[i];
      h *= 0x100000001b3ull;
    }
    h |= 1ull;
    for (auto v : seen)
      if (v == h) return true;
    seen[seen_next] = h;
    seen_next = (seen_next + 1) % kSeenKeys;
    return false;
  }
  ~GraphCache() { clear(); }
  void clear() {
    for (auto& e : entries)
      if (e.exec) {
        cudaGraphExecDestroy(e.exec);
        e.exec = nullptr;
      }
  }
  CachedGraph* find(const CallKey& k) {
    for (auto& e : entries)
      if (e.exec && memcmp(&e.key, &k, sizeof(CallKey)) == 0) {
        e.last_use = ++clock;
        return &e;
      }
    return nullptr;
  }
  CachedGraph* slot() {
    CachedGraph* v = &entries[0];
    for (auto& e : entries) {
      if (!e.exec) return &e;
      if (e.last_use < v->last_use) v = &e;
    }
    cudaGraphExecDestroy(v->exec);
    v->exec = nullptr;
    return v;
  }
};
thread_local GraphCache g_graphs;

// One sampling call: a single node set (xr == NULL) or a bipartite network
// whose rows are (xr, yr, rows) and candidates (x, y, n).
static int run_sample(int model, const double* x, const double* y, int64_t n, const mh_params* p, void* workspace,
                      size_t workspace_bytes, const Outputs& o, int64_t* h_counts, uint64_t* h_stats,
                      cudaStream_t s, const double* xr = nullptr, const double* yr = nullptr, int64_t rows = 0,
                      SegRange range = SegRange{}) {
  const bool bip = xr != nullptr;
  g_info = mh_call_info{0, 0, 0, 0.0, 0.0, 0.0, 0.0};  // describes this call, also when it is rejected
  if (!bip) rows = n;
  int rc = check_params_impl(model, rows, n, bip, p);
  if (rc != MH_OK) return rc;
  if (!x || (model == MH_UECM && (!y || (bip && !yr))) || !workspace || !h_counts) {
    set_error("x%s, workspace and h_edges_per_sample must be non-NULL", model == MH_UECM ? ", y" : "");
    return MH_ERR_ARG;
  }
  if (o.capacity < 0 || ((p->flags & MH_CSR_SYMMETRIC) && o.capacity > 0x7FFFFFFFll)) {
    set_error("capacity_edges must be >= 0 (and < 2^31 with MH_CSR_SYMMETRIC)");
    return MH_ERR_ARG;
  }
  if ((p->flags & MH_OUT_COO) && o.capacity > 0 && (!o.src || !o.dst)) {
    set_error("MH_OUT_COO needs src and dst");
    return MH_ERR_ARG;
  }
  if ((p->flags & MH_OUT_CSR) && (!o.csr_off || (o.capacity > 0 && !o.csr_idx))) {
    set_error("MH_OUT_CSR needs csr_offsets and csr_indices");
    return MH_ERR_ARG;
  }
  const Layout L = bip ? make_layout_bip(model, rows, n, *p, o.capacity) : make_layout(model, n, *p, o.capacity);
  if (workspace_bytes < L.total) {
    set_error("workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
    return MH_ERR_WORKSPACE;
  }
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  MH_CUDA(cudaStreamIsCapturing(s, &cap_status));
  if (cap_status != cudaStreamCaptureStatusNone) {
    set_error("sampling calls read results back and cannot be captured into a caller's graph");
    return MH_ERR_ARG;
  }
  char* ws = static_cast<char*>(workspace);
  Net g = make_net(model, *p, x, y, n, L, ws);
  if (!g.lntab) {
    set_error("the logarithm table could not be built on this device");
    return MH_ERR_CUDA;
  }
  if (bip) {
    g.x_r = xr;
    g.y_r = yr;
  }
  const bool timed = (p->flags & MH_TIMING) != 0 && (p->num_samples + L.spc - 1) / L.spc <= kTimedChunks;
  const size_t counts_bytes = 8 * static_cast<size_t>(p->num_samples);
  if (g_pinned.bytes < sizeof(Ctrl) + counts_bytes) {
    g_graphs.clear();  // cached graphs copy into the old buffer
    MH_CUDA(g_pinned.reserve(sizeof(Ctrl) + counts_bytes));
  }
  char* hbuf = static_cast<char*>(g_pinned.ptr);
  MH_CUDA(prepare_kernel_attributes(model));
  if (timed) MH_CUDA(g_timer.create());

  int dev = 0;
  MH_CUDA(cudaGetDevice(&dev));
  CallKey key;
  memset(&key, 0, sizeof(key));
  key.model = model;
  key.device = dev;
  key.n = n;
  key.capacity = o.capacity;
  key.x = x;
  key.y = y;
  key.xr = xr;
  key.yr = yr;
  key.rows = rows;
  key.ws = workspace;
  key.src = o.src;
  key.dst = o.dst;
  key.w = o.w;
  key.csr_off = o.csr_off;
  key.csr_idx = o.csr_idx;
  key.csr_w = o.csr_w;
  key.hbuf = hbuf;
  key.ws_bytes = workspace_bytes;
  key.params = *p;
  key.seg_begin = range.begin;
  key.seg_end = range.end;

  g_info = mh_call_info{0, 0, 0, 0.0, 0.0, 0.0, 0.0};
  CachedGraph* cg = g_graphs.find(key);
  if (!cg && dev >= 0 && dev < 64 && g_graphs.seen_before(key)) {
    cudaStream_t& cs = g_graphs.capture_stream[dev];
    if (!cs) MH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    g_launches = 0;
    cudaGraph_t graph = nullptr;
    MH_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_sample(g, L, ws, p, o, timed, hbuf, cs, range);
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (rc != MH_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec == cudaSuccess && graph) {
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei == cudaSuccess) {
        cg = g_graphs.slot();
        cg->key = key;
        cg->exec = exec;
        cg->launches = g_launches;
        cg->chunks = (p->num_samples + L.spc - 1) / L.spc;
        cg->timer_marks = g_timer.used;
        cg->last_use = ++g_graphs.clock;
      }
    }
    cudaGetLastError();  // a failed capture falls back to direct launches below
  }
  if (cg) {
    MH_CUDA(cudaGraphLaunch(cg->exec, s));
    g_timer.on = timed;
    g_timer.used = static_cast<int>(cg->timer_marks);
    g_info.kernel_launches = cg->launches;
    g_info.sample_chunks = cg->chunks;
  } else {
    g_launches = 0;
    rc = enqueue_sample(g, L, ws, p, o, timed, hbuf, s, range);
    if (rc != MH_OK) return rc;
    g_info.kernel_launches = g_launches;
    g_info.sample_chunks = (p->num_samples + L.spc - 1) / L.spc;
  }
  g_info.walk_launches = g_info.sample_chunks;
  MH_CUDA(cudaStreamSynchronize(s));
  if (timed) {
    g_info.prepare_ms = g_timer.between(0, 1);
    for (int64_t t = 0; t < g_info.sample_chunks; ++t) {
      g_info.walk_ms += g_timer.between(static_cast<int>(2 + 3 * t), static_cast<int>(3 + 3 * t));
      g_info.emit_ms += g_timer.between(static_cast<int>(3 + 3 * t), static_cast<int>(4 + 3 * t));
    }
    g_info.total_ms = g_timer.between(0, g_timer.used - 1);
  }
  Ctrl hc;
  memcpy(&hc, hbuf, sizeof(Ctrl));
  memcpy(h_counts, hbuf + sizeof(Ctrl), counts_bytes);
  if (h_stats)
    for (int t = 0; t < MH_NUM_STATS; ++t) h_stats[t] = hc.stats[t];
  rc = status_to_code(hc.status, hc.num_segments, L.max_segments);
  if (rc != MH_OK) return rc;
  int64_t total = 0;
  for (uint32_t t = 0; t < p->num_samples; ++t) total += h_counts[t];
  if (total > o.capacity || (hc.status & kStCapacity)) {
    set_error("the sample has %lld edges, capacity_edges is %lld", static_cast<long long>(total),
              static_cast<long long>(o.capacity));
    return MH_ERR_CAPACITY;
  }
  return MH_OK;
}

}  // namespace mh

using namespace mh;

extern "C" {

const char* mh_error_string(int code) {
  switch (code) {
    case MH_OK: return "MH_OK";
    case MH_ERR_ARG: return "MH_ERR_ARG: invalid argument";
    case MH_ERR_DOMAIN: return "MH_ERR_DOMAIN: parameter outside the model's domain";
    case MH_ERR_CAPACITY: return "MH_ERR_CAPACITY: output shorter than the sample";
    case MH_ERR_WORKSPACE: return "MH_ERR_WORKSPACE: workspace or segment table too small";
    case MH_ERR_OVERFLOW: return "MH_ERR_OVERFLOW: weight above INT32_MAX";
    case MH_ERR_DEVICE_TIMEOUT: return "MH_ERR_DEVICE_TIMEOUT: bounded device wait gave up";
    case MH_ERR_CUDA: return "MH_ERR_CUDA: CUDA runtime error";
    default: return "unknown error code";
  }
}

const char* mh_last_error_detail(void) { return g_detail; }

int mh_last_call_info(mh_call_info* h_info) {
  if (!h_info) {
    set_error("h_info is NULL");
    return MH_ERR_ARG;
  }
  *h_info = g_info;
  return MH_OK;
}

int mh_workspace_size(int model, int64_t n, const mh_params* params, int64_t capacity_edges, size_t* h_bytes) {
  int rc = check_params(model, n, params);
  if (rc != MH_OK) return rc;
  if (capacity_edges < 0 || !h_bytes) {
    set_error("capacity_edges must be >= 0 and h_bytes non-NULL");
    return MH_ERR_ARG;
  }
  *h_bytes = make_layout(model, n, *params, capacity_edges).total;
  return MH_OK;
}

int mh_sample_ubcm(const double* x, int64_t n, const mh_params* params, void* workspace, size_t workspace_bytes,
                   int32_t* src, int32_t* dst, int64_t* csr_offsets, int32_t* csr_indices, int64_t capacity_edges,
                   int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream) {
  Outputs o{src, dst, nullptr, reinterpret_cast<long long*>(csr_offsets), csr_indices, nullptr, capacity_edges};
  return run_sample(MH_UBCM, x, nullptr, n, params, workspace, workspace_bytes, o, h_edges_per_sample, h_stats,
                    reinterpret_cast<cudaStream_t>(stream));
}

int mh_sample_weighted(const double* x, const double* y, int64_t n, const mh_params* params, void* workspace,
                       size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w, int64_t* csr_offsets,
                       int32_t* csr_indices, int32_t* csr_weights, int64_t capacity_edges,
                       int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream) {
  Outputs o{src, dst, w, reinterpret_cast<long long*>(csr_offsets), csr_indices, csr_weights, capacity_edges};
  return run_sample(MH_UECM, x, y, n, params, workspace, workspace_bytes, o, h_edges_per_sample, h_stats,
                    reinterpret_cast<cudaStream_t>(stream));
}

int mh_sample_range(int model, const double* x, const double* y, int64_t n, const mh_params* params,
                    int64_t seg_begin, int64_t seg_end, void* workspace, size_t workspace_bytes, int32_t* src,
                    int32_t* dst, int32_t* w, int64_t capacity_edges, int64_t* h_edges_per_sample,
                    uint64_t* h_stats, mh_stream_t stream) {
  if (model != MH_UBCM && model != MH_UECM) {
    set_error("model must be MH_UBCM or MH_UECM");
    return MH_ERR_ARG;
  }
  if (!params || seg_begin < 0 || seg_end < seg_begin) {
    set_error("need params and 0 <= seg_begin <= seg_end");
    return MH_ERR_ARG;
  }
  if (params->flags & (MH_OUT_CSR | MH_CSR_SYMMETRIC)) {
    set_error("a segment range is drawn as COO only (no MH_OUT_CSR, no MH_CSR_SYMMETRIC)");
    return MH_ERR_ARG;
  }
  Outputs o{src, dst, model == MH_UECM ? w : nullptr, nullptr, nullptr, nullptr, capacity_edges};
  return run_sample(model, x, model == MH_UECM ? y : nullptr, n, params, workspace, workspace_bytes, o,
                    h_edges_per_sample, h_stats, reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr, 0,
                    SegRange{seg_begin, seg_end});
}

int mh_bipartite_workspace_size(int model, int64_t n_plus, int64_t n_minus, const mh_params* params,
                                int64_t capacity_edges, size_t* h_bytes) {
  int rc = check_params_impl(model, n_plus, n_minus, true, params);
  if (rc != MH_OK) return rc;
  if (capacity_edges < 0 || !h_bytes) {
    set_error("capacity_edges must be >= 0 and h_bytes non-NULL");
    return MH_ERR_ARG;
  }
  *h_bytes = make_layout_bip(model, n_plus, n_minus, *params, capacity_edges).total;
  return MH_OK;
}

int mh_sample_bipartite(int model, const double* x_plus, const double* y_plus, int64_t n_plus,
                        const double* x_minus, const double* y_minus, int64_t n_minus, const mh_params* params,
                        void* workspace, size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w,
                        int64_t* csr_offsets, int32_t* csr_indices, int32_t* csr_weights, int64_t capacity_edges,
                        int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream) {
  if (!x_plus) {
    set_error("x_plus must be non-NULL");
    return MH_ERR_ARG;
  }
  Outputs o{src, dst, w, reinterpret_cast<long long*>(csr_offsets), csr_indices, csr_weights, capacity_edges};
  return run_sample(model, x_minus, y_minus, n_minus, params, workspace, workspace_bytes, o, h_edges_per_sample,
                    h_stats, reinterpret_cast<cudaStream_t>(stream), x_plus, y_plus, n_plus);
}

int mh_segment_table(int model, const double* x, const double* y, int64_t n, const mh_params* params,
                     void* workspace, size_t workspace_bytes, int32_t* seg_row, int32_t* seg_k, int64_t* seg_a,
                     int64_t* seg_b, int32_t* perm, int64_t cap, int64_t* h_num_segments, mh_stream_t stream) {
  int rc = check_params(model, n, params);
  if (rc != MH_OK) return rc;
  if (!x || (model == MH_UECM && !y) || !workspace || !h_num_segments || cap < 0 ||
      (cap > 0 && (!seg_row || !seg_k || !seg_a || !seg_b))) {
    set_error("missing pointer or negative cap");
    return MH_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Layout L = make_layout(model, n, *params, 0);
  if (workspace_bytes < L.total) {
    set_error("workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
    return MH_ERR_WORKSPACE;
  }
  char* ws = static_cast<char*>(workspace);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  const Net g = make_net(model, *params, x, y, n, L, ws);
  if (!g.lntab) {
    set_error("the logarithm table could not be built on this device");
    return MH_ERR_CUDA;
  }
  rc = prepare(g, L, ws, ctrl, s);
  if (rc != MH_OK) return rc;
  if (cap > 0) MH_CUDA(launch_export_table(g, ctrl, seg_row, seg_k, seg_a, seg_b, cap, s));
  if (perm) MH_CUDA(cudaMemcpyAsync(perm, g.perm, 4 * static_cast<size_t>(n), cudaMemcpyDeviceToDevice, s));
  MH_CUDA(g_pinned.reserve(sizeof(Ctrl)));
  MH_CUDA(cudaMemcpyAsync(g_pinned.ptr, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  MH_CUDA(cudaStreamSynchronize(s));
  Ctrl hc;
  memcpy(&hc, g_pinned.ptr, sizeof(Ctrl));
  *h_num_segments = hc.num_segments;
  rc = status_to_code(hc.status, hc.num_segments, L.max_segments);
  if (rc != MH_OK) return rc;
  if (hc.num_segments > cap) {
    set_error("table has %lld rows, cap is %lld", hc.num_segments, static_cast<long long>(cap));
    return MH_ERR_CAPACITY;
  }
  return MH_OK;
}

// Checks shared by the row-range entry points: model, n and the range, in
// that order; an empty range needs no pointers.
static int check_row_range(const char* fn, int model, int64_t n, int64_t row_begin, int64_t row_count) {
  if ((model != MH_UBCM && model != MH_UECM) || n < 1) {
    set_error("%s: bad model or n", fn);
    return MH_ERR_ARG;
  }
  if (row_begin < 0 || row_count < 0 || row_begin > n || row_count > n - row_begin) {
    set_error("%s: rows [%lld, %lld + %lld) are not within [0, %lld)", fn, static_cast<long long>(row_begin),
              static_cast<long long>(row_begin), static_cast<long long>(row_count), static_cast<long long>(n));
    return MH_ERR_ARG;
  }
  return MH_OK;
}

int maxent_expected_fwd_rows(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                             int64_t row_count, double* k_out, double* s_out, mh_stream_t stream) {
  const int rc = check_row_range("maxent_expected_fwd", model, n, row_begin, row_count);
  if (rc != MH_OK) return rc;
  if (row_count == 0) return MH_OK;
  if (!x || !k_out || (model == MH_UECM && (!y || !s_out))) {
    set_error("maxent_expected_fwd: a required pointer is NULL");
    return MH_ERR_ARG;
  }
  MH_CUDA(launch_expected_fwd(model, x, y, n, row_begin, row_count, k_out, s_out,
                              reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_fwd(int model, const double* x, const double* y, int64_t n, double* k_out, double* s_out,
                        mh_stream_t stream) {
  return maxent_expected_fwd_rows(model, x, y, n, 0, n, k_out, s_out, stream);
}

int maxent_expected_jacobian_diag_rows(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                       int64_t row_count, double* dk_dx, double* dk_dy, double* ds_dx, double* ds_dy,
                                       mh_stream_t stream) {
  const int rc = check_row_range("maxent_expected_jacobian_diag", model, n, row_begin, row_count);
  if (rc != MH_OK) return rc;
  if (row_count == 0) return MH_OK;
  if (!x || !dk_dx || (model == MH_UECM && (!y || !dk_dy || !ds_dx || !ds_dy))) {
    set_error("maxent_expected_jacobian_diag: a required pointer is NULL");
    return MH_ERR_ARG;
  }
  MH_CUDA(mh::launch_expected_jacobian_diag(model, x, y, n, row_begin, row_count, dk_dx, dk_dy, ds_dx, ds_dy,
                                            reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_jacobian_diag(int model, const double* x, const double* y, int64_t n, double* dk_dx,
                                  double* dk_dy, double* ds_dx, double* ds_dy, mh_stream_t stream) {
  return maxent_expected_jacobian_diag_rows(model, x, y, n, 0, n, dk_dx, dk_dy, ds_dx, ds_dy, stream);
}

int maxent_expected_bwd_rows(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                             int64_t row_count, const double* g_k, const double* g_s, double* g_x, double* g_y,
                             mh_stream_t stream) {
  const int rc = check_row_range("maxent_expected_bwd", model, n, row_begin, row_count);
  if (rc != MH_OK) return rc;
  if (row_count == 0) return MH_OK;
  if (!x || !g_k || !g_x || (model == MH_UECM && (!y || !g_s || !g_y))) {
    set_error("maxent_expected_bwd: a required pointer is NULL");
    return MH_ERR_ARG;
  }
  MH_CUDA(launch_expected_bwd(model, x, y, n, row_begin, row_count, g_k, g_s, g_x, g_y,
                              reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_bwd(int model, const double* x, const double* y, int64_t n, const double* g_k,
                        const double* g_s, double* g_x, double* g_y, mh_stream_t stream) {
  return maxent_expected_bwd_rows(model, x, y, n, 0, n, g_k, g_s, g_x, g_y, stream);
}

int mh_debug_first_level(const uint64_t* N, const double* z, const int32_t* room, int64_t n, float* E_out,
                         float* lam_out, int32_t* fl_out, mh_stream_t stream) {
  if (n < 0 || (n > 0 && (!N || !z || !room || !E_out || !lam_out || !fl_out))) {
    set_error("mh_debug_first_level: n < 0 or a NULL pointer");
    return MH_ERR_ARG;
  }
  if (n == 0) return MH_OK;
  MH_CUDA(mh::launch_first_level_probe(reinterpret_cast<const unsigned long long*>(N), z, room, n, E_out, lam_out,
                                       fl_out, reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_sym_workspace_size(int model, int64_t n, size_t* h_bytes) {
  if ((model != MH_UBCM && model != MH_UECM) || n < 1 || n > (1ll << 31) || !h_bytes) {
    set_error("maxent_expected_sym_workspace_size: bad model, n or NULL h_bytes");
    return MH_ERR_ARG;
  }
  *h_bytes = mh::expected_sym_workspace_bytes(model, n);
  return MH_OK;
}

// Shared checks of the symmetric forms: model, n, workspace, then pointers.
static int check_sym(const char* fn, int model, int64_t n, const void* workspace, size_t workspace_bytes,
                     bool ptrs_ok) {
  if ((model != MH_UBCM && model != MH_UECM) || n < 1 || n > (1ll << 31)) {
    set_error("%s: bad model or n", fn);
    return MH_ERR_ARG;
  }
  const size_t need = mh::expected_sym_workspace_bytes(model, n);
  if (!workspace || workspace_bytes < need) {
    set_error("%s: the workspace needs %zu bytes, got %zu", fn, need, workspace ? workspace_bytes : 0);
    return MH_ERR_WORKSPACE;
  }
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) {
    set_error("%s: the workspace must be 256-byte aligned", fn);
    return MH_ERR_ARG;
  }
  if (!ptrs_ok) {
    set_error("%s: a required pointer is NULL", fn);
    return MH_ERR_ARG;
  }
  return MH_OK;
}

int maxent_expected_fwd_sym(int model, const double* x, const double* y, int64_t n, double* k_out, double* s_out,
                            void* workspace, size_t workspace_bytes, mh_stream_t stream) {
  const int rc = check_sym("maxent_expected_fwd_sym", model, n, workspace, workspace_bytes,
                           x && k_out && (model == MH_UBCM || (y && s_out)));
  if (rc != MH_OK) return rc;
  MH_CUDA(mh::launch_expected_sym(0, model, x, y, nullptr, nullptr, n, workspace, k_out, s_out, nullptr, nullptr,
                                  reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_jacobian_diag_sym(int model, const double* x, const double* y, int64_t n, double* dk_dx,
                                      double* dk_dy, double* ds_dx, double* ds_dy, void* workspace,
                                      size_t workspace_bytes, mh_stream_t stream) {
  const int rc = check_sym("maxent_expected_jacobian_diag_sym", model, n, workspace, workspace_bytes,
                           x && dk_dx && (model == MH_UBCM || (y && dk_dy && ds_dx && ds_dy)));
  if (rc != MH_OK) return rc;
  MH_CUDA(mh::launch_expected_sym(1, model, x, y, nullptr, nullptr, n, workspace, dk_dx, dk_dy, ds_dx, ds_dy,
                                  reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_bwd_sym(int model, const double* x, const double* y, int64_t n, const double* g_k,
                            const double* g_s, double* g_x, double* g_y, void* workspace, size_t workspace_bytes,
                            mh_stream_t stream) {
  const int rc = check_sym("maxent_expected_bwd_sym", model, n, workspace, workspace_bytes,
                           x && g_k && g_x && (model == MH_UBCM || (y && g_s && g_y)));
  if (rc != MH_OK) return rc;
  MH_CUDA(mh::launch_expected_sym(2, model, x, y, g_k, g_s, n, workspace, g_x, g_y, nullptr, nullptr,
                                  reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_jacobian_diag_sym_f32(int model, const double* x, const double* y, int64_t n, double* dk_dx,
                                          double* dk_dy, double* ds_dx, double* ds_dy, void* workspace,
                                          size_t workspace_bytes, mh_stream_t stream) {
  const int rc = check_sym("maxent_expected_jacobian_diag_sym_f32", model, n, workspace, workspace_bytes,
                           x && dk_dx && (model == MH_UBCM || (y && dk_dy && ds_dx && ds_dy)));
  if (rc != MH_OK) return rc;
  MH_CUDA(mh::launch_expected_sym(3, model, x, y, nullptr, nullptr, n, workspace, dk_dx, dk_dy, ds_dx, ds_dy,
                                  reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

int maxent_expected_bwd_sym_f32(int model, const double* x, const double* y, int64_t n, const double* g_k,
                                const double* g_s, double* g_x, double* g_y, void* workspace, size_t workspace_bytes,
                                mh_stream_t stream) {
  const int rc = check_sym("maxent_expected_bwd_sym_f32", model, n, workspace, workspace_bytes,
                           x && g_k && g_x && (model == MH_UBCM || (y && g_s && g_y)));
  if (rc != MH_OK) return rc;
  MH_CUDA(mh::launch_expected_sym(4, model, x, y, g_k, g_s, n, workspace, g_x, g_y, nullptr, nullptr,
                                  reinterpret_cast<cudaStream_t>(stream)));
  return MH_OK;
}

}  // extern "C"

// ---- forwarders for the fixed-scratch entry point (noalloc.cu) -------------------
namespace mh {
int check_sample_params(int model, int64_t n, const mh_params* p) { return check_params(model, n, p); }
Net net_view(int model, const mh_params& p, const double* x, const double* y, int64_t n, const Layout& L,
             char* ws) {
  return make_net(model, p, x, y, n, L, ws);
}
int enqueue_sample_direct(const Net& g, const Layout& L, char* ws, const mh_params* p, const Outputs& o, char* hbuf,
                          cudaStream_t s) {
  return enqueue_sample(g, L, ws, p, o, false, hbuf, s);
}
int status_code(unsigned status, long long num_segments, int64_t max_segments) {
  return status_to_code(status, num_segments, max_segments);
}
int prepare_network(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  return prepare(g, L, ws, ctrl, s);
}
int64_t default_segments(int64_t n) { return default_max_segments(n); }
int64_t take_launch_count() {
  const int64_t v = g_launches;
  g_launches = 0;
  return v;
}
void record_call_info(const mh_call_info& info) { g_info = info; }
}  // namespace mh
