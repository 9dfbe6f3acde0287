// Batched ensembles: many networks x many samples, drawn in waves.
//
// The samples are exactly those of the single-network calls (Sec. 2.4,
// Algorithm 1); batching changes only how the work is scheduled.
//
// Preparation (mh_batch_prepare).  Every network is validated, sorted,
// gathered and partitioned into row segments by the single-network kernels,
// writing into its own slice of concatenated arrays in the workspace.
// Networks are spread round-robin over up to kPrepLanes streams, each with
// its own sort / scan scratch, so small networks prepare concurrently.
//
// Waves (mh_sample_batched).  A wave is a contiguous range of (network,
// sample) pairs.  The host writes each network's share of the wave (first
// pair, first sample, pair count, CSR base, key word) to pinned memory; the
// wave's first step copies it to the device, so a captured wave graph
// replays for any range.  A one-block plan kernel turns the shares and the
// prepared segment counts into work-item ranges:
//   items of network t        = pairs_t x S_t    (S_t segment-table rows)
//   item_begin_t              = exclusive prefix over t (pair order)
//   queue of model m          = the items of model-m networks, in t order
// One persistent walk launch per model drains its queue (the UBCM and UECM
// launches run concurrently on two streams); both write item counts and
// staged ranks into the same per-item arrays.  An exclusive scan of the
// item counts in item order then places every pair's edges contiguously, in
// pair order, and the emit pass writes COO / CSR output as the single-network
// emit does, resolving each item's network by bisection of item_begin.
#include <cstdio>
#include <cstring>

#include "mh_internal.cuh"
#include "scan.cuh"
#include "walk_math.cuh"

namespace mh {

// Forwarders into api.cu.
int prepare_network(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s);
int64_t default_segments(int64_t n);
int64_t take_launch_count();
void record_call_info(const mh_call_info& info);

namespace {

constexpr int kPrepLanes = 8;
constexpr int kMaxNets = 65536;
constexpr int64_t kMaxWavePairs = 1 << 20;
constexpr int64_t kDefaultWaveItems = 1ll << 26;
constexpr int64_t kMaxWaveItems = 1ll << 30;
constexpr int64_t kMaxNodes = (1ll << 31) - (1ll << 20);
constexpr unsigned long long kBatchMagic = 0x3142484d31424853ull;

struct BatchHeader {
  unsigned long long magic;
  unsigned long long fingerprint;
  long long n_nets;
  long long pad[5];
};

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// Offsets (bytes from the workspace start) of everything a batch keeps.
struct BatchLayout {
  int n_nets = 0;
  int lanes = 1;
  int n_model[2] = {0, 0};
  int64_t nodes = 0, nodes1 = 0, segs = 0, n_max = 0, tiles_max = 0;
  // persistent part (the first `image` bytes are copied from the host)
  size_t header = 0, nets = 0, order = 0, image = 0, net_ctrl = 0, wave = 0, mb = 0, wave_ctrl = 0;
  size_t perm = 0, rank = 0, xs = 0, ys = 0, as = 0, xdf = 0, adf = 0, ydf = 0, lny = 0, top = 0, Q = 0,
         rowoff = 0, seg = 0, seg_c = 0, seg_cf = 0, rowoff_node = 0, seg_slot = 0, slot_ik = 0,
         persistent_end = 0;
  // preparation scratch of one lane, relative to the lane's start
  Layout lane;
  size_t lane_bytes = 0, prep_end = 0;
  // wave buffers (overlapping the preparation scratch)
  int64_t items_max = 0, pairs_max = 0, csr_max = 0, capacity = 0, staging_entries = 0, scan_tiles = 0;
  size_t item_cnt = 0, item_base = 0, item_off = 0, pair_counts = 0, staging = 0, zero_begin = 0,
         scan_counters = 0, scan_flags = 0, zero_end = 0, scan_values = 0, wave_end = 0;
  size_t total = 0;
};

int64_t net_segments_cap(const mh_params& p, const mh_network_desc& d) {
  if (d.max_segments > 0) return d.max_segments;
  return p.max_segments > 0 ? p.max_segments : default_segments(d.n);
}

BatchLayout make_batch_layout(const mh_network_desc* nets, int n_nets, const mh_params& p, int64_t items_max,
                              int64_t capacity) {
  BatchLayout B;
  B.n_nets = n_nets;
  B.lanes = n_nets < kPrepLanes ? n_nets : kPrepLanes;
  for (int t = 0; t < n_nets; ++t) {
    B.nodes += nets[t].n;
    B.nodes1 += nets[t].n + 1;
    B.segs += net_segments_cap(p, nets[t]);
    if (nets[t].n > B.n_max) B.n_max = nets[t].n;
    B.n_model[nets[t].model == MH_UECM] += 1;
  }
  B.tiles_max = (B.n_max + kSortTile - 1) / kSortTile;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t N = static_cast<size_t>(B.nodes), N1 = static_cast<size_t>(B.nodes1),
               SG = static_cast<size_t>(B.segs), T = static_cast<size_t>(n_nets);
  B.header = take(sizeof(BatchHeader));
  B.nets = take(sizeof(BatchNet) * T);
  B.order = take(4 * 2 * T);
  B.image = off;
  B.net_ctrl = take(sizeof(Ctrl) * T);
  B.wave = take(sizeof(WaveNet) * T);
  B.mb = take(8 * 2 * (T + 1));
  B.wave_ctrl = take(sizeof(Ctrl));
  B.perm = take(4 * N);
  B.rank = take(4 * N);
  B.xs = take(8 * N);
  B.ys = take(8 * N);
  B.as = take(8 * N);
  B.xdf = take(8 * N);
  B.adf = take(8 * N);
  B.ydf = take(8 * N);
  B.lny = take(8 * N);
  B.top = take(sizeof(Top2) * N1);
  B.Q = take(8 * N1);
  B.rowoff = take(8 * N1);
  B.seg = take(sizeof(int4) * SG);
  B.seg_c = take(8 * SG);
  B.seg_cf = take(16 * SG);
  B.rowoff_node = take(8 * N1);
  B.seg_slot = take(4 * SG);
  B.slot_ik = take(8 * SG);
  B.persistent_end = off;

  // one lane's sort and scan scratch, sized for the largest network
  {
    Layout& L = B.lane;
    size_t lo = 0;
    auto ltake = [&](size_t bytes) {
      const size_t at = lo;
      lo = align256(lo + bytes);
      return at;
    };
    const size_t nm = static_cast<size_t>(B.n_max);
    const size_t tiles = static_cast<size_t>(B.tiles_max > 0 ? B.tiles_max : 1);
    int64_t scan_len = 256 * B.tiles_max;
    if (B.n_max + 1 > scan_len) scan_len = B.n_max + 1;
    L.scan_tiles = scan_len / kScanTile + 2;
    L.keys0 = ltake(8 * nm);
    L.keys1 = ltake(8 * nm);
    L.vals0 = ltake(4 * nm);
    L.vals1 = ltake(4 * nm);
    L.tsuf = ltake(sizeof(Top2) * nm);
    L.tsuf2 = ltake(sizeof(Top2) * nm);
    L.hist = ltake(4 * 256 * tiles);
    L.zero_begin = lo;
    L.ghist = ltake(4 * 8 * 256);
    L.sort_counters = ltake(16);
    L.sort_state = ltake(2 * 8 * 256 * tiles);
    L.scan_counters = ltake(16);
    L.scan_flags = ltake(4 * static_cast<size_t>(L.scan_tiles));
    L.zero_end = lo;
    L.scan_values = ltake(2 * sizeof(Top2) * static_cast<size_t>(L.scan_tiles));
    B.lane_bytes = lo;
  }
  B.prep_end = B.persistent_end + B.lane_bytes * static_cast<size_t>(B.lanes);

  // wave buffers
  B.items_max = items_max;
  int64_t pairs = static_cast<int64_t>(n_nets) * p.num_samples;
  B.pairs_max = pairs < kMaxWavePairs ? pairs : kMaxWavePairs;
  // every row but the last has a segment, so n_t + 1 <= S_t + 2 per pair
  B.csr_max = items_max + 2 * B.pairs_max;
  B.capacity = capacity;
  // two walk launches may run at once, each with up to kMaxWalkWarps warps
  B.staging_entries = capacity + capacity / 16 + 2ll * kMaxWalkWarps * (kStageChunk + kSlot);
  int64_t scan_len = items_max + 1 > B.csr_max ? items_max + 1 : B.csr_max;
  B.scan_tiles = scan_len / kScanTile + 2;
  off = B.persistent_end;
  B.item_cnt = take(4 * static_cast<size_t>(items_max));
  B.item_base = take(8 * static_cast<size_t>(items_max));
  B.item_off = take(8 * (static_cast<size_t>(items_max) + 1));
  B.pair_counts = take(8 * static_cast<size_t>(B.pairs_max));
  B.staging = take(4 * static_cast<size_t>(B.staging_entries));
  B.zero_begin = off;
  B.scan_counters = take(16);
  B.scan_flags = take(4 * static_cast<size_t>(B.scan_tiles));
  B.zero_end = off;
  B.scan_values = take(2 * sizeof(Top2) * static_cast<size_t>(B.scan_tiles));
  B.wave_end = off;
  B.total = B.prep_end > B.wave_end ? B.prep_end : B.wave_end;
  return B;
}

// FNV-1a over what the prepared arrays depend on.
unsigned long long batch_fingerprint(const mh_network_desc* nets, int n_nets, const mh_params& p) {
  unsigned long long h = 0xcbf29ce484222325ull;
  auto mix = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xFFu;
      h *= 0x100000001b3ull;
    }
  };
  mix(static_cast<unsigned long long>(n_nets));
  for (int t = 0; t < n_nets; ++t) {
    mix(static_cast<unsigned long long>(nets[t].model));
    mix(static_cast<unsigned long long>(nets[t].n));
    mix(reinterpret_cast<uintptr_t>(nets[t].x));
    mix(reinterpret_cast<uintptr_t>(nets[t].y));
    mix(static_cast<unsigned long long>(net_segments_cap(p, nets[t])));
  }
  mix(p.seg_target ? p.seg_target : static_cast<unsigned>(kDefaultSegTarget));
  mix(p.flags & MH_BOUND_PAPER);
  mix(static_cast<unsigned long long>(p.max_segments));
  return h;
}

// Per-network Layout for the single-network preparation kernels: its slices
// of the concatenated arrays and its lane's scratch.
Layout net_layout(const BatchLayout& B, const BatchNet& bn, int lane) {
  Layout L = B.lane;
  const size_t lane_at = B.persistent_end + B.lane_bytes * static_cast<size_t>(lane);
  L.keys0 += lane_at;
  L.keys1 += lane_at;
  L.vals0 += lane_at;
  L.vals1 += lane_at;
  L.tsuf += lane_at;
  L.tsuf2 += lane_at;
  L.hist += lane_at;
  L.zero_begin += lane_at;
  L.ghist += lane_at;
  L.sort_counters += lane_at;
  L.sort_state += lane_at;
  L.scan_counters += lane_at;
  L.scan_flags += lane_at;
  L.zero_end += lane_at;
  L.scan_values += lane_at;
  L.n = bn.n;
  L.tiles = (bn.n + kSortTile - 1) / kSortTile;
  L.max_segments = bn.max_segments;
  const size_t nb = static_cast<size_t>(bn.node_base), n1b = static_cast<size_t>(bn.node1_base),
               sb = static_cast<size_t>(bn.seg_base);
  L.perm = B.perm + 4 * nb;
  L.rank = B.rank + 4 * nb;
  L.xs = B.xs + 8 * nb;
  L.ys = B.ys + 8 * nb;
  L.as = B.as + 8 * nb;
  L.xdf = B.xdf + 8 * nb;
  L.adf = B.adf + 8 * nb;
  L.ydf = B.ydf + 8 * nb;
  L.lny = B.lny + 8 * nb;
  L.top1 = B.top + sizeof(Top2) * n1b;
  L.Q = B.Q + 8 * n1b;
  L.rowoff = B.rowoff + 8 * n1b;
  L.seg = B.seg + sizeof(int4) * sb;
  L.seg_c = B.seg_c + 8 * sb;
  L.seg_cf = B.seg_cf + 16 * sb;
  return L;
}

// Rows of a one-set network: the same nodes and arrays as the candidates.
Net one_set_rows(Net g) {
  g.rows = g.n;
  g.bip = false;
  g.excl = nullptr;
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
  return g;
}

Net make_batch_net(int model, const mh_params& p, const double* x, const double* y, int64_t n, const Layout& L,
                   char* ws) {
  Net g;
  memset(&g, 0, sizeof(g));
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
  return one_set_rows(g);
}

// ---- device side -------------------------------------------------------------------
struct BatchView {
  const BatchHeader* header;
  const BatchNet* nets;
  WaveNet* wave;
  const int32_t* order;  // [2][n_nets]
  long long* mb;         // [2][n_nets + 1]
  const Ctrl* net_ctrl;
  Ctrl* wc;
  int n_nets;
  int n_model0, n_model1;
  unsigned long long fingerprint;
  long long items_max, csr_max;
};

// Exclusive scan of one long long per thread over a 1024-thread block.
__device__ long long block_exclusive_scan(long long v, long long* warp_sums, long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const long long w = warp_sums[lane];
    long long wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long o = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += o;
    }
    warp_sums[lane] = wi - w;  // exclusive prefix of the warps
    if (lane == 31) warp_sums[32] = wi;
  }
  __syncthreads();
  const long long r = warp_sums[warp] + incl - v;
  total = warp_sums[32];
  __syncthreads();
  return r;
}

// Work items of network t in this wave (0 when a preparation error is pending).
__device__ __forceinline__ long long wave_items_of(const BatchView& V, int t) {
  long long S = V.net_ctrl[t].num_segments;
  const long long cap = V.nets[t].max_segments;
  if (S > cap) S = cap;
  if (S < 0) S = 0;
  V.wave[t].S = S;
  return S * static_cast<long long>(V.wave[t].sample_cnt);
}

// One block of 1024 threads: item ranges, queues and totals of the wave; it
// also resets the wave's control block.
__global__ void __launch_bounds__(1024) batch_plan_kernel(BatchView V) {
  __shared__ long long warp_sums[33];
  __shared__ unsigned s_status;
  const int T = V.n_nets;
  const int per = (T + 1023) / 1024;
  const int t0 = threadIdx.x * per;
  const int t1 = t0 + per < T ? t0 + per : T;
  if (threadIdx.x == 0) s_status = 0;
  __syncthreads();

  unsigned st = 0;
  long long my_items = 0, my_csr = 0;
  for (int t = t0; t < t1; ++t) {
    st |= V.net_ctrl[t].status;
    my_items += wave_items_of(V, t);
    my_csr += static_cast<long long>(V.wave[t].sample_cnt) * (V.nets[t].n + 1);
  }
  if (st) atomicOr(&s_status, st);
  long long items_total = 0, csr_total = 0;
  long long at = block_exclusive_scan(my_items, warp_sums, items_total);
  for (int t = t0; t < t1; ++t) {
    V.wave[t].item_begin = at;
    at += V.wave[t].S * static_cast<long long>(V.wave[t].sample_cnt);
  }
  (void)block_exclusive_scan(my_csr, warp_sums, csr_total);

  // queue of each model: its networks' items in network order
  long long model_total[2] = {0, 0};
  for (int m = 0; m < 2; ++m) {
    const int cnt = m ? V.n_model1 : V.n_model0;
    const int32_t* order = V.order + static_cast<size_t>(m) * T;
    long long* mb = V.mb + static_cast<size_t>(m) * (T + 1);
    const int q_per = (cnt + 1023) / 1024;
    const int p0 = threadIdx.x * q_per;
    const int p1 = p0 + q_per < cnt ? p0 + q_per : cnt;
    long long mine = 0;
    for (int p = p0; p < p1; ++p) {
      const WaveNet& w = V.wave[order[p]];
      mine += w.S * static_cast<long long>(w.sample_cnt);
    }
    long long q = block_exclusive_scan(mine, warp_sums, model_total[m]);
    for (int p = p0; p < p1; ++p) {
      mb[p] = q;
      const WaveNet& w = V.wave[order[p]];
      q += w.S * static_cast<long long>(w.sample_cnt);
    }
    if (threadIdx.x == 0) mb[cnt] = model_total[m];
  }
  __syncthreads();

  if (threadIdx.x == 0) {
    unsigned status = s_status;
    if (V.header->magic != kBatchMagic || V.header->fingerprint != V.fingerprint ||
        V.header->n_nets != static_cast<long long>(T))
      status |= kStNotPrepared;
    if (items_total > V.items_max || csr_total > V.csr_max) status |= kStWaveItems;
    Ctrl* wc = V.wc;
    wc->status = status;
    wc->ticket = 0;
    wc->ticket2 = 0;
    wc->stage_used = 0;
    wc->out_base = 0;
    wc->out_end = 0;
    for (int k = 0; k < MH_NUM_STATS; ++k) wc->stats[k] = 0;
    const bool run = status == 0;
    wc->wave_items = run ? items_total : 0;
    wc->model_items[0] = run ? model_total[0] : 0;
    wc->model_items[1] = run ? model_total[1] : 0;
    wc->num_segments = run ? csr_total : 0;  // a wave's control block keeps its CSR length here
    // keep the over-sized totals visible to the host's message
    if (status & kStWaveItems) {
      wc->key_or = static_cast<unsigned long long>(items_total);
      wc->key_and = static_cast<unsigned long long>(csr_total);
    }
  }
}

// Last index t in [0, count) with key(t) <= v, for non-decreasing keys.
template <typename KeyOf>
__device__ __forceinline__ int last_at_or_below(int count, long long v, KeyOf key) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(mid) <= v)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Edges of each pair of the wave.
__global__ void batch_pair_counts_kernel(BatchView V, const long long* __restrict__ item_off,
                                         long long* __restrict__ pair_counts, int64_t pair_count) {
  const bool run = V.wc->wave_items > 0;
  for (int64_t pw = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; pw < pair_count;
       pw += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    long long c = 0;
    if (run) {
      const int t = last_at_or_below(V.n_nets, pw, [&](int k) { return V.wave[k].pair_base; });
      const WaveNet& w = V.wave[t];
      const long long s = pw - w.pair_base;
      if (s >= 0 && s < static_cast<long long>(w.sample_cnt)) {
        const long long b0 = w.item_begin + s * w.S;
        c = item_off[b0 + w.S] - item_off[b0];
      }
    }
    pair_counts[pw] = c;
  }
}

// CSR counts of every (pair, node) of the wave, in place of the offsets.
__global__ void batch_csr_count_kernel(BatchView V, const int32_t* __restrict__ rank,
                                       const long long* __restrict__ rowoff, const long long* __restrict__ item_off,
                                       long long* __restrict__ csr_off) {
  const long long total = V.wc->num_segments;
  for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < total;
       o += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int t = last_at_or_below(V.n_nets, o, [&](int k) { return V.wave[k].csr_base; });
    const WaveNet& w = V.wave[t];
    const BatchNet& bn = V.nets[t];
    // a wave holds fewer than 2^31 CSR offsets
    const unsigned n1 = static_cast<unsigned>(bn.n) + 1u;
    const unsigned rel = static_cast<unsigned>(o - w.csr_base);
    const long long s = rel / n1;
    const long long u = rel - static_cast<unsigned>(s) * n1;
    long long c = 0;
    if (u < bn.n) {
      const long long i = rank[bn.node_base + u];
      const long long b0 = w.item_begin + s * w.S;
      c = item_off[b0 + rowoff[bn.node1_base + i + 1]] - item_off[b0 + rowoff[bn.node1_base + i]];
    }
    csr_off[o] = c;
  }
}

// CSR offsets of a node-order wave: entry (pair, u) is the item offset of
// node u's first slot (u = n: the pair's end).  Blocks take chunks of
// consecutive entries; the network of the chunk's first entry is searched
// once and the threads scan forward from it.
constexpr int kCsrOffChunk = 4096;

__global__ void __launch_bounds__(256) batch_csr_off_kernel(BatchView V, const long long* __restrict__ rowoff_node,
                                                            const long long* __restrict__ item_off,
                                                            long long* __restrict__ csr_off) {
  __shared__ int t_first;
  const long long total = V.wc->num_segments;
  for (long long c0 = static_cast<long long>(blockIdx.x) * kCsrOffChunk; c0 < total;
       c0 += static_cast<long long>(gridDim.x) * kCsrOffChunk) {
    if (threadIdx.x == 0) t_first = last_at_or_below(V.n_nets, c0, [&](int k) { return V.wave[k].csr_base; });
    __syncthreads();
    int t = t_first;
    for (int k = threadIdx.x; k < kCsrOffChunk && c0 + k < total; k += blockDim.x) {
      const long long o = c0 + k;
      while (t + 1 < V.n_nets && V.wave[t + 1].csr_base <= o) ++t;
      const WaveNet& w = V.wave[t];
      const BatchNet& bn = V.nets[t];
      // a wave holds fewer than 2^31 CSR offsets
      const unsigned n1 = static_cast<unsigned>(bn.n) + 1u;
      const unsigned rel = static_cast<unsigned>(o - w.csr_base);
      const long long s = rel / n1;
      const long long u = rel - static_cast<unsigned>(s) * n1;
      csr_off[o] = item_off[w.item_begin + s * w.S + rowoff_node[bn.node1_base + u]];
    }
    __syncthreads();  // t_first is rewritten for the next chunk
  }
}

struct BatchEmitParams {
  BatchView V;
  Net g;  // concatenated arrays
  const int32_t* item_cnt;
  const long long* item_base;
  const long long* item_off;
  const int32_t* staging;
  int64_t staging_cap;
  Outputs o;
  uint32_t key0;
  bool any_uecm;
  const int2* slot_ik;  // node-order CSR wave: (row rank, segment index) of each slot (NULL: rank order)
};

// What every edge of a work item shares, set up once per item.
struct EmitItem {
  long long base;    // staging position of the item's first rank
  long long row_at;  // CSR: index position of the item's first edge
  int cnt;           // edges of the item
  int i;             // row rank within the network
  int u;             // original id of row i's node
  int k;             // segment index within the row
  uint32_t sample;
  uint32_t key1;
  int nb;            // the network's first slot in the node arrays
  int n;
  int uecm;
  float2 lnyi;
  double yi;
};
// Warps take groups of kEmitGroup consecutive work items: lane l sets up
// item l's EmitItem in the warp's shared slice, then the group's edges are
// written 32 at a time, lane l taking edge (pass * 32 + l) of the group.
// Its item is the last lane whose first-edge offset (relative to the group)
// is at most that index: a five-step search over the offsets held by the
// lanes.  Empty items share their offset with the next item, so the search
// never selects them.  No block-wide barrier: warps move on independently.
constexpr int kBatchEmitWarps = 8;

__global__ void __launch_bounds__(kBatchEmitWarps * 32) batch_emit_kernel(BatchEmitParams P) {
  const BatchView& V = P.V;
  const Net& g = P.g;
  Ctrl* wc = V.wc;
  __shared__ LnEntry tab[kLnTable];
  __shared__ EmitItem info_all[kBatchEmitWarps][kEmitGroup];
  if (P.any_uecm) ln_table_to_shared(tab, g.lntab);
  __syncthreads();
  const long long items = wc->wave_items;
  if (wc->stage_used > static_cast<unsigned long long>(P.staging_cap)) return;  // staging overflowed
  const bool fp64_only = (g.flags & MH_FP64_ONLY) != 0;
  const bool csr = P.o.csr_idx != nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  EmitItem* info = info_all[warp];
  unsigned long long fallbacks = 0, boundary = 0;  // weight draws left to FP64; boundary draws
  bool overflow = false, bad = false;
  const long long stride = static_cast<long long>(gridDim.x) * kBatchEmitWarps * kEmitGroup;
  for (long long g0 = (static_cast<long long>(blockIdx.x) * kBatchEmitWarps + warp) * kEmitGroup; g0 < items;
       g0 += stride) {
    const long long item = g0 + lane;
    const bool in = item < items;
    // the group's edges are [item_off[g0], item_off[g0 + 32]) (item_off holds items + 1 entries)
    const long long off_l = P.item_off[in ? item : items];
    const long long first = __shfl_sync(0xffffffffu, off_l, 0);
    const long long last = lane == 31 ? P.item_off[in ? item + 1 : items] : 0;
    const long long total = __shfl_sync(0xffffffffu, last, 31) - first;
    if (total == 0) continue;  // a group of empty items (common in sparse rows)
    if (total >= (1ll << 31)) {  // cannot happen: a group's edges fit the staging, well below 2^31
      bad = true;
      continue;
    }
    const unsigned rel = static_cast<unsigned>(off_l - first);
    const int my_cnt = in ? static_cast<int>(P.item_cnt[item]) : 0;
    if (my_cnt > 0) {
      const int t = last_at_or_below(V.n_nets, item, [&](int q) { return V.wave[q].item_begin; });
      const WaveNet& w = V.wave[t];
      const BatchNet& bn = V.nets[t];
      // a wave holds fewer than 2^31 items and a network fewer than 2^31 rows
      const unsigned local = static_cast<unsigned>(item - w.item_begin);
      const unsigned S = static_cast<unsigned>(w.S);
      const unsigned s_local = local / S;
      const unsigned slot = local - s_local * S;
      int2 ik;
      if (P.slot_ik) {
        ik = P.slot_ik[bn.seg_base + slot];  // read in slot order
      } else {
        const int4 sg = g.seg[bn.seg_base + slot];
        ik = make_int2(sg.x, sg.y);
      }
      const long long gi = bn.node_base + ik.x;
      EmitItem it;
      it.base = P.item_base[item];
      it.cnt = my_cnt;
      it.i = ik.x;
      it.u = P.o.src ? g.perm[gi] : 0;  // the row's id, for COO only
      it.k = ik.y;
      it.sample = w.sample_lo + s_local;
      it.key1 = w.key1;
      it.nb = static_cast<int>(bn.node_base);
      it.n = bn.n;
      it.uecm = bn.model == MH_UECM;
      it.row_at = 0;
      if (csr && P.slot_ik) {
        it.row_at = off_l;  // node-order wave: the item offset is the CSR position
      } else if (csr) {
        const long long row_first = w.item_begin + static_cast<long long>(s_local) * S + g.rowoff[bn.node1_base + ik.x];
        it.row_at = P.o.csr_off[w.csr_base + static_cast<long long>(s_local) * (bn.n + 1) + it.u] +
                    (off_l - P.item_off[row_first]);
      }
      it.yi = 0.0;
      it.lnyi = make_float2(0.f, 0.f);
      if (it.uecm) {
        it.yi = g.ys[gi];
        it.lnyi = g.lny[gi];
      }
      info[lane] = it;
    }
    __syncwarp();
    const unsigned tot = static_cast<unsigned>(total);
    // Lane state of a pass: its item, edge and staged rank, the rank loaded
    // one pass ahead so that the load overlaps the current pass's work.
    auto locate = [&](unsigned idx, int& l, int& e) -> bool {
      l = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const unsigned v = __shfl_sync(0xffffffffu, rel, l + step);
        if (v <= idx) l += step;
      }
      const unsigned rel_l = __shfl_sync(0xffffffffu, rel, l);
      if (idx >= tot) return false;
      e = static_cast<int>(idx - rel_l);
      if (e >= info[l].cnt) {  // offsets inconsistent with the counts: never read past a run
        bad = true;
        return false;
      }
      return true;
    };
    int l_n = 0, e_n = 0;
    int32_t gj_n = 0;
    bool ok_n = locate(lane, l_n, e_n);
    if (ok_n) gj_n = P.staging[info[l_n].base + e_n];
    for (unsigned p0 = 0; p0 < tot; p0 += 32) {
      const unsigned idx = p0 + lane;
      const int l = l_n, e = e_n;
      const int32_t gj = gj_n;
      const bool ok = ok_n;
      if (p0 + 32 < tot) {  // warp-uniform
        ok_n = locate(idx + 32, l_n, e_n);
        if (ok_n) gj_n = P.staging[info[l_n].base + e_n];
      }
      if (!ok) continue;
      const EmitItem& it = info[l];
      const int j = gj - it.nb;
      if (j <= it.i || j >= it.n) {  // cannot happen for a walked segment; never index with it
        bad = true;
        continue;
      }
      const int32_t v = g.perm[gj];
      int32_t wt = 1;
      if (it.uecm) {
        const float2 lj = g.lny[gj];
        wt = draw_weight(static_cast<uint32_t>(e), static_cast<uint32_t>(it.k), static_cast<uint32_t>(it.i),
                         it.sample, P.key0, it.key1, it.yi, &g.ys[gj], df2{it.lnyi.x, it.lnyi.y}, df2{lj.x, lj.y},
                         tab, fp64_only, overflow, fallbacks, boundary);
      }
      const long long pos = first + idx;
      if (pos < P.o.capacity && P.o.src) {
        P.o.src[pos] = it.u;
        P.o.dst[pos] = v;
        if (P.o.w) P.o.w[pos] = wt;
      }
      if (csr) {
        const long long at = it.row_at + e;
        if (at < P.o.capacity) {
          P.o.csr_idx[at] = v;
          if (P.o.csr_w) P.o.csr_w[at] = wt;
        }
      }
    }
    __syncwarp();  // the slice is rewritten by the next group
  }
  if (overflow) atomicOr(&wc->status, kStOverflow);
  if (bad) atomicOr(&wc->status, kStInternal);
  if (boundary) atomicAdd(&wc->stats[MH_STAT_BOUNDARY], boundary);
  (void)fallbacks;
}

// ---- host side ----------------------------------------------------------------------
#define MHB_CUDA(expr)                                                           \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      set_error("%s failed: %s", #expr, cudaGetErrorString(e_));                 \
      return MH_ERR_CUDA;                                                        \
    }                                                                            \
  } while (0)

// Library-owned streams and events of one device and host thread:
// preparation lanes, the second walk stream of a wave, fork / join events,
// timing events and a capture stream.
struct DeviceStreams {
  cudaStream_t lane[kPrepLanes] = {};
  cudaStream_t aux = nullptr;
  cudaStream_t capture = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kPrepLanes + 1] = {};
  cudaEvent_t timer[4] = {};
  bool ready = false;
};
thread_local DeviceStreams g_streams[64];

// An event record that becomes a graph node of its own inside a capture.
cudaError_t mark(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &st);
  if (e != cudaSuccess) return e;
  if (st == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  return cudaEventRecord(ev, s);
}

int device_streams(DeviceStreams** out) {
  int dev = 0;
  MHB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return MH_ERR_ARG;
  }
  DeviceStreams& d = g_streams[dev];
  if (!d.ready) {
    for (auto& s : d.lane) MHB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    MHB_CUDA(cudaStreamCreateWithFlags(&d.aux, cudaStreamNonBlocking));
    MHB_CUDA(cudaStreamCreateWithFlags(&d.capture, cudaStreamNonBlocking));
    MHB_CUDA(cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming));
    for (auto& e : d.join) MHB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : d.timer) MHB_CUDA(cudaEventCreate(&e));
    d.ready = true;
  }
  *out = &d;
  return MH_OK;
}

struct PinnedBuf {
  char* ptr = nullptr;
  size_t bytes = 0;
  ~PinnedBuf() {
    if (ptr) cudaFreeHost(ptr);
  }
  cudaError_t reserve(size_t want) {
    if (want <= bytes) return cudaSuccess;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&ptr), want, cudaHostAllocDefault);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
};

// A small thread-local cache of instantiated graphs.  A graph is captured
// the second time its key is seen, so one-off calls launch directly.
struct GraphSlot {
  unsigned char key[160];
  size_t key_len = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  uint64_t last_use = 0;
};
struct BatchGraphs {
  static constexpr int kSlots = 8;
  static constexpr int kSeen = 16;
  GraphSlot slot[kSlots];
  unsigned long long seen[kSeen] = {};
  int seen_next = 0;
  uint64_t clock = 0;
  ~BatchGraphs() { clear(); }
  void clear() {
    for (auto& s : slot)
      if (s.exec) {
        cudaGraphExecDestroy(s.exec);
        s.exec = nullptr;
      }
  }
  static unsigned long long hash(const void* k, size_t len) {
    unsigned long long h = 0xcbf29ce484222325ull;
    const unsigned char* b = static_cast<const unsigned char*>(k);
    for (size_t i = 0; i < len; ++i) {
      h ^= b[i];
      h *= 0x100000001b3ull;
    }
    return h | 1ull;
  }
  GraphSlot* find(const void* k, size_t len) {
    for (auto& s : slot)
      if (s.exec && s.key_len == len && memcmp(s.key, k, len) == 0) {
        s.last_use = ++clock;
        return &s;
      }
    return nullptr;
  }
  // true when the key was seen before (and remembers it otherwise)
  bool seen_before(const void* k, size_t len) {
    const unsigned long long h = hash(k, len);
    for (auto v : seen)
      if (v == h) return true;
    seen[seen_next] = h;
    seen_next = (seen_next + 1) % kSeen;
    return false;
  }
  GraphSlot* victim() {
    GraphSlot* v = &slot[0];
    for (auto& s : slot) {
      if (!s.exec) return &s;
      if (s.last_use < v->last_use) v = &s;
    }
    cudaGraphExecDestroy(v->exec);
    v->exec = nullptr;
    return v;
  }
};
thread_local BatchGraphs g_batch_graphs;
thread_local PinnedBuf g_prep_pinned;   // prepare: image + read-back of the network control blocks
thread_local PinnedBuf g_wave_pinned;   // waves: network shares + read-back of control block and counts

// Runs `enqueue` on `s`, through a cached graph when its key was seen before.
template <typename Enqueue>
int run_graphed(const void* key, size_t key_len, cudaStream_t s, DeviceStreams* ds, Enqueue enqueue,
                int64_t* launches) {
  BatchGraphs& G = g_batch_graphs;
  GraphSlot* gs = G.find(key, key_len);
  if (!gs && key_len <= sizeof(GraphSlot::key) && G.seen_before(key, key_len)) {
    take_launch_count();
    cudaGraph_t graph = nullptr;
    MHB_CUDA(cudaStreamBeginCapture(ds->capture, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue(ds->capture);
    const cudaError_t ec = cudaStreamEndCapture(ds->capture, &graph);
    if (rc != MH_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec == cudaSuccess && graph) {
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei == cudaSuccess) {
        gs = G.victim();
        memcpy(gs->key, key, key_len);
        gs->key_len = key_len;
        gs->exec = exec;
        gs->launches = take_launch_count();
        gs->last_use = ++G.clock;
      }
    }
    cudaGetLastError();  // a failed capture falls back to direct launches
  }
  if (gs) {
    MHB_CUDA(cudaGraphLaunch(gs->exec, s));
    *launches = gs->launches;
    return MH_OK;
  }
  take_launch_count();
  const int rc = enqueue(s);
  *launches = take_launch_count();
  return rc;
}

int check_batch(const mh_network_desc* nets, int32_t n_nets, const mh_params* p) {
  if (!nets || n_nets < 1 || n_nets > kMaxNets) {
    set_error("h_nets must be non-NULL and 1 <= n_nets <= %d (got %d)", kMaxNets, n_nets);
    return MH_ERR_ARG;
  }
  if (!p) {
    set_error("params is NULL");
    return MH_ERR_ARG;
  }
  if (p->network_id != 0) {
    set_error("params->network_id must be 0 for a batch (each network has its own)");
    return MH_ERR_ARG;
  }
  if (p->flags & (MH_CSR_SYMMETRIC | MH_CHUNG_LU)) {
    set_error("MH_CSR_SYMMETRIC and MH_CHUNG_LU apply to single-network calls only");
    return MH_ERR_ARG;
  }
  int64_t nodes = 0, segs = 0;
  for (int t = 0; t < n_nets; ++t) {
    const mh_network_desc& d = nets[t];
    const int rc = check_sample_params(d.model, d.n, p);
    if (rc != MH_OK) {
      char msg[400];
      snprintf(msg, sizeof(msg), "network %d: %s", t, mh_last_error_detail());
      set_error("%s", msg);
      return rc;
    }
    if (!d.x || (d.model == MH_UECM && !d.y)) {
      set_error("network %d: x%s must be non-NULL", t, d.model == MH_UECM ? " and y" : "");
      return MH_ERR_ARG;
    }
    if (d.max_segments < 0 || (d.max_segments > 0 && d.max_segments < d.n - 1) || d.max_segments >= (1ll << 31)) {
      set_error("network %d: max_segments must be 0 or in [n - 1, 2^31)", t);
      return MH_ERR_ARG;
    }
    nodes += d.n;
    segs += net_segments_cap(*p, d);
  }
  if (nodes > kMaxNodes || segs >= (1ll << 31)) {
    set_error("the batch holds %lld nodes and %lld segment rows; the limits are %lld and 2^31 - 1",
              static_cast<long long>(nodes), static_cast<long long>(segs), static_cast<long long>(kMaxNodes));
    return MH_ERR_ARG;
  }
  return MH_OK;
}

int64_t wave_items_arg(int64_t v) { return v == 0 ? kDefaultWaveItems : v; }

// Host image of the header, network records and model orders.
void fill_image(const BatchLayout& B, const mh_network_desc* nets, const mh_params& p, char* img) {
  memset(img, 0, B.image);
  BatchHeader* h = reinterpret_cast<BatchHeader*>(img + B.header);
  h->magic = kBatchMagic;
  h->fingerprint = batch_fingerprint(nets, B.n_nets, p);
  h->n_nets = B.n_nets;
  BatchNet* bn = reinterpret_cast<BatchNet*>(img + B.nets);
  int32_t* order = reinterpret_cast<int32_t*>(img + B.order);
  long long nb = 0, n1b = 0, sb = 0;
  int cnt[2] = {0, 0};
  for (int t = 0; t < B.n_nets; ++t) {
    bn[t].node_base = nb;
    bn[t].node1_base = n1b;
    bn[t].seg_base = sb;
    bn[t].max_segments = net_segments_cap(p, nets[t]);
    bn[t].n = static_cast<int>(nets[t].n);
    bn[t].model = nets[t].model;
    nb += nets[t].n;
    n1b += nets[t].n + 1;
    sb += bn[t].max_segments;
    const int m = nets[t].model == MH_UECM;
    order[m * B.n_nets + cnt[m]++] = t;
  }
}

Net concatenated_net(const BatchLayout& B, const mh_params& p, char* ws) {
  Net g;
  memset(&g, 0, sizeof(g));
  g.model = -1;
  g.flags = p.flags;
  g.n = B.nodes;
  g.perm = reinterpret_cast<int32_t*>(ws + B.perm);
  g.rank = reinterpret_cast<int32_t*>(ws + B.rank);
  g.xs = reinterpret_cast<double*>(ws + B.xs);
  g.ys = reinterpret_cast<double*>(ws + B.ys);
  g.as = reinterpret_cast<double*>(ws + B.as);
  g.top = reinterpret_cast<Top2*>(ws + B.top);
  g.Q = reinterpret_cast<unsigned long long*>(ws + B.Q);
  g.rowoff = reinterpret_cast<long long*>(ws + B.rowoff);
  g.seg = reinterpret_cast<int4*>(ws + B.seg);
  g.seg_c = reinterpret_cast<double*>(ws + B.seg_c);
  g.seg_cf = reinterpret_cast<float4*>(ws + B.seg_cf);
  g.xdf = reinterpret_cast<float2*>(ws + B.xdf);
  g.adf = reinterpret_cast<float2*>(ws + B.adf);
  g.ydf = reinterpret_cast<float2*>(ws + B.ydf);
  g.lny = reinterpret_cast<float2*>(ws + B.lny);
  g.lntab = ln_table_ptr();
  g.max_segments = B.segs;
  g.seg_target = p.seg_target ? static_cast<int>(p.seg_target) : kDefaultSegTarget;
  return one_set_rows(g);
}

// UBCM networks keep their x products in xs / xdf; the UBCM walk reads as /
// adf, so the concatenated view points those at the same arrays per model.
Net model_view(const Net& g, int model) {
  Net v = g;
  v.model = model;
  if (model == MH_UBCM) {
    v.as = g.xs;
    v.adf = g.xdf;
  }
  return one_set_rows(v);
}

}  // namespace

}  // namespace mh

using namespace mh;

extern "C" {

int mh_batch_workspace_size(const mh_network_desc* h_nets, int32_t n_nets, const mh_params* params,
                            int64_t max_wave_items, int64_t capacity_edges, size_t* h_bytes) {
  int rc = check_batch(h_nets, n_nets, params);
  if (rc != MH_OK) return rc;
  const int64_t items = wave_items_arg(max_wave_items);
  if (items < 1 || items > kMaxWaveItems || capacity_edges < 0 || !h_bytes) {
    set_error("max_wave_items must be 0 or in [1, 2^30], capacity_edges >= 0 and h_bytes non-NULL");
    return MH_ERR_ARG;
  }
  *h_bytes = make_batch_layout(h_nets, n_nets, *params, items, capacity_edges).total;
  return MH_OK;
}

int mh_batch_prepare(const mh_network_desc* h_nets, int32_t n_nets, const mh_params* params, void* workspace,
                     size_t workspace_bytes, int64_t* h_num_segments, mh_stream_t stream) {
  int rc = check_batch(h_nets, n_nets, params);
  if (rc != MH_OK) return rc;
  if (!workspace || !h_num_segments) {
    set_error("workspace and h_num_segments must be non-NULL");
    return MH_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MHB_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    set_error("batch calls read results back and cannot be captured into a caller's graph");
    return MH_ERR_ARG;
  }
  const BatchLayout B = make_batch_layout(h_nets, n_nets, *params, 1, 0);
  if (workspace_bytes < B.prep_end) {
    set_error("preparing the batch needs %zu workspace bytes, got %zu", B.prep_end, workspace_bytes);
    return MH_ERR_WORKSPACE;
  }
  DeviceStreams* ds = nullptr;
  rc = device_streams(&ds);
  if (rc != MH_OK) return rc;
  MHB_CUDA(prepare_kernel_attributes(MH_UBCM));
  MHB_CUDA(prepare_kernel_attributes(MH_UECM));
  const size_t back_bytes = sizeof(Ctrl) * static_cast<size_t>(n_nets);
  const size_t want = B.image + back_bytes;
  if (g_prep_pinned.bytes < want) {
    g_batch_graphs.clear();  // cached graphs copy from and into the old buffer
    MHB_CUDA(g_prep_pinned.reserve(want));
  }
  char* img = g_prep_pinned.ptr;
  char* back = img + B.image;
  fill_image(B, h_nets, *params, img);
  char* ws = static_cast<char*>(workspace);
  const BatchNet* bnets = reinterpret_cast<const BatchNet*>(img + B.nets);
  const bool timed = (params->flags & MH_TIMING) != 0;

  auto enqueue = [&](cudaStream_t q) -> int {
    MHB_CUDA(cudaMemcpyAsync(ws, img, B.image, cudaMemcpyHostToDevice, q));
    MHB_CUDA(cudaEventRecord(ds->fork, q));
    for (int l = 0; l < B.lanes; ++l) MHB_CUDA(cudaStreamWaitEvent(ds->lane[l], ds->fork, 0));
    for (int t = 0; t < n_nets; ++t) {
      const int l = t % B.lanes;
      const Layout L = net_layout(B, bnets[t], l);
      const Net g = make_batch_net(h_nets[t].model, *params, h_nets[t].x, h_nets[t].y, h_nets[t].n, L, ws);
      if (!g.lntab) {
        set_error("the logarithm table could not be built on this device");
        return MH_ERR_CUDA;
      }
      Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + B.net_ctrl) + t;
      const int r = prepare_network(g, L, ws, ctrl, ds->lane[l]);
      if (r != MH_OK) return r;
      // node-id order of the network's work items (CSR waves)
      {
        const BatchNet& bn = bnets[t];
        long long* rn = reinterpret_cast<long long*>(ws + B.rowoff_node) + bn.node1_base;
        int32_t* ss = reinterpret_cast<int32_t*>(ws + B.seg_slot) + bn.seg_base;
        int2* sl = reinterpret_cast<int2*>(ws + B.slot_ik) + bn.seg_base;
        const ScanState st{reinterpret_cast<unsigned*>(ws + L.scan_flags), ws + L.scan_values,
                           reinterpret_cast<unsigned*>(ws + L.scan_counters), ctrl, L.scan_tiles,
                           (params->flags & MH_TEST_WAIT_TIMEOUT) ? kTestStuckPolls : 0u};
        MHB_CUDA(launch_node_order(g, ctrl, rn, ss, sl, st, ds->lane[l]));
      }
    }
    for (int l = 0; l < B.lanes; ++l) {
      MHB_CUDA(cudaEventRecord(ds->join[l], ds->lane[l]));
      MHB_CUDA(cudaStreamWaitEvent(q, ds->join[l], 0));
    }
    MHB_CUDA(cudaMemcpyAsync(back, ws + B.net_ctrl, back_bytes, cudaMemcpyDeviceToHost, q));
    return MH_OK;
  };
  struct PrepKey {
    int tag, device;
    const void* ws;
    size_t ws_bytes;
    const void* pinned;
    unsigned long long fingerprint;
    int n_nets;
    uint32_t flags;
  } key;
  memset(&key, 0, sizeof(key));
  key.tag = 1;
  MHB_CUDA(cudaGetDevice(&key.device));
  key.ws = workspace;
  key.ws_bytes = workspace_bytes;
  key.pinned = img;
  key.fingerprint = batch_fingerprint(h_nets, n_nets, *params);
  key.n_nets = n_nets;
  key.flags = params->flags;
  if (timed) MHB_CUDA(cudaEventRecord(ds->timer[0], s));
  int64_t launches = 0;
  rc = run_graphed(&key, sizeof(key), s, ds, enqueue, &launches);
  if (rc != MH_OK) return rc;
  if (timed) MHB_CUDA(cudaEventRecord(ds->timer[1], s));
  MHB_CUDA(cudaStreamSynchronize(s));
  mh_call_info info{launches, 0, 0, 0.0, 0.0, 0.0, 0.0};
  if (timed) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ds->timer[0], ds->timer[1]);
    info.prepare_ms = info.total_ms = ms;
  }
  record_call_info(info);
  const Ctrl* hc = reinterpret_cast<const Ctrl*>(back);
  int first_bad = -1;
  unsigned bad_status = 0;
  for (int t = 0; t < n_nets; ++t) {
    long long S = hc[t].num_segments;
    h_num_segments[t] = S;
    if (hc[t].status && first_bad < 0) {
      first_bad = t;
      bad_status = hc[t].status;
    }
  }
  if (first_bad >= 0) {
    rc = status_code(bad_status, hc[first_bad].num_segments, bnets[first_bad].max_segments);
    char msg[400];
    snprintf(msg, sizeof(msg), "network %d: %s", first_bad, mh_last_error_detail());
    set_error("%s", msg);
    return rc;
  }
  return MH_OK;
}

int mh_sample_batched(const mh_network_desc* h_nets, int32_t n_nets, const mh_params* params,
                      int64_t max_wave_items, void* workspace, size_t workspace_bytes, int64_t pair_begin,
                      int64_t pair_count, int32_t* src, int32_t* dst, int32_t* w, int64_t* csr_offsets,
                      int32_t* csr_indices, int32_t* csr_weights, int64_t capacity_edges,
                      int64_t* h_edges_per_pair, uint64_t* h_stats, mh_stream_t stream) {
  int rc = check_batch(h_nets, n_nets, params);
  if (rc != MH_OK) return rc;
  const int64_t items_max = wave_items_arg(max_wave_items);
  const int64_t pairs_total = static_cast<int64_t>(n_nets) * params->num_samples;
  if (items_max < 1 || items_max > kMaxWaveItems) {
    set_error("max_wave_items must be 0 or in [1, 2^30]");
    return MH_ERR_ARG;
  }
  if (pair_begin < 0 || pair_count < 1 || pair_count > kMaxWavePairs || pair_begin + pair_count > pairs_total) {
    set_error("pairs [%lld, %lld) must be a non-empty range of at most 2^20 pairs within [0, %lld)",
              static_cast<long long>(pair_begin), static_cast<long long>(pair_begin + pair_count),
              static_cast<long long>(pairs_total));
    return MH_ERR_ARG;
  }
  if (!workspace || !h_edges_per_pair || capacity_edges < 0) {
    set_error("workspace and h_edges_per_pair must be non-NULL and capacity_edges >= 0");
    return MH_ERR_ARG;
  }
  const uint32_t fl = params->flags;
  if (fl & MH_CSR_SYMMETRIC) {
    set_error("MH_CSR_SYMMETRIC applies to mh_sample_ubcm and mh_sample_weighted only");
    return MH_ERR_ARG;
  }
  if ((fl & MH_OUT_COO) && capacity_edges > 0 && (!src || !dst)) {
    set_error("MH_OUT_COO needs src and dst");
    return MH_ERR_ARG;
  }
  if ((fl & MH_OUT_CSR) && (!csr_offsets || (capacity_edges > 0 && !csr_indices))) {
    set_error("MH_OUT_CSR needs csr_offsets and csr_indices");
    return MH_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MHB_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    set_error("batch calls read results back and cannot be captured into a caller's graph");
    return MH_ERR_ARG;
  }
  const BatchLayout B = make_batch_layout(h_nets, n_nets, *params, items_max, capacity_edges);
  if (workspace_bytes < B.wave_end) {
    set_error("a wave needs %zu workspace bytes, got %zu", B.wave_end, workspace_bytes);
    return MH_ERR_WORKSPACE;
  }
  DeviceStreams* ds = nullptr;
  rc = device_streams(&ds);
  if (rc != MH_OK) return rc;
  MHB_CUDA(prepare_kernel_attributes(MH_UBCM));
  MHB_CUDA(prepare_kernel_attributes(MH_UECM));

  // pinned: the networks' shares, then the read-back (control block, counts)
  const size_t share_bytes = sizeof(WaveNet) * static_cast<size_t>(n_nets);
  const size_t back_at = align256(share_bytes);
  const size_t want = back_at + sizeof(Ctrl) + 8 * static_cast<size_t>(pair_count);
  if (g_wave_pinned.bytes < want) {
    g_batch_graphs.clear();
    MHB_CUDA(g_wave_pinned.reserve(want < (1u << 20) ? (1u << 20) : want));
  }
  char* hshare = g_wave_pinned.ptr;
  char* hback = hshare + back_at;
  {
    WaveNet* sh = reinterpret_cast<WaveNet*>(hshare);
    memset(sh, 0, share_bytes);
    const uint32_t key1_base = static_cast<uint32_t>(params->seed >> 32);
    const int64_t spn = params->num_samples;
    long long pair_at = 0, csr_at = 0;
    for (int t = 0; t < n_nets; ++t) {
      const int64_t first = static_cast<int64_t>(t) * spn, last = first + spn;  // pairs of network t
      const int64_t lo = pair_begin > first ? pair_begin : first;
      const int64_t hi = pair_begin + pair_count < last ? pair_begin + pair_count : last;
      sh[t].pair_base = pair_at;
      sh[t].csr_base = csr_at;
      sh[t].key1 = key1_base + h_nets[t].network_id;
      if (hi > lo) {
        sh[t].sample_lo = params->sample_begin + static_cast<uint32_t>(lo - first);
        sh[t].sample_cnt = static_cast<uint32_t>(hi - lo);
        pair_at += hi - lo;
        csr_at += (hi - lo) * (h_nets[t].n + 1);
      } else {
        sh[t].sample_lo = params->sample_begin;
      }
    }
  }

  char* ws = static_cast<char*>(workspace);
  Ctrl* wc = reinterpret_cast<Ctrl*>(ws + B.wave_ctrl);
  BatchView V;
  V.header = reinterpret_cast<const BatchHeader*>(ws + B.header);
  V.nets = reinterpret_cast<const BatchNet*>(ws + B.nets);
  V.wave = reinterpret_cast<WaveNet*>(ws + B.wave);
  V.order = reinterpret_cast<const int32_t*>(ws + B.order);
  V.mb = reinterpret_cast<long long*>(ws + B.mb);
  V.net_ctrl = reinterpret_cast<const Ctrl*>(ws + B.net_ctrl);
  V.wc = wc;
  V.n_nets = n_nets;
  V.n_model0 = B.n_model[0];
  V.n_model1 = B.n_model[1];
  V.fingerprint = batch_fingerprint(h_nets, n_nets, *params);
  V.items_max = items_max;
  V.csr_max = B.csr_max;

  const Net gall = concatenated_net(B, *params, ws);
  if (!gall.lntab) {
    set_error("the logarithm table could not be built on this device");
    return MH_ERR_CUDA;
  }
  Outputs out{src, dst, w, reinterpret_cast<long long*>(csr_offsets), csr_indices, csr_weights, capacity_edges};
  if (!(fl & MH_OUT_COO)) out.src = out.dst = out.w = nullptr;
  if (!(fl & MH_OUT_CSR)) out.csr_off = nullptr, out.csr_idx = nullptr, out.csr_w = nullptr;
  if (B.n_model[1] == 0) out.w = out.csr_w = nullptr;

  ChunkArgs c;
  memset(&c, 0, sizeof(c));
  c.key0 = static_cast<uint32_t>(params->seed);
  c.key1 = static_cast<uint32_t>(params->seed >> 32);
  c.item_cnt = reinterpret_cast<int32_t*>(ws + B.item_cnt);
  c.item_base = reinterpret_cast<long long*>(ws + B.item_base);
  c.item_off = reinterpret_cast<long long*>(ws + B.item_off);
  c.staging = reinterpret_cast<int32_t*>(ws + B.staging);
  c.staging_cap = B.staging_entries;
  c.items_max = items_max;
  c.walk_ctas_per_sm = static_cast<int>(params->walk_ctas_per_sm);
  const ScanState scan_state{reinterpret_cast<unsigned*>(ws + B.scan_flags), ws + B.scan_values,
                             reinterpret_cast<unsigned*>(ws + B.scan_counters), wc, B.scan_tiles,
                             (fl & MH_TEST_WAIT_TIMEOUT) ? kTestStuckPolls : 0u};
  long long* pair_counts = reinterpret_cast<long long*>(ws + B.pair_counts);
  const bool timed = (fl & MH_TIMING) != 0;
  // CSR-only waves number their work items by node id (the COO order stays
  // the canonical rank order)
  const bool node_order = out.csr_off != nullptr && out.src == nullptr;

  auto enqueue = [&](cudaStream_t q) -> int {
    MHB_CUDA(cudaMemcpyAsync(V.wave, hshare, share_bytes, cudaMemcpyHostToDevice, q));
    MHB_CUDA(cudaMemsetAsync(ws + B.zero_begin, 0, B.zero_end - B.zero_begin, q));
    batch_plan_kernel<<<1, 1024, 0, q>>>(V);
    note_launches(1);
    MHB_CUDA(cudaGetLastError());
    if (timed) MHB_CUDA(mark(ds->timer[1], q));
    // one persistent walk per model; with both models the UECM walk runs on
    // a second stream, forked after the plan kernel and joined before the scan
    const bool both = B.n_model[0] > 0 && B.n_model[1] > 0;
    if (both) {
      MHB_CUDA(cudaEventRecord(ds->fork, q));
      MHB_CUDA(cudaStreamWaitEvent(ds->aux, ds->fork, 0));
    }
    for (int m = 0; m < 2; ++m) {
      if (B.n_model[m] == 0) continue;
      BatchQueue bq;
      bq.nets = V.nets;
      bq.wave = V.wave;
      bq.order = V.order + static_cast<size_t>(m) * n_nets;
      bq.mb = V.mb + static_cast<size_t>(m) * (n_nets + 1);
      bq.n_order = B.n_model[m];
      bq.ticket = m ? &wc->ticket2 : &wc->ticket;
      bq.total = &wc->model_items[m];
      bq.seg_slot = node_order ? reinterpret_cast<const int32_t*>(ws + B.seg_slot) : nullptr;
      MHB_CUDA(launch_walk_batched(model_view(gall, m), c, bq, wc, m, (m == 1 && both) ? ds->aux : q));
    }
    if (both) {
      MHB_CUDA(cudaEventRecord(ds->join[0], ds->aux));
      MHB_CUDA(cudaStreamWaitEvent(q, ds->join[0], 0));
    }
    if (timed) MHB_CUDA(mark(ds->timer[2], q));
    cudaError_t e = scan_any<long long, SumOp<long long>, false, int32_t>(c.item_cnt, c.item_off,
                                                                         ScanLen{items_max, &wc->wave_items, 1},
                                                        true, nullptr, &wc->out_end, true, scan_state, q);
    MHB_CUDA(e);
    batch_pair_counts_kernel<<<grid_for(pair_count, 256, 1024), 256, 0, q>>>(V, c.item_off, pair_counts,
                                                                              pair_count);
    note_launches(1);
    MHB_CUDA(cudaGetLastError());
    if (out.csr_off && node_order) {
      batch_csr_off_kernel<<<grid_for(B.csr_max, kCsrOffChunk, static_cast<unsigned>(sm_count()) * 8u), 256, 0, q>>>(
          V, reinterpret_cast<const long long*>(ws + B.rowoff_node), c.item_off, out.csr_off);
      note_launches(1);
      MHB_CUDA(cudaGetLastError());
    } else if (out.csr_off) {
      batch_csr_count_kernel<<<grid_for(B.csr_max, 256, static_cast<unsigned>(sm_count()) * 8u), 256, 0, q>>>(
          V, gall.rank, gall.rowoff, c.item_off, out.csr_off);
      note_launches(1);
      MHB_CUDA(cudaGetLastError());
      e = scan_any<long long, SumOp<long long>>(out.csr_off, out.csr_off, ScanLen{B.csr_max, &wc->num_segments, 1},
                                                true, nullptr, nullptr, false, scan_state, q);
      MHB_CUDA(e);
    }
    BatchEmitParams P{V, gall, c.item_cnt, c.item_base, c.item_off, c.staging, c.staging_cap, out, c.key0,
                      B.n_model[1] > 0, node_order ? reinterpret_cast<const int2*>(ws + B.slot_ik) : nullptr};
    batch_emit_kernel<<<grid_for(items_max, kBatchEmitWarps * kEmitGroup, static_cast<unsigned>(sm_count()) * 5u),
                        kBatchEmitWarps * 32, 0, q>>>(P);
    note_launches(1);
    MHB_CUDA(cudaGetLastError());
    MHB_CUDA(cudaMemcpyAsync(hback, wc, sizeof(Ctrl), cudaMemcpyDeviceToHost, q));
    MHB_CUDA(cudaMemcpyAsync(hback + sizeof(Ctrl), pair_counts, 8 * static_cast<size_t>(pair_count),
                             cudaMemcpyDeviceToHost, q));
    return MH_OK;
  };
  struct WaveKey {
    int tag, device;
    const void *ws, *src, *dst, *w, *csr_off, *csr_idx, *csr_w, *pinned;
    size_t ws_bytes;
    int64_t items_max, pair_count, capacity;
    unsigned long long fingerprint, seed;
    uint32_t flags, num_samples;
    int n_nets, timed;
  } key;
  memset(&key, 0, sizeof(key));
  key.tag = 2;
  MHB_CUDA(cudaGetDevice(&key.device));
  key.ws = workspace;
  key.src = out.src;
  key.dst = out.dst;
  key.w = out.w;
  key.csr_off = out.csr_off;
  key.csr_idx = out.csr_idx;
  key.csr_w = out.csr_w;
  key.pinned = hshare;
  key.ws_bytes = workspace_bytes;
  key.items_max = items_max;
  key.pair_count = pair_count;
  key.capacity = capacity_edges;
  key.fingerprint = V.fingerprint;
  key.seed = params->seed;
  key.flags = fl;
  key.num_samples = params->num_samples;
  key.n_nets = n_nets;
  key.timed = timed;

  if (timed) MHB_CUDA(cudaEventRecord(ds->timer[0], s));
  int64_t launches = 0;
  rc = run_graphed(&key, sizeof(key), s, ds, enqueue, &launches);
  if (rc != MH_OK) return rc;
  if (timed) MHB_CUDA(cudaEventRecord(ds->timer[3], s));
  MHB_CUDA(cudaStreamSynchronize(s));
  mh_call_info info{launches, (B.n_model[0] > 0) + (B.n_model[1] > 0), 1, 0.0, 0.0, 0.0, 0.0};
  if (timed) {
    float a = 0.f, b = 0.f, t = 0.f;
    cudaEventElapsedTime(&a, ds->timer[1], ds->timer[2]);
    cudaEventElapsedTime(&b, ds->timer[2], ds->timer[3]);
    cudaEventElapsedTime(&t, ds->timer[0], ds->timer[3]);
    info.walk_ms = a;
    info.emit_ms = b;
    info.total_ms = t;
  }
  record_call_info(info);
  Ctrl hc;
  memcpy(&hc, hback, sizeof(Ctrl));
  memcpy(h_edges_per_pair, hback + sizeof(Ctrl), 8 * static_cast<size_t>(pair_count));
  if (h_stats)
    for (int k = 0; k < MH_NUM_STATS; ++k) h_stats[k] = hc.stats[k];
  if (hc.status & kStNotPrepared) {
    set_error("the workspace does not hold mh_batch_prepare's result for these networks and params");
    return MH_ERR_ARG;
  }
  if (hc.status & kStWaveItems) {
    set_error("the wave has %llu work items and %llu CSR offsets; max_wave_items allows %lld and %lld", hc.key_or,
              hc.key_and, static_cast<long long>(items_max), static_cast<long long>(B.csr_max));
    return MH_ERR_WORKSPACE;
  }
  rc = status_code(hc.status & ~kStCapacity, 0, 0);
  if (rc != MH_OK) return rc;
  int64_t total = 0;
  for (int64_t k = 0; k < pair_count; ++k) total += h_edges_per_pair[k];
  if (total > capacity_edges || (hc.status & kStCapacity)) {
    set_error("the wave has %lld edges, capacity_edges is %lld", static_cast<long long>(total),
              static_cast<long long>(capacity_edges));
    return MH_ERR_CAPACITY;
  }
  return MH_OK;
}

}  // extern "C"
