// Node order (Sec. 2.4 step (i): ascending alpha; Algorithm 1: ascending
// alpha + beta), i.e. descending x for UBCM and descending a = x*y for UECM,
// ties by ascending original id; then the rank-order copies the walk reads.
//
// Keys are non-negative doubles, whose bit patterns order like the values;
// the sort key is the complement, which turns descending values into
// ascending integers.  Three paths by set size, with the same result:
//  * up to 24,576 nodes: 512-key tile sorts in shared memory, a merge of
//    groups of four tiles into 2048-key runs, and a merge that ranks every
//    node against the other runs with all keys in shared memory and writes
//    the rank-order arrays and the suffix top-2 of y directly;
//  * up to 65,536 nodes: 2048-key tile sorts and a merge that searches every
//    32nd key in shared memory;
//  * larger sets: LSD radix sort of the key bits, 8 bits per pass, stable
//    (one-sweep passes up to 2 M keys, histogram + scan + scatter beyond),
//    then a gather and, for UECM, a reverse scan for the suffix top-2.
//    Passes whose digit is the same for every key (found from the OR and AND
//    of all keys) copy instead of ranking, so the buffer parity never depends
//    on the data.
// The same radix kernels sort the symmetric CSR layout's (sample, rank) keys.
#include <atomic>
#include <mutex>

#include "mh_internal.cuh"
#include "scan.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

__device__ __forceinline__ unsigned long long warp_or(unsigned long long v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}
__device__ __forceinline__ unsigned long long warp_and(unsigned long long v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) v &= __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Checks the parameter domain, writes (key, id) pairs and accumulates the
// histograms of all eight 8-bit digits (one read of the keys for all passes).
__global__ void __launch_bounds__(256) validate_keys_kernel(int model, const double* __restrict__ x,
                                                             const double* __restrict__ y, int64_t n,
                                                             unsigned long long* __restrict__ keys,
                                                             int32_t* __restrict__ vals, unsigned* ghist,
                                                             Ctrl* ctrl) {
  __shared__ unsigned hist[8 * 256];
  for (int t = threadIdx.x; t < 8 * 256; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  unsigned long long kor = 0, kand = ~0ull;
  bool bad = false;
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < n;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double xu = x[u];
    bad |= !(xu >= 0.0 && xu <= 1e150);
    double v = xu;
    if (model == MH_UECM) {
      const double yu = y[u];
      bad |= !(yu >= 0.0 && yu < 1.0);
      v = xu * yu;
    }
    v = (v > 0.0) ? v : 0.0;  // -0.0 sorts as +0.0; a bad input is reported through the status
    const unsigned long long key = ~static_cast<unsigned long long>(__double_as_longlong(v));
    keys[u] = key;
    vals[u] = static_cast<int32_t>(u);
    kor |= key;
    kand &= key;
#pragma unroll
    for (int p = 0; p < 8; ++p) atomicAdd(&hist[p * 256 + static_cast<int>((key >> (8 * p)) & 0xFF)], 1u);
  }
  kor = warp_or(kor);
  kand = warp_and(kand);
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&ctrl->key_or, kor);
    atomicAnd(&ctrl->key_and, kand);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctrl->status, kStDomain);
  __syncthreads();
  for (int t = threadIdx.x; t < 8 * 256; t += blockDim.x)
    if (hist[t]) atomicAdd(&ghist[t], hist[t]);
}

__device__ __forceinline__ bool digit_constant(const Ctrl* ctrl, int shift) {
  return (((ctrl->key_or ^ ctrl->key_and) >> shift) & 0xFFull) == 0ull;
}

// Length of a sort: n, or the device count *dev_len when given (at most n).
__device__ __forceinline__ int64_t sort_len(int64_t n, const long long* dev_len) {
  if (!dev_len) return n;
  const long long v = *dev_len;
  return v < 0 ? 0 : (v < n ? v : n);
}

// hist[d * tiles + tile] = number of keys with digit d in the tile.  With
// ctrl, passes whose digit is constant over all keys are skipped (copy).
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const unsigned long long* __restrict__ keys,
                                                                  int64_t n, int shift, unsigned* __restrict__ hist,
                                                                  int64_t tiles, const Ctrl* ctrl,
                                                                  const long long* dev_len) {
  if (ctrl && digit_constant(ctrl, shift)) return;
  n = sort_len(n, dev_len);
  __shared__ unsigned counts[256];
  counts[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortIPT; ++r) {
    const int64_t e = base + r * kSortThreads + threadIdx.x;
    if (e < n) atomicAdd(&counts[(keys[e] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  hist[static_cast<int64_t>(threadIdx.x) * tiles + blockIdx.x] = counts[threadIdx.x];
}

// Stable scatter: the tile is processed in rounds of 256 keys in position
// order; a key's destination is its digit's global base + the count of equal
// digits in earlier rounds + in earlier warps of this round + earlier lanes.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const unsigned long long* __restrict__ kin, const int32_t* __restrict__ vin, unsigned long long* __restrict__ kout,
    int32_t* __restrict__ vout, int64_t n, int shift, const unsigned* __restrict__ hist, int64_t tiles,
    const Ctrl* ctrl, const long long* dev_len) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
  n = sort_len(n, dev_len);
  if (ctrl && digit_constant(ctrl, shift)) {
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const int64_t e = base + r * kSortThreads + threadIdx.x;
      if (e < n) {
        kout[e] = kin[e];
        vout[e] = vin[e];
      }
    }
    return;
  }
  constexpr int kWarps = kSortThreads / 32;
  __shared__ unsigned wcount[kWarps][256];
  __shared__ unsigned run[256];
  __shared__ unsigned gbase[256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  gbase[t] = hist[static_cast<int64_t>(t) * tiles + blockIdx.x];
  run[t] = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) wcount[w][t] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortIPT; ++r) {
    const int64_t e = base + r * kSortThreads + t;
    const bool valid = e < n;
    const unsigned long long k = valid ? kin[e] : 0ull;
    const int32_t v = valid ? vin[e] : 0;
    const unsigned d = valid ? static_cast<unsigned>((k >> shift) & 0xFF) : 0x100u + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank_in_warp = __popc(peers & lt);
    if (valid && rank_in_warp == 0) wcount[warp][d] = __popc(peers);
    __syncthreads();
    {
      unsigned acc = run[t];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const unsigned c = wcount[w][t];
        wcount[w][t] = acc;
        acc += c;
      }
      run[t] = acc;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = gbase[d] + wcount[warp][d] + rank_in_warp;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcount[w][t] = 0;
    __syncthreads();
  }
}

__device__ __forceinline__ float2 split2(double v) {
  const df2 d = df_from_double(v);
  return make_float2(d.hi, d.lo);
}

constexpr int kSortLookBack = 8;  // predecessor tiles read per look-back step

// Two sets of look-back state, used by passes of alternate parity: a pass
// clears, tile by tile, the set the next pass uses (the previous pass, its
// last user, has finished), so no block clears the whole state alone.
struct SortState {
  unsigned long long* words[2];  // per (tile, digit): count << 2 | flag (1 aggregate, 2 inclusive)
  unsigned* counters[2];         // [0] tile ticket
};

// One LSD pass (one-sweep): a tile claimed by ticket ranks its keys stably
// (rounds of 256 keys in position order: earlier rounds, earlier warps,
// earlier lanes), finds each digit's count in earlier tiles by decoupled
// look-back, and scatters to digit base + earlier-tile count + local rank.
// Passes whose digit is the same for every key copy instead.
__global__ void __launch_bounds__(kSortThreads, 2) onesweep_kernel(
    const unsigned long long* __restrict__ kin, const int32_t* __restrict__ vin, unsigned long long* __restrict__ kout,
    int32_t* __restrict__ vout, int64_t n, int pass, const unsigned* __restrict__ ghist, SortState st, Ctrl* ctrl) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ unsigned s_tile;
  __shared__ unsigned wcount[kWarps][256];
  __shared__ unsigned run[256];
  __shared__ unsigned long long dbase[256];  // global start of each digit + earlier tiles
  const int shift = 8 * pass;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  unsigned long long* const words = st.words[pass & 1];
  if (t == 0) s_tile = atomicAdd(&st.counters[pass & 1][0], 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kSortTile;
  st.words[(pass + 1) & 1][tile * 256 + t] = 0ull;  // this tile's share of the next pass's state
  if (tile == 0 && t == 0) st.counters[(pass + 1) & 1][0] = 0u;
  if (digit_constant(ctrl, shift)) {
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const int64_t e = base + r * kSortThreads + t;
      if (e < n) {
        kout[e] = kin[e];
        vout[e] = vin[e];
      }
    }
  } else {
    // exclusive prefix of the digit histogram (thread t owns digit t)
    {
      unsigned v = ghist[pass * 256 + t];
      unsigned inc = v;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, inc, dd);
        if (lane >= dd) inc += o;
      }
      if (lane == 31) wcount[0][warp] = inc;
      __syncthreads();
      unsigned wp = 0;
      for (int w = 0; w < warp; ++w) wp += wcount[0][w];
      dbase[t] = static_cast<unsigned long long>(wp + inc - v);
      run[t] = 0;
      __syncthreads();
#pragma unroll
      for (int w = 0; w < kWarps; ++w) wcount[w][t] = 0;
      __syncthreads();
    }
    // stable local ranks
    unsigned long long k[kSortIPT];
    int32_t v[kSortIPT];
    unsigned dig[kSortIPT], lr[kSortIPT];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const int64_t e = base + r * kSortThreads + t;
      const bool valid = e < n;
      k[r] = valid ? kin[e] : 0ull;
      v[r] = valid ? vin[e] : 0;
      const unsigned d = valid ? static_cast<unsigned>((k[r] >> shift) & 0xFF) : 0x100u + lane;
      dig[r] = d;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const unsigned rank_in_warp = __popc(peers & lt);
      if (valid && rank_in_warp == 0) wcount[warp][d] = __popc(peers);
      __syncthreads();
      {
        unsigned acc = run[t];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const unsigned c = wcount[w][t];
          wcount[w][t] = acc;
          acc += c;
        }
        run[t] = acc;
      }
      __syncthreads();
      lr[r] = valid ? wcount[warp][d] + rank_in_warp : 0u;
      __syncthreads();
#pragma unroll
      for (int w = 0; w < kWarps; ++w) wcount[w][t] = 0;
      __syncthreads();
    }
    // decoupled look-back per digit: counts of digit t in earlier tiles
    {
      const unsigned long long cnt = run[t];
      unsigned long long* my = &words[tile * 256 + t];
      unsigned long long prefix = 0;
      if (tile == 0) {
        atomicExch(my, (cnt << 2) | 2ull);
      } else {
        atomicExch(my, (cnt << 2) | 1ull);
        int64_t p = tile - 1;
        bool done = false;
        while (!done) {  // kSortLookBack predecessor tiles per step
          unsigned long long w[kSortLookBack];
#pragma unroll
          for (int q = 0; q < kSortLookBack; ++q)
            w[q] = (p - q >= 0) ? *reinterpret_cast<const volatile unsigned long long*>(&words[(p - q) * 256 + t])
                                : 2ull;
#pragma unroll
          for (int q = 0; q < kSortLookBack; ++q) {
            if (done) break;
            if (p - q < 0) {
              done = true;
              break;
            }
            for (unsigned it = 0; (w[q] & 3ull) == 0ull; ++it) {
              if (it >= kSpinLimit) {
                atomicOr(&ctrl->status, kStTimeout);
                w[q] = 2ull;  // give up; the call reports MH_ERR_DEVICE_TIMEOUT
                break;
              }
              __nanosleep(32);
              w[q] = *reinterpret_cast<const volatile unsigned long long*>(&words[(p - q) * 256 + t]);
            }
            prefix += w[q] >> 2;
            if ((w[q] & 3ull) == 2ull) done = true;
          }
          p -= kSortLookBack;
        }
        atomicExch(my, ((prefix + cnt) << 2) | 2ull);
      }
      dbase[t] += prefix;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
      const int64_t e = base + r * kSortThreads + t;
      if (e < n) {
        const unsigned long long pos = dbase[dig[r]] + lr[r];
        if (pos < static_cast<unsigned long long>(n)) {
          kout[pos] = k[r];
          vout[pos] = v[r];
        } else {
          atomicOr(&ctrl->status, kStInternal);
        }
      }
    }
  }
}


// Rank-order copies of the parameters (FP64 and double-float), ln y for the
// weights, the inverse permutation and the fixed-point segment cost
// floor(min(v, 2^20) * 2^F) (scanned afterwards) of the node u at rank r.
__device__ __forceinline__ void gather_rank(const Net& g, int64_t r, int32_t u, int F) {
  g.perm[r] = u;
  g.rank[u] = static_cast<int32_t>(r);
  const double xu = g.x[u];
  g.xs[r] = xu;
  g.xdf[r] = split2(xu);
  double v = xu;
  if (g.model == MH_UECM) {
    const double yu = g.y[u];
    g.ys[r] = yu;
    v = xu * yu;
    g.as[r] = v;
    g.adf[r] = split2(v);
    g.ydf[r] = split2(yu);
    g.lny[r] = split2(log(yu));
    g.top[r] = Top2{top2_entry(yu), 0.0};  // scanned in reverse into suffix top-2
  }
  const double vc = v > 0x1p20 ? 0x1p20 : v;
  g.Q[r] = static_cast<unsigned long long>(ldexp(vc, F));
}

// Block 0's share of a gather: the sentinel top[n].
__device__ __forceinline__ void gather_tables(const Net& g) {
  if (threadIdx.x == 0 && g.model == MH_UECM) g.top[g.n] = Top2{0.0, 0.0};
}

__device__ __forceinline__ int top_scale(const Net& g, int32_t top) {
  const double vmax = (g.model == MH_UBCM) ? g.x[top] : g.x[top] * g.y[top];
  return proxy_scale(vmax, g.n);
}

__global__ void __launch_bounds__(256) gather_kernel(Net g, const int32_t* __restrict__ sorted_ids) {
  if (blockIdx.x == 0) gather_tables(g);
  const int F = top_scale(g, sorted_ids[0]);
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < g.n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    gather_rank(g, r, sorted_ids[r], F);
}

// ---- small node sets: tile sorts + merge by rank ---------------------------------
// Up to kMergeMaxTiles tiles of kSortTile keys.  Each block validates and
// sorts one tile in shared memory by (key, id), a total order since ids are
// distinct: every warp sorts 64 entries with a bitonic network over
// shuffles, then five merge levels double the sorted runs, each entry moving
// to its own position in its run plus the number of smaller entries in the
// partner run (a binary search).  For UECM the block also writes, for every
// position of the sorted tile, the two largest y at that position or later.
// The merge kernel then finds every node's rank as its position in its own
// tile plus, for every other tile, the number of smaller entries there (a
// search over every 32nd entry kept in shared memory, then five steps in the
// tile); the two largest y among ranks >= r combine the tiles' suffixes at
// those positions.  The order is the radix sort's: descending value, ties by
// ascending id.
constexpr int kMergeThreads = 256;
constexpr int kMergeGroup = 8;                             // threads per node in the merge
constexpr int kMergeStride = 32;                           // tile entries per shared sample
constexpr int kMergeSamples = kSortTile / kMergeStride;    // samples per tile

__device__ __forceinline__ bool key_less(unsigned long long ka, int32_t ia, unsigned long long kb, int32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Entries of 64-long warp runs: lane holds indices lane and lane + 32.
__device__ __forceinline__ void warp_bitonic64(unsigned long long& k0, int32_t& i0, unsigned long long& k1,
                                               int32_t& i1) {
  const unsigned lane = threadIdx.x & 31;
#pragma unroll
  for (unsigned k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (unsigned j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // partner in the same lane; k == 64, ascending
        if (key_less(k1, i1, k0, i0)) {
          const unsigned long long tk = k0;
          const int32_t ti = i0;
          k0 = k1;
          i0 = i1;
          k1 = tk;
          i1 = ti;
        }
      } else {
        const unsigned long long pk0 = __shfl_xor_sync(0xffffffffu, k0, j);
        const int32_t pi0 = __shfl_xor_sync(0xffffffffu, i0, j);
        const unsigned long long pk1 = __shfl_xor_sync(0xffffffffu, k1, j);
        const int32_t pi1 = __shfl_xor_sync(0xffffffffu, i1, j);
        const bool lower = (lane & j) == 0;
        // index lane: ascending iff bit k of lane is clear; index lane + 32: bit k of lane + 32
        const bool asc0 = (lane & k) == 0, asc1 = ((lane + 32) & k) == 0;
        const bool pl0 = key_less(pk0, pi0, k0, i0), pl1 = key_less(pk1, pi1, k1, i1);
        if ((asc0 == lower) == pl0) {  // keep the smaller when asc0 == lower
          k0 = pk0;
          i0 = pi0;
        }
        if ((asc1 == lower) == pl1) {
          k1 = pk1;
          i1 = pi1;
        }
      }
    }
  }
}

// Number of entries of the sorted run [run, run + len) below (k, id); len a power of two.
__device__ __forceinline__ int smem_rank(const unsigned long long* sk, const int32_t* si, int run, int len,
                                         unsigned long long k, int32_t id) {
  int pos = 0;
  for (int step = len; step >= 1; step >>= 1)
    if (pos + step <= len && key_less(sk[run + pos + step - 1], si[run + pos + step - 1], k, id)) pos += step;
  return pos;
}

template <int kTile>
__global__ void __launch_bounds__(kTile / 2) tile_sort_kernel(int model, const double* __restrict__ x,
                                                                 const double* __restrict__ y, int64_t n,
                                                                 unsigned long long* __restrict__ kout,
                                                                 int32_t* __restrict__ vout, Top2* __restrict__ tsuf,
                                                                 Ctrl* ctrl, unsigned* clear, int64_t clear_words) {
  __shared__ unsigned long long sk[kTile];
  __shared__ int32_t si[kTile];
  __shared__ Top2 warp_sums[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + t; w < clear_words;
       w += static_cast<int64_t>(gridDim.x) * blockDim.x)
    clear[w] = 0u;  // single-pass scan states for the bound prep that follows
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  bool bad = false;
  unsigned long long k[2];
  int32_t id[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t u = base + 64 * warp + 32 * h + lane;
    k[h] = ~0ull;  // padding: distinct ids above every node id sort after all nodes, zero-valued ones included
    id[h] = INT32_MAX - (64 * warp + 32 * h + lane);
    if (u < n) {
      const double xu = x[u];
      bad |= !(xu >= 0.0 && xu <= 1e150);
      double v = xu;
      if (model == MH_UECM) {
        const double yu = y[u];
        bad |= !(yu >= 0.0 && yu < 1.0);
        v = xu * yu;
      }
      v = (v > 0.0) ? v : 0.0;  // -0.0 sorts as +0.0; a bad input is reported through the status
      k[h] = ~static_cast<unsigned long long>(__double_as_longlong(v));
      id[h] = static_cast<int32_t>(u);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&ctrl->status, kStDomain);
  warp_bitonic64(k[0], id[0], k[1], id[1]);
  int pos[2] = {64 * warp + lane, 64 * warp + 32 + lane};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    sk[pos[h]] = k[h];
    si[pos[h]] = id[h];
  }
  __syncthreads();
  for (int len = 64; len < kTile; len <<= 1) {
    int np[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int run = pos[h] & ~(len - 1), partner = run ^ len;
      np[h] = (run & ~(2 * len - 1)) + (pos[h] - run) + smem_rank(sk, si, partner, len, k[h], id[h]);
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      pos[h] = np[h];
      sk[pos[h]] = k[h];
      si[pos[h]] = id[h];
    }
    __syncthreads();
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (base + pos[h] < n) {
      kout[base + pos[h]] = k[h];
      vout[base + pos[h]] = id[h];
    }
  }
  if (model != MH_UECM) return;
  // suffix top-2 of y in sorted order: thread t holds positions kTile - 1 - 2t
  // and kTile - 2 - 2t, so an inclusive scan in thread order runs from the
  // tile's end
  double* sy = reinterpret_cast<double*>(sk);
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) sy[pos[h]] = (base + pos[h] < n) ? top2_entry(y[id[h]]) : 0.0;
  __syncthreads();
  const int p_hi = kTile - 1 - 2 * t, p_lo = p_hi - 1;
  const Top2 one_hi{sy[p_hi], 0.0}, one_lo{sy[p_lo], 0.0};
  Top2Op op;
  Top2 v = op(one_hi, one_lo);
  block_inclusive_scan<Top2, Top2Op>(v, warp_sums);  // suffix from p_lo on
  Top2 prev = shfl_up(v, 1);
  __shared__ Top2 last_of_warp[32];
  if (lane == 31) last_of_warp[warp] = v;
  __syncthreads();
  if (lane == 0) prev = warp > 0 ? last_of_warp[warp - 1] : Top2Op::identity();
  if (base + p_hi < n) tsuf[base + p_hi] = op(prev, one_hi);
  if (base + p_lo < n) tsuf[base + p_lo] = v;
}

__global__ void __launch_bounds__(kMergeThreads) merge_gather_kernel(Net g, const unsigned long long* __restrict__ keys,
                                                                     const int32_t* __restrict__ ids,
                                                                     const Top2* __restrict__ tsuf, int tiles,
                                                                     Ctrl* ctrl) {
  // tile q's samples start at q * kSampleStride: the padding puts the eight
  // tiles a warp searches at once in different banks
  constexpr int kSampleStride = kMergeSamples + 1;
  __shared__ unsigned long long sk[kMergeMaxTiles * kSampleStride];
  __shared__ int32_t si[kMergeMaxTiles * kSampleStride];
  __shared__ int32_t s_top;
  const int64_t n = g.n;
  for (int q = threadIdx.x; q < tiles * kMergeSamples; q += blockDim.x) {
    const int tq = q / kMergeSamples, sq = q % kMergeSamples;
    const int64_t e = static_cast<int64_t>(tq) * kSortTile + static_cast<int64_t>(sq) * kMergeStride;
    sk[tq * kSampleStride + sq] = e < n ? keys[e] : ~0ull;
    si[tq * kSampleStride + sq] = e < n ? ids[e] : INT32_MAX;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the largest value heads one of the tiles
    int best = 0;
    for (int q = 1; q < tiles; ++q)
      if (key_less(sk[q * kSampleStride], si[q * kSampleStride], sk[best * kSampleStride], si[best * kSampleStride]))
        best = q;
    s_top = si[best * kSampleStride];
  }
  if (blockIdx.x == 0) gather_tables(g);
  __syncthreads();
  const bool uecm = g.model == MH_UECM;
  const int F = top_scale(g, s_top);
  const int64_t e = blockIdx.x * static_cast<int64_t>(kMergeThreads / kMergeGroup) + threadIdx.x / kMergeGroup;
  const int gl = threadIdx.x % kMergeGroup;
  const bool live = e < n;
  const unsigned long long k = live ? keys[e] : 0ull;
  const int32_t id = live ? ids[e] : 0;
  const int own = static_cast<int>(e / kSortTile);
  long long below = 0;     // entries of this thread's tiles below (k, id)
  Top2 above{0.0, 0.0};    // two largest y of those tiles' entries above (k, id)
  Top2Op op;
  for (int q = gl; live && q < tiles; q += kMergeGroup) {
    if (q == own) continue;
    const int64_t tb = static_cast<int64_t>(q) * kSortTile;
    const int len = static_cast<int>((n - tb) < kSortTile ? (n - tb) : kSortTile);
    const int ns = (len + kMergeStride - 1) / kMergeStride;
    const unsigned long long* qk = sk + q * kSampleStride;
    const int32_t* qi = si + q * kSampleStride;
    int s = 0;  // samples below (k, id)
#pragma unroll
    for (int half = kMergeSamples; half >= 1; half >>= 1)
      if (s + half <= ns && key_less(qk[s + half - 1], qi[s + half - 1], k, id)) s += half;
    int c = 0;  // entries of tile q below (k, id)
    if (s > 0) {
      c = (s - 1) * kMergeStride + 1;
#pragma unroll
      for (int half = kMergeStride / 2; half >= 1; half >>= 1) {
        const int at = c + half - 1;
        if (at < len) {
          const unsigned long long ka = keys[tb + at];
          if (ka < k || (ka == k && ids[tb + at] < id)) c += half;  // ids only on a tie
        }
      }
    }
    below += c;
    if (uecm && c < len) above = op(above, tsuf[tb + c]);
  }
#pragma unroll
  for (int d = kMergeGroup / 2; d; d >>= 1) {
    below += __shfl_xor_sync(0xffffffffu, below, d);
    above = op(above, Top2{__shfl_xor_sync(0xffffffffu, above.a, d), __shfl_xor_sync(0xffffffffu, above.b, d)});
  }
  if (!live || gl != 0) return;
  const int64_t r = e - static_cast<int64_t>(own) * kSortTile + below;
  if (r >= n) {
    atomicOr(&ctrl->status, kStInternal);
    return;
  }
  gather_rank(g, r, id, F);
  if (uecm) g.top[r] = op(tsuf[e], above);  // two largest y among ranks >= r
}

// Sets of at most kMergeSmemMax nodes: tiles of kSmallTile keys; groups of
// kGroupTiles tiles merged into runs of kRun keys; then every merge block
// holds all run-sorted keys in shared memory, so a node's searches in the
// other runs (kMergeGroup threads per node, a binary search per run; ids are
// read only on equal keys) never leave the SM.  The node's rank-order
// copies are then written by one thread per node.
constexpr int kSmallTile = 512;
constexpr int kGroupTiles = 4;
constexpr int kRun = kSmallTile * kGroupTiles;      // 2048
constexpr int kMergeSmemMax = 24576;                // 8-byte keys in shared memory
constexpr int kSmemThreads = 1024;
constexpr int kSmemNodes = kSmemThreads / kMergeGroup;  // nodes per block

// Merges the kGroupTiles sorted tiles of a group into one run: block b
// places the entries of tile b at their positions in the run (own position
// plus a binary search in each other tile of the group), and combines the
// tiles' suffix top-2 at those positions into the run's.
__global__ void __launch_bounds__(kSmallTile / 2) group_merge_kernel(
    int64_t n, const unsigned long long* __restrict__ kin, const int32_t* __restrict__ vin,
    const Top2* __restrict__ sin, unsigned long long* __restrict__ kout, int32_t* __restrict__ vout,
    Top2* __restrict__ sout, int uecm) {
  __shared__ unsigned long long sk[kRun];
  __shared__ int32_t si[kRun];
  const int tile = blockIdx.x;
  const int64_t gbase = static_cast<int64_t>(tile / kGroupTiles) * kRun;
  const int own = tile % kGroupTiles;
  const int64_t glen64 = n - gbase < kRun ? n - gbase : kRun;
  const int glen = static_cast<int>(glen64);
  {
    constexpr int kPer = kRun / (kSmallTile / 2);  // entries per thread, all loads in flight together
    unsigned long long kv[kPer];
    int32_t iv[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int t = threadIdx.x + u * (kSmallTile / 2);
      if (t < glen) {
        kv[u] = kin[gbase + t];
        iv[u] = vin[gbase + t];
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int t = threadIdx.x + u * (kSmallTile / 2);
      if (t < glen) {
        sk[t] = kv[u];
        si[t] = iv[u];
      }
    }
  }
  __syncthreads();
  Top2Op op;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = threadIdx.x + h * (kSmallTile / 2);
    const int p = own * kSmallTile + l;  // position within the group
    if (p >= glen) continue;
    const unsigned long long k = sk[p];
    const int32_t id = si[p];
    int r = l;
    Top2 suf = uecm ? sin[gbase + p] : Top2{0.0, 0.0};
    for (int q = 0; q < kGroupTiles; ++q) {
      if (q == own) continue;
      const int tb = q * kSmallTile;
      const int len = glen - tb < kSmallTile ? glen - tb : kSmallTile;
      if (len <= 0) continue;
      int c = 0;
#pragma unroll
      for (int step = kSmallTile; step >= 1; step >>= 1) {
        const int at = c + step - 1;
        if (at < len && key_less(sk[tb + at], si[tb + at], k, id)) c += step;
      }
      r += c;
      if (uecm && c < len) suf = op(suf, sin[gbase + tb + c]);
    }
    kout[gbase + r] = k;
    vout[gbase + r] = id;
    if (uecm) sout[gbase + r] = suf;
  }
}

// Run q's keys start at q * kRunStride in shared memory: the padding puts
// the eight runs a warp searches at once in different banks.
constexpr int kRunStride = kRun + 2;

__host__ __device__ inline size_t merge_smem_bytes(int64_t n) {
  return 8 * static_cast<size_t>((n + kRun - 1) / kRun) * kRunStride;
}

__global__ void __launch_bounds__(kSmemThreads) merge_smem_kernel(Net g, const unsigned long long* __restrict__ keys,
                                                                  const int32_t* __restrict__ ids,
                                                                  const Top2* __restrict__ tsuf, int runs,
                                                                  Ctrl* ctrl) {
  extern __shared__ unsigned long long smk[];
  __shared__ long long s_rank[kSmemNodes];
  __shared__ Top2 s_above[kSmemNodes];
  __shared__ int32_t s_top;
  const int64_t n = g.n;
  {
    // pairs of keys by 16-byte loads (the key array is 256-byte aligned), eight in flight per thread
    constexpr int kUnroll = 8;
    const int64_t pairs = n / 2;
    const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys);
    for (int64_t p0 = threadIdx.x; p0 < pairs; p0 += static_cast<int64_t>(kUnroll) * blockDim.x) {
      ulonglong2 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t p = p0 + static_cast<int64_t>(u) * blockDim.x;
        if (p < pairs) v[u] = k2[p];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t p = p0 + static_cast<int64_t>(u) * blockDim.x;
        if (p < pairs) {
          const int64_t e = 2 * p;  // e and e + 1 share a run (kRun is even)
          unsigned long long* d = smk + (e / kRun) * kRunStride + e % kRun;
          d[0] = v[u].x;
          d[1] = v[u].y;
        }
      }
    }
    if ((n & 1) && threadIdx.x == 0) smk[((n - 1) / kRun) * kRunStride + (n - 1) % kRun] = keys[n - 1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the largest value heads one of the runs
    int best = 0;
    for (int q = 1; q < runs; ++q) {
      const unsigned long long kq = smk[q * kRunStride], kb = smk[best * kRunStride];
      if (kq < kb || (kq == kb && ids[q * kRun] < ids[best * kRun])) best = q;
    }
    s_top = ids[best * kRun];
  }
  if (blockIdx.x == 0) gather_tables(g);
  __syncthreads();
  const bool uecm = g.model == MH_UECM;
  const int F = top_scale(g, s_top);
  const int local = threadIdx.x / kMergeGroup, gl = threadIdx.x % kMergeGroup;
  Top2Op op;
  // batches of kSmemNodes nodes, one block per SM holding the keys once
  for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * kSmemNodes; e0 < n;
       e0 += static_cast<int64_t>(gridDim.x) * kSmemNodes) {
    const int64_t e = e0 + local;
    const bool live = e < n;
    const int own = static_cast<int>(e / kRun);
    const unsigned long long k = live ? smk[own * kRunStride + e % kRun] : 0ull;
    const int32_t id = live ? ids[e] : 0;
    long long below = 0;
    Top2 above{0.0, 0.0};
    for (int q = gl; live && q < runs; q += kMergeGroup) {
      if (q == own) continue;
      const int64_t tb = static_cast<int64_t>(q) * kRun;
      const unsigned long long* tk = smk + q * kRunStride;
      const int len = static_cast<int>((n - tb) < kRun ? (n - tb) : kRun);
      int c = 0;  // entries of run q below (k, id)
#pragma unroll
      for (int step = kRun; step >= 1; step >>= 1) {
        const int at = c + step - 1;
        if (at < len) {
          const unsigned long long ka = tk[at];
          if (ka < k || (ka == k && ids[tb + at] < id)) c += step;  // ids only on a tie
        }
      }
      below += c;
      if (uecm && c < len) above = op(above, tsuf[tb + c]);
    }
#pragma unroll
    for (int d = kMergeGroup / 2; d; d >>= 1) {
      below += __shfl_xor_sync(0xffffffffu, below, d);
      above = op(above, Top2{__shfl_xor_sync(0xffffffffu, above.a, d), __shfl_xor_sync(0xffffffffu, above.b, d)});
    }
    if (live && gl == 0) {
      s_rank[local] = e - static_cast<int64_t>(own) * kRun + below;
      s_above[local] = above;
    }
    __syncthreads();
    const int64_t e2 = e0 + threadIdx.x;
    if (threadIdx.x < kSmemNodes && e2 < n) {
      const long long r = s_rank[threadIdx.x];
      if (r >= n) {
        atomicOr(&ctrl->status, kStInternal);
      } else {
        gather_rank(g, r, ids[e2], F);
        if (uecm) g.top[r] = op(tsuf[e2], s_above[threadIdx.x]);  // two largest y among ranks >= r
      }
    }
    __syncthreads();
  }
}

// The logarithm table of the walk's and the emit's double-float logarithm
// (Tang's method).  It depends on nothing but its index, so it is built once
// per device (FP64 divisions and logarithms, slow at GB300's FP64 rate) and
// every call reads it.
__device__ LnEntry g_ln_table[kLnTable];

__global__ void ln_table_kernel(LnEntry* tab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kLnTable) ln_table_entry(tab, k);
}

}  // namespace

// The table is built once per device, under a lock (calls on several host
// threads may race to build it), by one kernel on `s` (or on a stream of its
// own when s is null), waited for before the pointer is published.
LnEntry* ln_table_ptr(cudaStream_t s) {
  static std::atomic<LnEntry*> ptr[64];
  static std::mutex build_lock;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  LnEntry* p = ptr[dev].load(std::memory_order_acquire);
  if (p) return p;
  std::lock_guard<std::mutex> guard(build_lock);
  p = ptr[dev].load(std::memory_order_acquire);
  if (p) return p;
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_ln_table) != cudaSuccess) return nullptr;
  cudaStream_t st = s;
  if (!st && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  ln_table_kernel<<<(kLnTable + 255) / 256, 256, 0, st>>>(static_cast<LnEntry*>(sym));
  const bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  if (!s) cudaStreamDestroy(st);
  if (!ok) return nullptr;
  p = static_cast<LnEntry*>(sym);
  ptr[dev].store(p, std::memory_order_release);
  return p;
}

cudaError_t launch_validate_keys(const Net& g, unsigned long long* keys, int32_t* vals, unsigned* ghist, Ctrl* ctrl,
                                 cudaStream_t s) {
  const unsigned grid = grid_for(g.n, 256, static_cast<unsigned>(sm_count()) * 4u);
  validate_keys_kernel<<<grid, 256, 0, s>>>(g.model, g.x, g.y, g.n, keys, vals, ghist, ctrl);
  note_launches(1);
  return cudaGetLastError();
}

// Small inputs: eight one-sweep passes (one launch each).  Large inputs:
// per pass a tile histogram, a scan of the (digit, tile) counts and a stable
// scatter, which keeps every launch bandwidth-bound.
constexpr int64_t kOneSweepMaxTiles = 1024;

cudaError_t launch_sort(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  auto* k0 = reinterpret_cast<unsigned long long*>(ws + L.keys0);
  auto* k1 = reinterpret_cast<unsigned long long*>(ws + L.keys1);
  auto* v0 = reinterpret_cast<int32_t*>(ws + L.vals0);
  auto* v1 = reinterpret_cast<int32_t*>(ws + L.vals1);
  const unsigned* ghist = reinterpret_cast<const unsigned*>(ws + L.ghist);
  auto* sw = reinterpret_cast<unsigned long long*>(ws + L.sort_state);
  auto* sc = reinterpret_cast<unsigned*>(ws + L.sort_counters);
  const int64_t set_words = 256 * (L.tiles > 0 ? L.tiles : 1);
  SortState st{{sw, sw + set_words}, {sc, sc + 2}};
  const ScanState sst{reinterpret_cast<unsigned*>(ws + L.scan_flags), ws + L.scan_values,
                      reinterpret_cast<unsigned*>(ws + L.scan_counters), ctrl, L.scan_tiles};
  auto* hist = reinterpret_cast<unsigned*>(ws + L.hist);
  const unsigned tiles = static_cast<unsigned>(L.tiles);
  for (int pass = 0; pass < 8; ++pass) {
    cudaError_t e;
    if (L.tiles <= kOneSweepMaxTiles) {
      onesweep_kernel<<<tiles, kSortThreads, 0, s>>>(k0, v0, k1, v1, g.n, pass, ghist, st, ctrl);
      note_launches(1);
      e = cudaGetLastError();
    } else {
      const int shift = pass * 8;
      radix_hist_kernel<<<tiles, kSortThreads, 0, s>>>(k0, g.n, shift, hist, L.tiles, ctrl, nullptr);
      note_launches(1);
      e = scan_any<unsigned, SumOp<unsigned>>(hist, hist, ScanLen{256 * L.tiles, nullptr, 1}, true, nullptr, nullptr,
                                              false, sst, s);
      if (e != cudaSuccess) return e;
      radix_scatter_kernel<<<tiles, kSortThreads, 0, s>>>(k0, v0, k1, v1, g.n, shift, hist, L.tiles, ctrl,
                                                            nullptr);
      note_launches(1);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    unsigned long long* kt = k0;
    k0 = k1;
    k1 = kt;
    int32_t* vt = v0;
    v0 = v1;
    v1 = vt;
  }
  return cudaSuccess;  // eight passes: the result is back in keys0 / vals0
}

cudaError_t sort_kernel_attributes(int dev) {
  static bool done[64] = {};
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (done[dev]) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(merge_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(merge_smem_bytes(kMergeSmemMax)));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

cudaError_t launch_sort_merge(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  auto* k1 = reinterpret_cast<unsigned long long*>(ws + L.keys1);
  auto* v1 = reinterpret_cast<int32_t*>(ws + L.vals1);
  auto* clear = reinterpret_cast<unsigned*>(ws + L.scan_counters);
  const int64_t clear_words = static_cast<int64_t>((L.zero_end - L.scan_counters) / 4);
  auto* tsuf = reinterpret_cast<Top2*>(ws + L.tsuf);
  if (g.n <= kMergeSmemMax) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = sort_kernel_attributes(dev);
    if (e != cudaSuccess) return e;
    const int tiles = static_cast<int>((g.n + kSmallTile - 1) / kSmallTile);
    const int runs = static_cast<int>((g.n + kRun - 1) / kRun);
    auto* k0 = reinterpret_cast<unsigned long long*>(ws + L.keys0);
    auto* v0 = reinterpret_cast<int32_t*>(ws + L.vals0);
    auto* tsuf2 = reinterpret_cast<Top2*>(ws + L.tsuf2);
    tile_sort_kernel<kSmallTile><<<tiles, kSmallTile / 2, 0, s>>>(g.model, g.x, g.y, g.n, k1, v1, tsuf, ctrl,
                                                                   clear, clear_words);
    group_merge_kernel<<<tiles, kSmallTile / 2, 0, s>>>(g.n, k1, v1, tsuf, k0, v0, tsuf2, g.model == MH_UECM);
    merge_smem_kernel<<<grid_for(g.n, kSmemNodes, static_cast<unsigned>(sm_count())), kSmemThreads,
                        merge_smem_bytes(g.n), s>>>(g, k0, v0, tsuf2, runs, ctrl);
    note_launches(3);
    return cudaGetLastError();
  }
  const int tiles = static_cast<int>((g.n + kSortTile - 1) / kSortTile);
  tile_sort_kernel<kSortTile><<<tiles, kSortTile / 2, 0, s>>>(g.model, g.x, g.y, g.n, k1, v1, tsuf, ctrl, clear,
                                                               clear_words);
  merge_gather_kernel<<<grid_for(g.n, kMergeThreads / kMergeGroup), kMergeThreads, 0, s>>>(g, k1, v1, tsuf, tiles,
                                                                                            ctrl);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_pair_sort(unsigned long long* keys[2], int32_t* vals[2], int64_t host_len,
                             const long long* dev_len, const int* shifts, int passes, unsigned* hist,
                             const void* scan_state, Ctrl* ctrl, int* out_buf, cudaStream_t s) {
  (void)ctrl;
  const ScanState& sst = *static_cast<const ScanState*>(scan_state);
  const int64_t tiles = (host_len + kSortTile - 1) / kSortTile > 0 ? (host_len + kSortTile - 1) / kSortTile : 1;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    radix_hist_kernel<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(keys[cur], host_len, shifts[p], hist,
                                                                           tiles, nullptr, dev_len);
    note_launches(1);
    cudaError_t e = scan_any<unsigned, SumOp<unsigned>>(hist, hist, ScanLen{256 * tiles, nullptr, 1}, true, nullptr,
                                                        nullptr, false, sst, s);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(
        keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], host_len, shifts[p], hist, tiles, nullptr, dev_len);
    note_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  *out_buf = cur;
  return cudaSuccess;
}

cudaError_t launch_gather(const Net& g, const int32_t* sorted_vals, Ctrl* ctrl, cudaStream_t s) {
  (void)ctrl;
  const unsigned grid = grid_for(g.n, 256, static_cast<unsigned>(sm_count()) * 8u);
  gather_kernel<<<grid, 256, 0, s>>>(g, sorted_vals);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh
