// Device-wide scans in one launch (chained tiles with decoupled look-back).
//
// The length may come from device memory (len = min(host_len, *dev_len *
// mult)) so a scan can follow a kernel that decides the size without a host
// round trip.  Operators are exact (integer sums, max, top-2), so the result
// does not depend on the tiling or on the order tiles finish in.
#pragma once

#include "mh_internal.cuh"

namespace mh {

template <typename T>
struct SumOp {
  __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
  __device__ __forceinline__ static T identity() { return T(0); }
};
struct MaxOp {
  __device__ __forceinline__ double operator()(double a, double b) const { return a > b ? a : b; }
  __device__ __forceinline__ static double identity() { return 0.0; }
};
// Two largest of non-negative doubles.  Every y entering a Top2 is >= +0.0
// (-0.0 is stored as +0.0), so the comparisons use the bit patterns, which
// order like the values: integer compares instead of GB300's slow FP64 pipe.
struct Top2Op {
  __device__ __forceinline__ static bool gt(double a, double b) {
    return static_cast<unsigned long long>(__double_as_longlong(a)) >
           static_cast<unsigned long long>(__double_as_longlong(b));
  }
  __device__ __forceinline__ Top2 operator()(Top2 u, Top2 v) const {
    Top2 r;
    const bool ua = gt(u.a, v.a);
    r.a = ua ? u.a : v.a;
    const double lo = ua ? v.a : u.a;
    const double sb = gt(u.b, v.b) ? u.b : v.b;
    r.b = gt(lo, sb) ? lo : sb;
    return r;
  }
  __device__ __forceinline__ static Top2 identity() { return Top2{0.0, 0.0}; }
};

// y as it enters a Top2: -0.0 becomes +0.0 (the domain check admits y in [0, 1)).
__device__ __forceinline__ double top2_entry(double y) { return y > 0.0 ? y : 0.0; }

__device__ __forceinline__ unsigned shfl_up(unsigned v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ unsigned long long shfl_up(unsigned long long v, int d) {
  return __shfl_up_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ long long shfl_up(long long v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ Top2 shfl_up(Top2 v, int d) {
  return Top2{__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d)};
}

struct ScanLen {
  int64_t host_len;               // upper bound, sizes the grid
  const long long* dev_len;       // optional device length
  int64_t mult;                   // dev length multiplier
  __device__ __forceinline__ int64_t get() const {
    if (!dev_len) return host_len;
    const int64_t v = static_cast<int64_t>(*dev_len) * mult;
    return v < host_len ? v : host_len;
  }
};

// Element e of the logical sequence lives at index e (forward) or len-1-e (reverse).
template <bool kReverse>
__device__ __forceinline__ int64_t scan_index(int64_t e, int64_t len) {
  return kReverse ? len - 1 - e : e;
}

// Inclusive scan of one block's values; returns the block aggregate.
template <typename T, typename Op>
__device__ __forceinline__ T block_inclusive_scan(T& v, T* warp_sums) {
  Op op;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = shfl_up(v, d);
    if (lane >= d) v = op(o, v);
  }
  if (lane == 31) warp_sums[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_sums[lane] : Op::identity();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T o = shfl_up(w, d);
      if (lane >= d) w = op(o, w);
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v = op(warp_sums[warp - 1], v);
  const T agg = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return agg;
}

// Tile aggregates.  The operators are exact and commutative, so a thread
// takes elements k * kScanThreads + tid of the tile (k = 0 .. kScanIPT - 1):
// every load of the warp is one contiguous run.
template <typename T, typename Op, bool kReverse, typename TIn = T>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const TIn* __restrict__ in, ScanLen L,
                                                                    T* __restrict__ partial) {
  __shared__ T warp_sums[kScanThreads / 32];
  const int64_t len = L.get();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  if (base >= len) return;
  Op op;
  T acc = Op::identity();
#pragma unroll
  for (int k = 0; k < kScanIPT; ++k) {
    const int64_t e = base + static_cast<int64_t>(k) * kScanThreads + threadIdx.x;
    if (e < len) acc = op(acc, static_cast<T>(in[scan_index<kReverse>(e, len)]));
  }
  const T agg = block_inclusive_scan<T, Op>(acc, warp_sums);
  if (threadIdx.x == 0) partial[blockIdx.x] = agg;
}

// Exclusive scan of the tile partials with an optional carry-in; writes the
// grand total to *total (which may alias *base: it is read before written).
template <typename T, typename Op>
__global__ void __launch_bounds__(1024) scan_partials_kernel(T* __restrict__ partial, ScanLen L, const T* base,
                                                              T* total) {
  __shared__ T warp_sums[32];
  __shared__ T last_of_warp[32];
  const int64_t len = L.get();
  const int64_t tiles = (len + kScanTile - 1) / kScanTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Op op;
  T carry = base ? *base : Op::identity();
  __syncthreads();
  for (int64_t t0 = 0; t0 < tiles; t0 += blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    T inc = t < tiles ? partial[t] : Op::identity();
    const T agg = block_inclusive_scan<T, Op>(inc, warp_sums);
    T prev = shfl_up(inc, 1);
    if (lane == 31) last_of_warp[warp] = inc;
    __syncthreads();
    if (lane == 0) prev = warp > 0 ? last_of_warp[warp - 1] : Op::identity();
    if (t < tiles) partial[t] = op(carry, prev);
    carry = op(carry, agg);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[tiles] = carry;  // grand total, read by the final pass when len == 0
    if (total) *total = carry;
  }
}

// Scan of each tile with its carry-in.  The tile moves between global and
// shared memory in rounds of kScanThreads contiguous elements (coalesced),
// and each thread scans kScanIPT consecutive elements from shared memory
// (element i stored at i + i / 32, which spreads a thread's consecutive
// elements over the banks).
__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }

template <typename T, typename Op, bool kReverse, typename TIn = T>
__global__ void __launch_bounds__(kScanThreads) scan_final_kernel(const TIn* in, T* out, ScanLen L,
                                                                   const T* __restrict__ partial, bool exclusive,
                                                                   bool write_total_at_len) {
  // `in` and `out` may alias: a block reads all of its tile before it writes.
  __shared__ T warp_sums[kScanThreads / 32];
  __shared__ T last_of_warp[kScanThreads / 32];
  __shared__ T tile[kScanTile + kScanTile / 32];
  const int64_t len = L.get();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  if (len == 0 && blockIdx.x == 0 && threadIdx.x == 0 && write_total_at_len) out[0] = partial[0];
  if (base >= len) return;
  Op op;
#pragma unroll
  for (int k = 0; k < kScanIPT; ++k) {
    const int i = k * kScanThreads + threadIdx.x;
    const int64_t e = base + i;
    tile[scan_pad(i)] = e < len ? static_cast<T>(in[scan_index<kReverse>(e, len)]) : Op::identity();
  }
  __syncthreads();
  T vals[kScanIPT];
  T acc = Op::identity();
#pragma unroll
  for (int k = 0; k < kScanIPT; ++k) {
    vals[k] = tile[scan_pad(threadIdx.x * kScanIPT + k)];
    acc = op(acc, vals[k]);
  }
  T inc = acc;
  block_inclusive_scan<T, Op>(inc, warp_sums);
  // exclusive prefix of this thread = carry-in (+) inclusive of the previous thread
  T prev = shfl_up(inc, 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 31) last_of_warp[warp] = inc;
  __syncthreads();
  if (lane == 0) prev = warp > 0 ? last_of_warp[warp - 1] : Op::identity();
  T run = op(partial[blockIdx.x], prev);
#pragma unroll
  for (int k = 0; k < kScanIPT; ++k) {
    const int i = threadIdx.x * kScanIPT + k;
    const T next = op(run, vals[k]);
    tile[scan_pad(i)] = exclusive ? run : next;
    if (write_total_at_len && base + i == len - 1) out[len] = next;
    run = next;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanIPT; ++k) {
    const int i = k * kScanThreads + threadIdx.x;
    const int64_t e = base + i;
    if (e < len) out[scan_index<kReverse>(e, len)] = tile[scan_pad(i)];
  }
}

// Multi-kernel form (reduce, scan of partials, scan with carry-in) for long
// inputs, where a single-pass look-back would walk back over many tiles.
// scan_tmp must hold ceil(host_len / kScanTile) + 2 elements of T.
template <typename T, typename Op, bool kReverse = false, typename TIn = T>
cudaError_t device_scan(const TIn* in, T* out, ScanLen L, bool exclusive, const T* base, T* total,
                        bool write_total_at_len, T* scan_tmp, cudaStream_t s) {
  const unsigned tiles = grid_for(L.host_len, kScanTile);
  scan_reduce_kernel<T, Op, kReverse, TIn><<<tiles, kScanThreads, 0, s>>>(in, L, scan_tmp);
  scan_partials_kernel<T, Op><<<1, 1024, 0, s>>>(scan_tmp, L, base, total);
  scan_final_kernel<T, Op, kReverse, TIn><<<tiles, kScanThreads, 0, s>>>(in, out, L, scan_tmp, exclusive,
                                                                      write_total_at_len);
  note_launches(3);
  return cudaGetLastError();
}


// ---- single-pass scan (chained tiles, decoupled look-back) ---------------------
// Tiles are claimed in ticket order, so a tile only ever waits on tiles that
// are already running.  Each tile publishes its aggregate, then walks back
// over its predecessors until it meets an inclusive prefix, and publishes
// its own.  Every wait is bounded: after kSpinLimit polls the tile records
// kStTimeout in the status word and publishes anyway, so no block waits
// forever (the call then reports MH_ERR_DEVICE_TIMEOUT).  The last block to
// finish clears the tile states and tickets for the next scan.
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned poll_flag(const unsigned* f) {
  return *reinterpret_cast<const volatile unsigned*>(f);
}

struct ScanState {
  unsigned* flags;     // per tile: 0 empty, 1 aggregate published, 2 inclusive prefix published
  void* values;        // 2 x tiles values of the scanned type: aggregates, then inclusive prefixes
  unsigned* counters;  // [0] tile ticket, [1] finished blocks
  Ctrl* ctrl;          // status word for timeouts
  int64_t max_tiles;   // capacity of `values` (per half)
  unsigned test_stuck_polls = 0;  // MH_TEST_WAIT_TIMEOUT: tile 1 first waits this long on a flag never set
};

// Polls for the MH_TEST_WAIT_TIMEOUT hook; the hook's wait gives up after these.
constexpr unsigned kTestStuckPolls = 4096u;

// A device word that nothing ever writes: the MH_TEST_WAIT_TIMEOUT hook
// waits on it, so that wait can only end by running out of polls.
static __device__ unsigned g_never_set = 0u;

// The hook's wait: the same bounded poll as the look-back's, on a flag that
// is never set, so it always gives up and records kStTimeout.  The scan then
// goes on with its real look-back, so its output stays correct.
__device__ __forceinline__ void test_stuck_wait(Ctrl* ctrl, unsigned polls) {
  for (unsigned it = 0;; ++it) {
    if (poll_flag(&g_never_set) != 0u) return;
    if (it >= polls) {
      atomicOr(&ctrl->status, kStTimeout);
      return;
    }
    __nanosleep(32);
  }
}

// Loads through L2 (a value another block published after a fence).
__device__ __forceinline__ unsigned load_cg(const unsigned* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long load_cg(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ long long load_cg(const long long* p) { return __ldcg(p); }
__device__ __forceinline__ double load_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ Top2 load_cg(const Top2* p) {
  const double* d = reinterpret_cast<const double*>(p);
  return Top2{__ldcg(d), __ldcg(d + 1)};
}

__device__ __forceinline__ unsigned long long shfl_xor(unsigned long long v, int d) {
  return __shfl_xor_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ long long shfl_xor(long long v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ __forceinline__ unsigned shfl_xor(unsigned v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_xor(double v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ __forceinline__ Top2 shfl_xor(Top2 v, int d) {
  return Top2{__shfl_xor_sync(0xffffffffu, v.a, d), __shfl_xor_sync(0xffffffffu, v.b, d)};
}

// Exclusive prefix of tile `tile` from its predecessors' published values,
// by one full warp: lane q reads tile - 1 - q - 32 w in step w, so 32 flags
// and values are in flight at once.  The lanes up to the nearest inclusive
// prefix are combined in lane order's reverse, which is exact because every
// operator here is commutative (integer sums, max, top-2).  Waits on a flag
// are bounded: after kSpinLimit polls the lane records kStTimeout and stops
// waiting (the call then reports MH_ERR_DEVICE_TIMEOUT).
template <typename T, typename Op>
__device__ __forceinline__ T warp_look_back(int64_t tile, const unsigned* flags, const T* agg_v, const T* inc_v,
                                            Ctrl* ctrl) {
  Op op;
  const int lane = threadIdx.x & 31;
  T prefix = Op::identity();
  for (int64_t top = tile - 1;; top -= 32) {
    const int64_t tq = top - lane;
    unsigned f = tq >= 0 ? poll_flag(&flags[tq]) : 2u;  // before tile 0: an empty inclusive prefix
    for (unsigned it = 0; __any_sync(0xffffffffu, f == 0u); ++it) {
      if (f == 0u) {
        if (it >= kSpinLimit) {
          atomicOr(&ctrl->status, kStTimeout);
          f = 2u;  // give up: publish below so successors finish
        } else {
          __nanosleep(32);
          f = poll_flag(&flags[tq]);
        }
      }
    }
    const unsigned inc = __ballot_sync(0xffffffffu, f == 2u);
    const int stop = inc ? __ffs(inc) - 1 : 31;  // nearest lane holding an inclusive prefix
    __threadfence();
    T v = Op::identity();
    if (lane <= stop && tq >= 0) v = load_cg(f == 2u ? &inc_v[tq] : &agg_v[tq]);
#pragma unroll
    for (int d = 16; d; d >>= 1) v = op(v, shfl_xor(v, d));
    prefix = op(v, prefix);
    if (inc) return prefix;
  }
}

template <typename T, typename Op, bool kReverse, typename TIn = T>
__global__ void __launch_bounds__(kScanThreads) scan_onepass_kernel(const TIn* in, T* out, ScanLen L, bool exclusive,
                                                                     const T* base, T* total,
                                                                     bool write_total_at_len, ScanState st) {
  __shared__ T warp_sums[kScanThreads / 32];
  __shared__ T last_of_warp[kScanThreads / 32];
  __shared__ unsigned s_tile;
  __shared__ T s_prefix;
  __shared__ bool s_last;
  Op op;
  // Aggregates and inclusive prefixes live in separate arrays: each entry is
  // written once, before its flag, so a reader never sees one replaced by
  // the other.
  T* agg_v = static_cast<T*>(st.values);
  T* inc_v = agg_v + st.max_tiles;
  const int64_t len = L.get();
  const int64_t tiles = (len + kScanTile - 1) / kScanTile;
  if (threadIdx.x == 0) s_tile = atomicAdd(&st.counters[0], 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile < tiles) {
    const int64_t b0 = tile * kScanTile;
    T vals[kScanIPT];
    T acc = Op::identity();
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
      const int64_t e = b0 + static_cast<int64_t>(threadIdx.x) * kScanIPT + k;
      vals[k] = e < len ? static_cast<T>(in[scan_index<kReverse>(e, len)]) : Op::identity();
      acc = op(acc, vals[k]);
    }
    T inc = acc;
    const T agg = block_inclusive_scan<T, Op>(inc, warp_sums);
    if (threadIdx.x < 32) {
      T prefix = Op::identity();
      if (tile == 0) {
        if (base) prefix = *base;
      } else {
        if (threadIdx.x == 0) {
          agg_v[tile] = agg;
          __threadfence();
          atomicExch(&st.flags[tile], 1u);
        }
        if (st.test_stuck_polls && tile == 1 && threadIdx.x == 0) test_stuck_wait(st.ctrl, st.test_stuck_polls);
        __syncwarp();
        prefix = warp_look_back<T, Op>(tile, st.flags, agg_v, inc_v, st.ctrl);
      }
      if (threadIdx.x == 0) {
        inc_v[tile] = op(prefix, agg);
        __threadfence();
        atomicExch(&st.flags[tile], 2u);
        s_prefix = prefix;
      }
    }
    T prev = shfl_up(inc, 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) last_of_warp[warp] = inc;
    __syncthreads();
    if (lane == 0) prev = warp > 0 ? last_of_warp[warp - 1] : Op::identity();
    T run = op(s_prefix, prev);
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
      const int64_t e = b0 + static_cast<int64_t>(threadIdx.x) * kScanIPT + k;
      const T next = op(run, vals[k]);
      if (e < len) out[scan_index<kReverse>(e, len)] = exclusive ? run : next;
      if (e == len - 1) {
        if (write_total_at_len) out[len] = next;
        if (total) *total = next;
      }
      run = next;
    }
  } else if (tile == 0 && threadIdx.x == 0) {  // empty input
    const T v = base ? *base : Op::identity();
    if (write_total_at_len) out[0] = v;
    if (total) *total = v;
  }
  // the last block to finish resets the tile states
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&st.counters[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) st.flags[t] = 0u;
    if (threadIdx.x == 0) {
      st.counters[0] = 0u;
      st.counters[1] = 0u;
    }
  }
}

// One launch; `st` must hold ceil(host_len / kScanTile) flags and values and
// start cleared (it is left cleared).
template <typename T, typename Op, bool kReverse = false, typename TIn = T>
cudaError_t device_scan_1p(const TIn* in, T* out, ScanLen L, bool exclusive, const T* base, T* total,
                           bool write_total_at_len, const ScanState& st, cudaStream_t s) {
  const unsigned tiles = grid_for(L.host_len, kScanTile);
  scan_onepass_kernel<T, Op, kReverse, TIn><<<tiles, kScanThreads, 0, s>>>(in, out, L, exclusive, base, total,
                                                                       write_total_at_len, st);
  note_launches(1);
  return cudaGetLastError();
}

// Single pass for short inputs (launch count dominates), three kernels for
// long ones (when every tile starts at once, look-backs would walk back over
// many tiles).  `st.values` doubles as the three-kernel form's partials.
constexpr int64_t kOnePassMaxTiles = 1024;

// TIn: the input's element type when it differs from the sum's (int32 counts
// scanned into int64 offsets); such a scan cannot run in place.
template <typename T, typename Op, bool kReverse = false, typename TIn = T>
cudaError_t scan_any(const TIn* in, T* out, ScanLen L, bool exclusive, const T* base, T* total, bool write_total_at_len,
                     const ScanState& st, cudaStream_t s) {
  if ((L.host_len + kScanTile - 1) / kScanTile <= kOnePassMaxTiles)
    return device_scan_1p<T, Op, kReverse, TIn>(in, out, L, exclusive, base, total, write_total_at_len, st, s);
  return device_scan<T, Op, kReverse, TIn>(in, out, L, exclusive, base, total, write_total_at_len,
                                      static_cast<T*>(st.values), s);
}

}  // namespace mh
