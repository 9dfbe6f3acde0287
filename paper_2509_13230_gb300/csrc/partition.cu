// Proposal-bound preparation and the row-segment table.
//
// Bound (Sec. 2.5, Eq. 5): the UECM walk proposes with
//   phat_ij = A / (1 - c + A),   c >= r_ij = y_i y_j over the candidates proposed.
// The paper takes c = exp(-beta_min), the product of the two largest y among
// nodes not yet processed; the default here is c = y_i * max_{j >= a} y_j for
// the segment starting at rank a, which also bounds every r_ij ahead.  Both
// need suffix maxima of y in rank order (exact, order-free operators).
//
// Segments: row i's candidates [i+1, n) (bipartite: all candidates [0, n) of
// the other set, Sec. 2.6) are cut into pieces [a, b) of about
// T expected proposals.  A walk restarted at every piece head with q = p at
// the head is exact because q only has to bound p on the candidates it
// proposes, and p is non-increasing along the sorted order (Sec. 2.3).  The
// cost of candidate j is min(1, w_i v_j) with v = x (UBCM) or v = x*y (UECM),
// w_i = v_i (UBCM) or v_i / (1 - c_row) (UECM); cumulative costs use integer
// prefix sums and an exact 64x64 -> 128-bit product, so cut points are
// reproducible and strictly increasing for T >= 2.
#include "mh_internal.cuh"
#include "scan.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

// Bound of row i over all its candidates (from row_start on).
__device__ __forceinline__ double row_c(const Net& g, int64_t i) {
  if (g.flags & MH_BOUND_PAPER) return g.top[i].a * g.top[i].b;
  return g.ys_r[i] * g.top[row_start(g, i)].a;
}

__device__ __forceinline__ double row_weight(const Net& g, int64_t i) {
  if (g.model == MH_UBCM) return g.xs_r[i];
  return g.as_r[i] / (1.0 - row_c(g, i));
}

__device__ __forceinline__ unsigned long long weight_fixed(double w) {
  const double wq = ldexp(w, 40);
  if (!(wq < 0x1p64)) return ~0ull;
  return static_cast<unsigned long long>(wq);
}

// First candidate j of row i with w v_j < 1, else n.
__device__ __forceinline__ int64_t unit_cut(const Net& g, int64_t i, double w) {
  const double* v = (g.model == MH_UBCM) ? g.xs : g.as;
  int64_t lo = row_start(g, i), hi = g.n;
  if (lo < hi && w * v[lo] < 1.0) return lo;  // the common case: no candidate costs a whole unit
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (w * v[mid] < 1.0)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

struct RowCost {
  int64_t start, J;  // first candidate of the row, unit cut
  unsigned long long qw;
  int F;
  // cumulative cost up to candidate b, given Qb = Q[b] and QJ = Q[J]
  __device__ __forceinline__ unsigned long long at(int64_t b, unsigned long long Qb, unsigned long long QJ) const {
    const int64_t units = (b < J ? b : J) - start;
    unsigned long long c = static_cast<unsigned long long>(units) << F;
    if (b > J) {
      const unsigned long long dq = Qb - QJ;
      const unsigned long long lo = qw * dq, hi = __umul64hi(qw, dq);
      c += (hi << 24) | (lo >> 40);
    }
    return c;
  }
  __device__ __forceinline__ unsigned long long operator()(const unsigned long long* Q, int64_t b) const {
    return at(b, b > J ? Q[b] : 0ull, b > J ? Q[J] : 0ull);
  }
};

__device__ __forceinline__ int proxy_F(const Net& g) {
  const double vmax = (g.model == MH_UBCM) ? g.xs[0] : g.as[0];
  return proxy_scale(vmax, g.n);
}

__device__ __forceinline__ RowCost make_row_cost(const Net& g, int64_t i, int F) {
  const double w = row_weight(g, i);
  RowCost rc;
  rc.start = row_start(g, i);
  rc.J = unit_cut(g, i, w);
  rc.qw = weight_fixed(w);
  rc.F = F;
  return rc;
}

// Segments of row i: max(1, floor(C(n) / 2^F) / T), 0 for a row without candidates.
__device__ __forceinline__ long long row_segments(const Net& g, int64_t i, int F) {
  if (row_start(g, i) >= g.n) return 0;
  const RowCost rc = make_row_cost(g, i, F);
  const unsigned long long total = rc(g.Q, g.n);
  const unsigned long long ns = (total >> F) / static_cast<unsigned long long>(g.seg_target);
  return ns < 1 ? 1 : static_cast<long long>(ns);
}

__global__ void __launch_bounds__(256) row_count_kernel(Net g) {
  const int F = proxy_F(g);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < g.rows;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    g.rowoff[i] = row_segments(g, i, F);
}


// Last row whose first table row is <= s, within [lo, hi].
__device__ __forceinline__ int64_t row_of(const Net& g, long long s, int64_t lo, int64_t hi) {
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (g.rowoff[mid] <= s)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Last row r in [lo, hi] with rowoff[r] <= s (rowoff[lo] <= s), by a whole
// warp: 32 evenly spaced probes per round narrow the range 32-fold, so three
// rounds of loads cover 20,000 rows.  Every lane returns the answer.
__device__ __forceinline__ int64_t row_of_warp(const Net& g, long long s, int64_t lo, int64_t hi) {
  const int lane = threadIdx.x & 31;
  while (hi > lo) {
    const int64_t step = (hi - lo) / 32 + 1;
    const int64_t p = lo + lane * step;
    const bool ok = p <= hi && g.rowoff[p] <= s;  // true for a prefix of the lanes (lane 0 always)
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    const int last = 31 - __clz(mask);
    lo += last * step;
    const int64_t top = lo + step - 1;
    if (top < hi) hi = top;
  }
  return lo;
}

// First b in [lo, n] with cost(b) >= target, where cost(n) >= target: a
// bisection over every stride-th entry of Q (sQ, in shared memory) and then
// over the stride between two of them in global memory.
__device__ __forceinline__ int64_t cut_search(const Net& g, const RowCost& rc, unsigned long long QJ,
                                              unsigned long long target, int64_t lo,
                                              const unsigned long long* sQ, int64_t stride, int64_t ms) {
  const int64_t n = g.n;
  int64_t hi = n;
  int64_t mlo = (lo + stride - 1) / stride, mhi = ms;  // sample indices inside [lo, n]
  while (mlo < mhi) {
    const int64_t mid = mlo + (mhi - mlo) / 2;
    if (rc.at(mid * stride, sQ[mid], QJ) >= target)
      mhi = mid;
    else
      mlo = mid + 1;
  }
  if (mlo <= ms && mlo * stride >= lo && rc.at(mlo * stride, sQ[mlo], QJ) >= target) {
    hi = mlo * stride;
    if ((mlo - 1) * stride + 1 > lo) lo = (mlo - 1) * stride + 1;
  } else if (ms * stride + 1 > lo) {
    lo = ms * stride + 1;
  }
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (rc.at(mid, g.Q[mid], QJ) >= target)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// One thread per table row: finds its row (a block's table rows belong to a
// few consecutive rows, whose range two warps find first), then, for rows of
// more than one segment, its cut points by cut_search.  A segment's start is
// the previous segment's end, taken from the neighbouring lane when it walks
// the same row.
constexpr int kFillSamples = 2048;

__global__ void __launch_bounds__(256) seg_fill_kernel(Net g, Ctrl* ctrl) {
  __shared__ int64_t s_lo, s_hi;
  __shared__ unsigned long long sQ[kFillSamples + 1];
  const long long S = ctrl->num_segments;
  if (blockIdx.x == 0 && threadIdx.x == 0 && S > g.max_segments) atomicOr(&ctrl->status, kStSegments);
  const long long lim = S < g.max_segments ? S : g.max_segments;
  const int F = proxy_F(g);
  const int64_t n = g.n;
  const int64_t stride = n / kFillSamples + 1;  // samples m * stride <= n for m <= ms
  const int64_t ms = n / stride;
  {
    constexpr int kUnroll = kFillSamples / 256 + 1;  // every sample load in flight at once
    unsigned long long v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t m = threadIdx.x + static_cast<int64_t>(u) * blockDim.x;
      if (m <= ms) v[u] = g.Q[m * stride];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t m = threadIdx.x + static_cast<int64_t>(u) * blockDim.x;
      if (m <= ms) sQ[m] = v[u];
    }
  }
  const int lane = threadIdx.x & 31;
  for (long long s0 = blockIdx.x * static_cast<long long>(blockDim.x); s0 < lim;
       s0 += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long s1 = (s0 + blockDim.x < lim ? s0 + blockDim.x : lim) - 1;
    __syncthreads();
    if (threadIdx.x < 32) {
      const int64_t r = row_of_warp(g, s0, 0, g.rows - 1);
      if (lane == 0) s_lo = r;
    } else if (threadIdx.x < 64) {
      const int64_t r = row_of_warp(g, s1, 0, g.rows - 1);
      if (lane == 0) s_hi = r;
    }
    __syncthreads();
    const long long s = s0 + threadIdx.x;
    const bool live = s <= s1;
    int64_t i = 0, a = 0, b = n;
    long long k = 0, nseg = 1;
    RowCost rc{};
    unsigned long long QJ = 0, Tc = 0;
    if (live) {
      i = row_of(g, s, s_lo, s_hi);
      k = s - g.rowoff[i];
      nseg = g.rowoff[i + 1] - g.rowoff[i];
      a = row_start(g, i);
      if (nseg > 1) {
        rc = make_row_cost(g, i, F);
        QJ = g.Q[rc.J];
        Tc = rc(g.Q, n) / static_cast<unsigned long long>(nseg);
        if (k + 1 < nseg) b = cut_search(g, rc, QJ, Tc * static_cast<unsigned long long>(k + 1), rc.start + 1, sQ,
                                         stride, ms);
      }
    }
    // the end of segment k - 1 of the same row is this segment's start
    const int64_t prev_b = __shfl_up_sync(0xffffffffu, b, 1);
    const int64_t prev_i = __shfl_up_sync(0xffffffffu, i, 1);
    if (live && k > 0) {
      if (lane > 0 && prev_i == i)
        a = prev_b;
      else
        a = cut_search(g, rc, QJ, Tc * static_cast<unsigned long long>(k), rc.start + 1, sQ, stride, ms);
    }
    if (!live) continue;
    g.seg[s] = make_int4(static_cast<int>(i), static_cast<int>(k), static_cast<int>(a), static_cast<int>(b));
    if (g.model == MH_UECM) {
      // exp(-beta_min) of this segment and the walk's FP32 / double-float forms
      const double c = (g.flags & MH_BOUND_PAPER) ? g.top[i].a * g.top[i].b : g.ys_r[i] * g.top[a].a;
      const double omc = 1.0 - c;
      const df2 inv = df_from_double(1.0 / omc);
      g.seg_c[s] = c;
      g.seg_cf[s] = make_float4(inv.hi, inv.lo, static_cast<float>(omc), 0.0f);
    }
  }
}

__global__ void export_table_kernel(const int4* __restrict__ seg, const Ctrl* ctrl, int64_t max_segments,
                                    int32_t* row, int32_t* k, int64_t* a, int64_t* b, int64_t cap) {
  long long S = ctrl->num_segments;
  if (S > max_segments) S = max_segments;
  if (S > cap) S = cap;
  for (long long s = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; s < S;
       s += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int4 e = seg[s];
    row[s] = e.x;
    k[s] = e.y;
    a[s] = e.z;
    b[s] = e.w;
  }
}

// Node-id order of a network's work items, for CSR waves: rowoff_node[u] =
// the first slot of node u's row (an exclusive scan over node ids of each
// row's segment count; rowoff_node[n] = S), seg_slot[sg] = the slot of
// segment-table row sg, and slot_ik[slot] = (row rank, segment index) of the
// row at that slot, which the emit reads in slot order.  A CSR wave numbers its items
// (sample, node id, segment), so the item scan gives every edge's CSR
// position at once: the index array lists rows by node id.
__global__ void node_seg_count_kernel(Net g, const Ctrl* ctrl, long long* __restrict__ rowoff_node) {
  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;  // a truncated table fails the batch; stay in bounds
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u <= g.rows;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    long long c = 0;
    if (u < g.rows) {
      const int64_t r = g.rank[u];
      long long lo = g.rowoff[r], hi = g.rowoff[r + 1];
      lo = lo < S ? lo : S;
      hi = hi < S ? hi : S;
      c = hi - lo;
    }
    rowoff_node[u] = c;
  }
}

__global__ void seg_slot_kernel(Net g, Ctrl* ctrl, const long long* __restrict__ rowoff_node,
                                int32_t* __restrict__ seg_slot, int2* __restrict__ slot_ik) {
  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;
  for (int64_t sg = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; sg < S;
       sg += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int4 e = g.seg[sg];
    const long long slot = rowoff_node[g.perm[e.x]] + e.y;
    if (slot < 0 || slot >= S) {  // cannot happen for a consistent table; never index with it
      atomicOr(&ctrl->status, kStInternal);
      continue;
    }
    seg_slot[sg] = static_cast<int32_t>(slot);
    slot_ik[slot] = make_int2(e.x, e.y);
  }
}

}  // namespace

cudaError_t launch_bounds_and_partition(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  const ScanState st{reinterpret_cast<unsigned*>(ws + L.scan_flags), ws + L.scan_values,
                     reinterpret_cast<unsigned*>(ws + L.scan_counters), ctrl, L.scan_tiles,
                     (g.flags & MH_TEST_WAIT_TIMEOUT) ? kTestStuckPolls : 0u};
  cudaError_t e;
  // Q = exclusive prefix of the fixed-point costs, Q[n] = total.
  e = scan_any<unsigned long long, SumOp<unsigned long long>>(g.Q, g.Q, ScanLen{g.n, nullptr, 1}, true,
                                                                    nullptr, nullptr, true, st, s);
  if (e != cudaSuccess) return e;
  if (g.model == MH_UECM && !merge_sorted(g.n)) {
    // top[i] = two largest y among ranks >= i; top[i].a is the suffix maximum
    // (the tile sorts + merge of small node sets leave it already)
    e = scan_any<Top2, Top2Op, true>(g.top, g.top, ScanLen{g.n, nullptr, 1}, false, nullptr, nullptr, false,
                                           st, s);
    if (e != cudaSuccess) return e;
  }
  // one thread per row (a scan tile computing its 2048 rows itself is
  // latency-bound), then the row offsets
  const unsigned blocks = grid_for(g.rows + 1, 256, static_cast<unsigned>(sm_count()) * 8u);
  row_count_kernel<<<blocks, 256, 0, s>>>(g);
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_any<long long, SumOp<long long>>(g.rowoff, g.rowoff, ScanLen{g.rows, nullptr, 1}, true, nullptr,
                                                  &ctrl->num_segments, true, st, s);
  if (e != cudaSuccess) return e;
  const unsigned fill_blocks = grid_for(g.max_segments, 256, static_cast<unsigned>(sm_count()) * 16u);
  seg_fill_kernel<<<fill_blocks, 256, 0, s>>>(g, ctrl);
  note_launches(1);
  return cudaGetLastError();
}

namespace {
// Directed networks (Sec. 2.6): row i (the out-copy of node perm_r[i]) never
// proposes its own in-copy, the candidate of rank rank[perm_r[i]].
__global__ void exclusions_kernel(Net g) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < g.rows;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    g.excl[i] = g.rank[g.perm_r[i]];
}
}  // namespace

cudaError_t launch_exclusions(const Net& g, cudaStream_t s) {
  exclusions_kernel<<<grid_for(g.rows, 256, static_cast<unsigned>(sm_count()) * 4u), 256, 0, s>>>(g);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_export_table(const Net& g, const Ctrl* ctrl, int32_t* row, int32_t* k, int64_t* a, int64_t* b,
                                int64_t cap, cudaStream_t s) {
  const unsigned blocks = grid_for(g.max_segments, 256, static_cast<unsigned>(sm_count()) * 8u);
  export_table_kernel<<<blocks, 256, 0, s>>>(g.seg, ctrl, g.max_segments, row, k, a, b, cap);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_node_order(const Net& g, Ctrl* ctrl, long long* rowoff_node, int32_t* seg_slot, int2* slot_ik,
                              const ScanState& st, cudaStream_t s) {
  const unsigned sms = static_cast<unsigned>(sm_count());
  node_seg_count_kernel<<<grid_for(g.rows + 1, 256, sms * 4u), 256, 0, s>>>(g, ctrl, rowoff_node);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_any<long long, SumOp<long long>>(rowoff_node, rowoff_node, ScanLen{g.rows + 1, nullptr, 1}, true, nullptr,
                                            nullptr, false, st, s);
  if (e != cudaSuccess) return e;
  seg_slot_kernel<<<grid_for(g.max_segments, 256, sms * 4u), 256, 0, s>>>(g, ctrl, rowoff_node, seg_slot, slot_ik);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh
