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
  __device__ __forceinline__ unsigned long long operator()(const unsigned long long* Q, int64_t b) const {
    const int64_t units = (b < J ? b : J) - start;
    unsigned long long c = static_cast<unsigned long long>(units) << F;
    if (b > J) {
      const unsigned long long dq = Q[b] - Q[J];
      const unsigned long long lo = qw * dq, hi = __umul64hi(qw, dq);
      c += (hi << 24) | (lo >> 40);
    }
    return c;
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

__global__ void __launch_bounds__(256) row_count_kernel(Net g) {
  const int F = proxy_F(g);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < g.rows;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    long long nseg = 0;
    if (row_start(g, i) < g.n) {
      const RowCost rc = make_row_cost(g, i, F);
      const unsigned long long total = rc(g.Q, g.n);
      unsigned long long ns = (total >> F) / static_cast<unsigned long long>(g.seg_target);
      nseg = ns < 1 ? 1 : static_cast<long long>(ns);
    }
    g.rowoff[i] = nseg;
  }
}

// One thread per table row: finds its row by bisection of rowoff, then its
// two cut points by bisection of the cumulative cost.
__global__ void __launch_bounds__(256) seg_fill_kernel(Net g, Ctrl* ctrl) {
  const long long S = ctrl->num_segments;
  if (blockIdx.x == 0 && threadIdx.x == 0 && S > g.max_segments) atomicOr(&ctrl->status, kStSegments);
  const long long lim = S < g.max_segments ? S : g.max_segments;
  const int F = proxy_F(g);
  for (long long s = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; s < lim;
       s += static_cast<long long>(gridDim.x) * blockDim.x) {
    int64_t lo = 0, hi = g.rows - 1;  // last row with rowoff[row] <= s
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo + 1) / 2;
      if (g.rowoff[mid] <= s)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int64_t i = lo;
    const long long k = s - g.rowoff[i];
    const long long nseg = g.rowoff[i + 1] - g.rowoff[i];
    const RowCost rc = make_row_cost(g, i, F);
    const unsigned long long total = rc(g.Q, g.n);
    const unsigned long long Tc = total / static_cast<unsigned long long>(nseg);
    auto cut = [&](long long kk) -> int64_t {  // first b in [start+1, n] with cost(b) >= kk * Tc
      const unsigned long long target = Tc * static_cast<unsigned long long>(kk);
      int64_t a = rc.start + 1, b = g.n;
      while (a < b) {
        const int64_t mid = a + (b - a) / 2;
        if (rc(g.Q, mid) >= target)
          b = mid;
        else
          a = mid + 1;
      }
      return a;
    };
    const int64_t a = (k == 0) ? rc.start : cut(k);
    const int64_t b = (k + 1 == nseg) ? g.n : cut(k + 1);
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

}  // namespace

cudaError_t launch_bounds_and_partition(const Net& g, const Layout& L, char* ws, Ctrl* ctrl, cudaStream_t s) {
  const ScanState st{reinterpret_cast<unsigned*>(ws + L.scan_flags), ws + L.scan_values,
                     reinterpret_cast<unsigned*>(ws + L.scan_counters), ctrl, L.scan_tiles};
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

}  // namespace mh
