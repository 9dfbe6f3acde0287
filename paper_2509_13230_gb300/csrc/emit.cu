// Edge output: canonical order, COO and CSR layouts, UECM weights.
//
// After the walk every work item (sample, segment) has an edge count and a
// contiguous run of accepted ranks j in the staging buffer.  An exclusive
// scan of the counts in item order gives each item's place in the output, so
// a sample's edges come out in (row rank, segment, candidate) order no matter
// which lane walked which segment.  The emit pass maps ranks to original ids
// (perm), draws the UECM weight of each edge (Eq. 4), and writes:
//   COO  src[e] = perm[i], dst[e] = perm[j], w[e]
//   CSR  csr_idx[off[s(n+1) + perm[i]] + position within row i] = perm[j]
// CSR rows are original node ids; row u holds the edges whose higher-ranked
// endpoint is u (bipartite: whose + endpoint is u), and offsets are
// positions in the concatenated index array.
#include "mh_internal.cuh"
#include "scan.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

// csr_off[(chunk_first + s)(rows+1) + u] = edges of row u in sample s (0 for
// u = rows); an in-place exclusive scan then turns counts into offsets.
__global__ void csr_count_kernel(Net g, const long long* __restrict__ item_off, const Ctrl* ctrl,
                                 int64_t chunk_first, int64_t chunk_samples, long long* csr_off) {
  // A segment table that outgrew max_segments was truncated: rowoff still
  // holds the full prefix, which would index past item_off.  The call fails
  // with MH_ERR_WORKSPACE, so nothing is counted.
  if (ctrl->num_segments > g.max_segments) return;
  const long long S = ctrl->num_segments;
  const int64_t n1 = g.rows + 1;
  const int64_t total = chunk_samples * n1;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t s = t / n1, u = t - s * n1;
    long long c = 0;
    if (u < g.rows) {
      const int64_t i = g.rank_r[u];
      c = item_off[s * S + g.rowoff[i + 1]] - item_off[s * S + g.rowoff[i]];
    }
    csr_off[chunk_first * n1 + t] = c;
  }
}

struct EmitParams {
  Net g;
  ChunkArgs c;
  Outputs o;
  Ctrl* ctrl;
};

// Each block owns kEmitItems consecutive work items and writes their output
// range with consecutive threads on consecutive edges.
__global__ void __launch_bounds__(256) emit_kernel(EmitParams P) {
  const Net& g = P.g;
  Ctrl* ctrl = P.ctrl;
  __shared__ LnEntry tab[kLnTable];
  if (g.model == MH_UECM) {
    ln_table_to_shared(tab, g.lntab);
    __syncthreads();
  }
  const bool fp64_only = (g.flags & MH_FP64_ONLY) != 0;
  unsigned long long fallbacks = 0;
  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;
  const long long items = S * P.c.chunk_samples;
  if (blockIdx.x == 0) {
    // per-sample edge counts of this chunk; the next chunk continues after it
    for (int64_t s = threadIdx.x; s < P.c.chunk_samples; s += blockDim.x)
      P.c.sample_counts[P.c.chunk_first + s] = P.c.item_off[(s + 1) * S] - P.c.item_off[s * S];
    if (threadIdx.x == 0) ctrl->out_base = ctrl->out_end;
  }
  const long long it0 = static_cast<long long>(blockIdx.x) * kEmitItems;
  if (it0 >= items || ctrl->num_segments > g.max_segments) return;  // truncated table: the call fails
  // Staging that did not fit was never written: emit nothing (the call
  // reports MH_ERR_CAPACITY with exact counts).
  if (ctrl->stage_used > static_cast<unsigned long long>(P.c.staging_cap)) return;
  const long long it1 = it0 + kEmitItems < items ? it0 + kEmitItems : items;
  __shared__ long long off[kEmitItems + 1];
  for (long long t = threadIdx.x; t <= it1 - it0; t += blockDim.x) off[t] = P.c.item_off[it0 + t];
  __syncthreads();
  const long long o0 = off[0], o1 = off[it1 - it0];
  const long long n1 = g.rows + 1;
  bool overflow = false;
  for (long long pos = o0 + threadIdx.x; pos < o1; pos += blockDim.x) {
    int lo = 0, hi = static_cast<int>(it1 - it0) - 1;  // last local item with off <= pos
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= pos)
        lo = mid;
      else
        hi = mid - 1;
    }
    const long long item = it0 + lo;
    const long long e = pos - off[lo];
    if (e >= P.c.item_cnt[item]) {  // offsets inconsistent with the counts: never read past a run
      atomicOr(&ctrl->status, kStInternal);
      continue;
    }
    const long long s_local = static_cast<unsigned>(item) / static_cast<unsigned>(S);  // items < 2^31
    const long long seg = item - s_local * S;
    const int4 sg = g.seg[seg];
    const int32_t i = sg.x;
    const int32_t j = P.c.staging[P.c.item_base[item] + e];
    if (j < row_start(g, i) || j >= g.n || (g.excl && j == g.excl[i])) {
      // cannot happen for a walked segment; never index with it
      atomicOr(&ctrl->status, kStInternal);
      continue;
    }
    const int32_t u = g.perm_r[i], v = g.perm[j];
    int32_t wt = 1;
    if (g.model == MH_UECM) {
      const float2 li = g.lny_r[i], lj = g.lny[j];
      wt = draw_weight(static_cast<uint32_t>(e), static_cast<uint32_t>(sg.y), static_cast<uint32_t>(i),
                       P.c.sample0 + static_cast<uint32_t>(s_local), P.c.key0, P.c.key1, g.ys_r[i], g.ys[j],
                       df2{li.x, li.y}, df2{lj.x, lj.y}, tab, fp64_only, overflow, fallbacks);
    }
    if (pos < P.o.capacity) {
      if (P.o.src) {
        P.o.src[pos] = u;
        P.o.dst[pos] = v;
        if (P.o.w) P.o.w[pos] = wt;
      }
      if (P.o.csr_idx) {
        const long long s_all = P.c.chunk_first + s_local;
        const long long row_first = s_local * S + g.rowoff[i];
        const long long at = P.o.csr_off[s_all * n1 + u] + (P.c.item_off[item] - P.c.item_off[row_first]) + e;
        if (at < P.o.capacity) {
          P.o.csr_idx[at] = v;
          if (P.o.csr_w) P.o.csr_w[at] = wt;
        }
      }
    }
  }
  if (overflow) atomicOr(&ctrl->status, kStOverflow);
  (void)fallbacks;
}

}  // namespace

cudaError_t launch_emit(const Net& g, const ChunkArgs& c, const Outputs& o, Ctrl* ctrl, cudaStream_t s) {
  const ScanState& st = *static_cast<const ScanState*>(c.scan_state);
  cudaError_t e;
  // item offsets (continuing from the edges of earlier chunks)
  e = scan_any<long long, SumOp<long long>>(c.item_cnt, c.item_off,
                                                  ScanLen{c.items_max, &ctrl->num_segments, c.chunk_samples}, true,
                                                  &ctrl->out_base, &ctrl->out_end, true, st, s);
  if (e != cudaSuccess) return e;
  if (o.csr_off) {
    const int64_t len = c.chunk_samples * (g.rows + 1);
    csr_count_kernel<<<grid_for(len, 256, static_cast<unsigned>(sm_count()) * 8u), 256, 0, s>>>(
        g, c.item_off, ctrl, c.chunk_first, c.chunk_samples, o.csr_off);
    note_launches(1);
    long long* region = o.csr_off + c.chunk_first * (g.rows + 1);
    e = scan_any<long long, SumOp<long long>>(region, region, ScanLen{len, nullptr, 1}, true, &ctrl->out_base,
                                                    nullptr, false, st, s);
    if (e != cudaSuccess) return e;
  }
  EmitParams P{g, c, o, ctrl};
  emit_kernel<<<grid_for(c.items_max, kEmitItems), 256, 0, s>>>(P);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh
