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
// positions in the concatenated index array.  The symmetric layout
// (MH_CSR_SYMMETRIC) lists every edge in both endpoint rows: see
// launch_emit for its passes.
#include "mh_internal.cuh"
#include "scan.cuh"
#include "walk_math.cuh"

namespace mh {

#define MH_CUDA_RET(expr)                     \
  do {                                        \
    const cudaError_t e_ = (expr);            \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

namespace {

// csr_off[(chunk_first + s)(rows+1) + u] = edges of row u in sample s (0 for
// u = rows); an in-place exclusive scan then turns counts into offsets.
// With `rev` (symmetric layout) the count adds the edges arriving at u.
__global__ void csr_count_kernel(Net g, const long long* __restrict__ item_off, const Ctrl* ctrl,
                                 int64_t chunk_first, int64_t chunk_samples, long long* csr_off,
                                 const long long* __restrict__ rev) {
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
      if (rev) c += rev[s * n1 + i];
    }
    csr_off[chunk_first * n1 + t] = c;
  }
}

// CSR offsets of a node-order chunk: entry (sample, u) is the item offset of
// node u's first slot (u = rows: the sample's end), positions that already
// continue from earlier chunks.
__global__ void csr_off_node_kernel(Net g, const long long* __restrict__ item_off,
                                    const long long* __restrict__ rowoff_node, const Ctrl* ctrl, int64_t chunk_first,
                                    int64_t chunk_samples, long long* __restrict__ csr_off) {
  if (ctrl->num_segments > g.max_segments) return;  // a truncated table fails the call
  const long long S = ctrl->num_segments;
  const int64_t n1 = g.rows + 1;
  const int64_t total = chunk_samples * n1;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t s = t / n1, u = t - s * n1;
    csr_off[chunk_first * n1 + t] = item_off[s * S + rowoff_node[u]];
  }
}

// Emit modes.  kEmitPlain writes COO and the one-row CSR.  The symmetric
// layout takes two passes: kEmitSymPairs writes COO, the (sample, rank of
// the lower endpoint) key and position of every edge for the key sort, the
// edge's source and weight by position, and counts the edges arriving at
// each rank; kEmitSymForward writes every edge into its higher-ranked
// endpoint's row, after the row's arriving edges.
enum EmitMode { kEmitPlain = 0, kEmitSymPairs = 1, kEmitSymForward = 2 };

struct EmitParams {
  Net g;
  ChunkArgs c;
  Outputs o;
  Ctrl* ctrl;
  int mode;
};

// What every edge of a work item shares, set up once per item by one thread.
struct ItemRec {
  long long base;    // staging position of the item's first rank
  long long at;      // CSR: index position of the item's first edge (one-row or symmetric forward)
  int cnt;           // edges of the item
  int i;             // row rank
  int u;             // original id of row i's node
  int k;             // segment index within the row
  int s_local;       // sample within the chunk
  int ex;            // directed: the excluded candidate rank, else -1
  float2 lnyi;
  double yi;
};

// Warps take groups of kEmitGroup consecutive work items of the chunk (a
// grid-stride loop): lane l sets up item l's ItemRec in the warp's shared
// slice, then the group's edges are written 32 at a time, lane l taking
// edge (pass * 32 + l) of the group.  Its item is the last lane whose
// first-edge offset (relative to the group) is at most that index, found by
// a five-step search over the offsets the lanes hold; empty items share
// their offset with the next item and are never selected.  Warps move on
// independently (no block-wide barrier after the logarithm table).
__global__ void __launch_bounds__(kEmitWarps * 32) emit_kernel(EmitParams P) {
  const Net& g = P.g;
  Ctrl* ctrl = P.ctrl;
  __shared__ LnEntry tab[kLnTable];
  __shared__ ItemRec info_all[kEmitWarps][kEmitGroup];
  const bool uecm = g.model == MH_UECM;
  if (uecm && P.mode != kEmitSymForward) ln_table_to_shared(tab, g.lntab);
  const bool fp64_only = (g.flags & MH_FP64_ONLY) != 0;
  unsigned long long fallbacks = 0, boundary = 0;  // weight draws left to FP64; boundary draws
  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;
  const long long items = S * P.c.chunk_samples;
  const bool unwritten = ctrl->num_segments > g.max_segments ||  // truncated table: the call fails
                         ctrl->stage_used > static_cast<unsigned long long>(P.c.staging_cap);
  const long long chunk_first_edge = P.c.item_off[0];
  if (blockIdx.x == 0 && P.mode != kEmitSymForward) {
    // per-sample edge counts of this chunk; the next chunk continues after it
    for (int64_t s = threadIdx.x; s < P.c.chunk_samples; s += blockDim.x)
      P.c.sample_counts[P.c.chunk_first + s] = P.c.item_off[(s + 1) * S] - P.c.item_off[s * S];
    if (threadIdx.x == 0) {
      ctrl->out_base = ctrl->out_end;
      if (P.mode == kEmitSymPairs) {
        // the chunk's edges that have a place in the output (none when the
        // walk's output was not kept), and where its CSR entries start
        long long len = P.c.item_off[items] - chunk_first_edge;
        const long long room = P.o.capacity - chunk_first_edge;
        if (len > room) len = room;
        ctrl->sym_len = (unwritten || len < 0) ? 0 : len;
        ctrl->sym_base = 2 * chunk_first_edge;
      }
    }
  }
  // Staging that did not fit was never written: emit nothing (the call
  // reports MH_ERR_CAPACITY with exact counts).
  if (unwritten) return;
  __syncthreads();  // the logarithm table
  const long long n1 = g.rows + 1;
  const bool one_row_csr = P.mode == kEmitPlain && P.o.csr_idx != nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ItemRec* info = info_all[warp];
  bool overflow = false, bad = false;
  const long long stride = static_cast<long long>(gridDim.x) * kEmitWarps * kEmitGroup;
  for (long long g0 = (static_cast<long long>(blockIdx.x) * kEmitWarps + warp) * kEmitGroup; g0 < items;
       g0 += stride) {
    const long long item = g0 + lane;
    const bool in = item < items;
    // the group's edges are [item_off[g0], item_off[g0 + 32]) (item_off holds items + 1 entries)
    const long long off_l = P.c.item_off[in ? item : items];
    const long long first = __shfl_sync(0xffffffffu, off_l, 0);
    const long long last = lane == 31 ? P.c.item_off[in ? item + 1 : items] : 0;
    const long long total = __shfl_sync(0xffffffffu, last, 31) - first;
    if (total == 0) continue;  // a group of empty items (common in sparse rows)
    if (total >= (1ll << 31)) {  // cannot happen: a group's edges fit the staging, well below 2^31
      bad = true;
      continue;
    }
    const unsigned rel = static_cast<unsigned>(off_l - first);
    const int my_cnt = in ? static_cast<int>(P.c.item_cnt[item]) : 0;
    if (my_cnt > 0) {
      const int s_local = static_cast<int>(static_cast<unsigned>(item) / static_cast<unsigned>(S));  // items < 2^31
      const long long seg = item - static_cast<long long>(s_local) * S;  // the slot, in node order
      int2 ik;
      if (P.c.slot_ik) {
        ik = P.c.slot_ik[seg];  // read in slot order
      } else {
        const int4 sg = g.seg[seg];
        ik = make_int2(sg.x, sg.y);
      }
      ItemRec r;
      r.base = P.c.item_base[item];
      r.cnt = my_cnt;
      r.i = ik.x;
      r.u = P.c.slot_ik ? 0 : g.perm_r[ik.x];  // the row's id, for COO and rank-order CSR only
      r.k = ik.y;
      r.s_local = s_local;
      r.ex = g.excl ? g.excl[ik.x] : -1;
      r.at = 0;
      if (one_row_csr && P.c.slot_ik) {
        r.at = off_l;  // node order: the item offset is the CSR position
      } else if (one_row_csr || P.mode == kEmitSymForward) {
        const long long s_all = P.c.chunk_first + s_local;
        const long long row_first = static_cast<long long>(s_local) * S + g.rowoff[ik.x];
        r.at = P.o.csr_off[s_all * n1 + r.u] + (off_l - P.c.item_off[row_first]);
        if (P.mode == kEmitSymForward) {  // after the row's arriving edges
          const long long* rv = P.c.sym.rev + static_cast<long long>(s_local) * n1;
          r.at += rv[ik.x + 1] - rv[ik.x];
        }
      }
      r.yi = 0.0;
      r.lnyi = make_float2(0.f, 0.f);
      if (uecm) {
        r.yi = g.ys_r[ik.x];
        r.lnyi = g.lny_r[ik.x];
      }
      info[lane] = r;
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
    int32_t j_n = 0;
    bool ok_n = locate(lane, l_n, e_n);
    if (ok_n) j_n = P.c.staging[info[l_n].base + e_n];
    for (unsigned p0 = 0; p0 < tot; p0 += 32) {
      const unsigned idx = p0 + lane;
      const int l = l_n, e = e_n;
      const int32_t j = j_n;
      const bool ok = ok_n;
      if (p0 + 32 < tot) {  // warp-uniform
        ok_n = locate(idx + 32, l_n, e_n);
        if (ok_n) j_n = P.c.staging[info[l_n].base + e_n];
      }
      if (!ok) continue;
      const ItemRec& r = info[l];
      if (j < row_start(g, r.i) || j >= g.n || j == r.ex) {  // cannot happen for a walked segment
        bad = true;
        continue;
      }
      const int32_t v = g.perm[j];
      const long long pos = first + idx;
      const long long q = pos - chunk_first_edge;  // position within the chunk
      if (P.mode == kEmitSymForward) {
        if (pos >= P.o.capacity) continue;
        const long long at = r.at + e;
        if (at >= 0 && at < 2 * P.o.capacity) {
          P.o.csr_idx[at] = v;
          if (P.o.csr_w) P.o.csr_w[at] = P.c.sym.w[q];
        }
        continue;
      }
      int32_t wt = 1;
      if (uecm) {
        const float2 lj = g.lny[j];
        wt = draw_weight(static_cast<uint32_t>(e), static_cast<uint32_t>(r.k), static_cast<uint32_t>(r.i),
                         P.c.sample0 + static_cast<uint32_t>(r.s_local), P.c.key0, P.c.key1, r.yi, &g.ys[j],
                         df2{r.lnyi.x, r.lnyi.y}, df2{lj.x, lj.y}, tab, fp64_only, overflow, fallbacks, boundary);
      }
      if (pos < P.o.capacity) {
        if (P.o.src) {
          P.o.src[pos] = r.u;
          P.o.dst[pos] = v;
          if (P.o.w) P.o.w[pos] = wt;
        }
        if (P.mode == kEmitSymPairs) {
          P.c.sym.keys[0][q] = (static_cast<unsigned long long>(r.s_local) << 32) | static_cast<uint32_t>(j);
          P.c.sym.vals[0][q] = static_cast<int32_t>(q);
          P.c.sym.src[q] = r.u;
          P.c.sym.w[q] = wt;
          atomicAdd(reinterpret_cast<unsigned long long*>(&P.c.sym.rev[static_cast<long long>(r.s_local) * n1 + j]),
                    1ull);
        } else if (one_row_csr) {
          const long long at = r.at + e;
          if (at < P.o.capacity) {
            P.o.csr_idx[at] = v;
            if (P.o.csr_w) P.o.csr_w[at] = wt;
          }
        }
      }
    }
    __syncwarp();  // the slice is rewritten by the next group
  }
  if (overflow) atomicOr(&ctrl->status, kStOverflow);
  if (bad) atomicOr(&ctrl->status, kStInternal);
  if (boundary) atomicAdd(&ctrl->stats[MH_STAT_BOUNDARY], boundary);
  (void)fallbacks;
}

// Symmetric layout, second half: the sorted keys list every edge by
// (sample, rank of its lower-ranked endpoint j), ties in output order, i.e.
// by the rank of the other endpoint.  Entry t goes to row perm[j] at
// position t - (first entry of its key), which the scan of the arriving
// counts gives.
__global__ void __launch_bounds__(256) sym_reverse_kernel(Net g, SymArgs sym, const unsigned long long* keys,
                                                          const int32_t* vals, const Ctrl* ctrl, int64_t chunk_first,
                                                          int64_t chunk_samples, Outputs o, Ctrl* status) {
  const long long len = ctrl->sym_len;
  const int64_t n1 = g.n + 1;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < len;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long key = keys[t];
    const long long s_local = static_cast<long long>(key >> 32);
    const int64_t j = static_cast<int64_t>(key & 0xFFFFFFFFull);
    const long long q = vals[t];
    if (s_local >= chunk_samples || j >= g.n || q < 0 || q >= len) {  // cannot happen: never index with it
      atomicOr(&status->status, kStInternal);
      continue;
    }
    const long long first = sym.rev[s_local * n1 + j];
    const long long at = o.csr_off[(chunk_first + s_local) * n1 + g.perm[j]] + (t - first);
    if (at >= 0 && at < 2 * o.capacity) {
      o.csr_idx[at] = sym.src[q];
      if (o.csr_w) o.csr_w[at] = sym.w[q];
    }
  }
}

}  // namespace

cudaError_t launch_emit(const Net& g, const ChunkArgs& c, const Outputs& o, Ctrl* ctrl, cudaStream_t s) {
  const ScanState& st = *static_cast<const ScanState*>(c.scan_state);
  cudaError_t e;
  // item offsets (continuing from the edges of earlier chunks)
  e = scan_any<long long, SumOp<long long>, false, int32_t>(c.item_cnt, c.item_off,
                                                  ScanLen{c.items_max, &ctrl->num_segments, c.chunk_samples}, true,
                                                  &ctrl->out_base, &ctrl->out_end, true, st, s);
  if (e != cudaSuccess) return e;
  const int64_t len = c.chunk_samples * (g.rows + 1);
  const unsigned emit_blocks = grid_for(c.items_max, kEmitWarps * kEmitGroup, static_cast<unsigned>(sm_count()) * 5u);
  long long* region = o.csr_off ? o.csr_off + c.chunk_first * (g.rows + 1) : nullptr;
  if (c.sym.rev && o.csr_off) {
    // symmetric layout: keys and arriving counts, the key sort, offsets from
    // both counts, then each edge into both of its rows
    MH_CUDA_RET(cudaMemsetAsync(c.sym.rev, 0, 8 * static_cast<size_t>(len), s));
    EmitParams P1{g, c, o, ctrl, kEmitSymPairs};
    emit_kernel<<<emit_blocks, kEmitWarps * 32, 0, s>>>(P1);
    note_launches(1);
    csr_count_kernel<<<grid_for(len, 256, static_cast<unsigned>(sm_count()) * 8u), 256, 0, s>>>(
        g, c.item_off, ctrl, c.chunk_first, c.chunk_samples, o.csr_off, c.sym.rev);
    note_launches(1);
    e = scan_any<long long, SumOp<long long>>(region, region, ScanLen{len, nullptr, 1}, true, &ctrl->sym_base,
                                                    nullptr, false, st, s);
    if (e != cudaSuccess) return e;
    e = scan_any<long long, SumOp<long long>>(c.sym.rev, c.sym.rev, ScanLen{len, nullptr, 1}, true, nullptr,
                                                    nullptr, false, st, s);
    if (e != cudaSuccess) return e;
    // digits of the rank (bytes 0..) and of the sample within the chunk (bytes 4..)
    int shifts[8], passes = 0;
    for (int b = 0; b < 4 && (b == 0 || ((g.n - 1) >> (8 * b)) != 0); ++b) shifts[passes++] = 8 * b;
    for (int b = 0; b < 4 && ((c.chunk_samples - 1) >> (8 * b)) != 0; ++b) shifts[passes++] = 32 + 8 * b;
    SymArgs sym = c.sym;
    int buf = 0;
    e = launch_pair_sort(sym.keys, sym.vals, o.capacity, &ctrl->sym_len, shifts, passes, sym.hist, &st, ctrl, &buf,
                         s);
    if (e != cudaSuccess) return e;
    EmitParams P2{g, c, o, ctrl, kEmitSymForward};
    emit_kernel<<<emit_blocks, kEmitWarps * 32, 0, s>>>(P2);
    note_launches(1);
    sym_reverse_kernel<<<grid_for(o.capacity, 256, static_cast<unsigned>(sm_count()) * 8u), 256, 0, s>>>(
        g, sym, sym.keys[buf], sym.vals[buf], ctrl, c.chunk_first, c.chunk_samples, o, ctrl);
    note_launches(1);
    return cudaGetLastError();
  }
  if (o.csr_off && c.rowoff_node) {
    csr_off_node_kernel<<<grid_for(len, 256, static_cast<unsigned>(sm_count()) * 8u), 256, 0, s>>>(
        g, c.item_off, c.rowoff_node, ctrl, c.chunk_first, c.chunk_samples, o.csr_off);
    note_launches(1);
    MH_CUDA_RET(cudaGetLastError());
  } else if (o.csr_off) {
    csr_count_kernel<<<grid_for(len, 256, static_cast<unsigned>(sm_count()) * 8u), 256, 0, s>>>(
        g, c.item_off, ctrl, c.chunk_first, c.chunk_samples, o.csr_off, nullptr);
    note_launches(1);
    e = scan_any<long long, SumOp<long long>>(region, region, ScanLen{len, nullptr, 1}, true, &ctrl->out_base,
                                                    nullptr, false, st, s);
    if (e != cudaSuccess) return e;
  }
  EmitParams P{g, c, o, ctrl, kEmitPlain};
  emit_kernel<<<emit_blocks, kEmitWarps * 32, 0, s>>>(P);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh
