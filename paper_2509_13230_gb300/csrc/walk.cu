// Miller-Hagberg proposal walk (Sec. 2.3; Sec. 2.4 steps (ii)-(iv);
// Algorithm 1), one lane per (sample, row segment) work item.
//
// Per candidate, with q the current proposal probability:
//   L = 1 + floor(t),  t = ln U / ln(1 - q),  U uniform on (0, 1]
//       (geometric skip, P(L) = q (1-q)^(L-1), Fig. 2)
//   j = pos + L; the segment ends when j >= b, i.e. when t >= b - pos - 1
//   keep j when V < p_ij / q, V uniform on [0, 1)
//   q <- p_ij (UBCM, step (iii)) or phat_ij (UECM, Algorithm 1)
// Random words: Philox4x32-10 of counter {d, k, i, s} (draw d of segment k of
// row i in sample s); U from words (1,0), V from words (3,2).
//
// Decision arithmetic (walk_math.cuh).  The skip needs floor(t) exactly and
// the acceptance test compares V with p/q; both use FP64 values computed in
// one fixed order, so they match the serial definition bit for bit except for
// draws within a few ulp of an integer boundary of t.
//
// Scheduling.  Warps take chunks of work items from a global ticket; an idle
// lane takes the chunk's next item, so lanes stay busy when segment lengths
// differ.  A lane buffers accepted ranks j in its shared-memory slot; when
// its segment ends, the warp reserves staging space with one atomic and
// copies the slot out with coalesced stores.  A segment with more than kSlot
// edges is re-walked by a second kernel that writes straight to staging.
#include "mh_internal.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

struct WalkParams {
  Net g;
  ChunkArgs c;
  Ctrl* ctrl;
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// One segment's walk state.
struct SegWalker {
  int32_t i, k, b, pos;
  uint32_t sample, d, cnt;
  double q;       // current proposal probability (FP64 value of p or phat)
  double xi;      // x_i (UBCM) or a_i = x_i y_i (UECM)
  double yi;      // y_i (UECM)
  double c;       // UECM bound constant exp(-beta_min)
  bool uecm;

  __device__ __forceinline__ void init(const Net& g, long long item, long long S, uint32_t sample0) {
    const long long s_local = item / S;
    const long long seg = item - s_local * S;
    const int4 e = g.seg[seg];
    i = e.x;
    k = e.y;
    const int32_t a = e.z;
    b = e.w;
    pos = a - 1;
    sample = sample0 + static_cast<uint32_t>(s_local);
    d = 0;
    cnt = 0;
    uecm = (g.model == MH_UECM);
    const int32_t head = (g.flags & MH_INIT_PREV) ? a - 1 : a;
    if (!uecm) {
      xi = g.xs[i];
      q = prob_ubcm(xi, g.xs[head]);
    } else {
      xi = g.as[i];
      yi = g.ys[i];
      c = (g.flags & MH_BOUND_PAPER) ? g.top[i].a * g.top[i].b : yi * g.ymax[a];
      q = prob_hat(xi, g.as[head], c);
    }
  }

  // One candidate.  Returns false when the segment has ended; otherwise sets
  // `accepted` and `j`.
  __device__ __forceinline__ bool step(const Net& g, uint32_t key0, uint32_t key1, bool fp64_only,
                                       unsigned long long& fallbacks, bool& accepted, int32_t& j) {
    accepted = false;
    if (!(q > 0.0)) return false;
    const uint4 r = philox4x32_10(make_uint4(d, static_cast<uint32_t>(k), static_cast<uint32_t>(i), sample), key0,
                                  key1);
    d += 1;
    const int64_t room = static_cast<int64_t>(b) - pos - 1;  // candidates left in the segment
    int64_t skip;  // floor(t), or >= room when the segment ends
    if (q >= 1.0) {
      skip = 0;
    } else {
      skip = skip_floor(r.y, r.x, q, room, fp64_only, fallbacks);
    }
    if (skip >= room) return false;
    j = pos + 1 + static_cast<int32_t>(skip);
    const double V = unit_open1(r.w, r.z);
    double p, qn;
    if (!uecm) {
      p = prob_ubcm(xi, g.xs[j]);
      qn = p;
    } else {
      const double aj = g.as[j];
      p = prob_uecm(xi, aj, yi * g.ys[j]);
      qn = prob_hat(xi, aj, c);
    }
    accepted = V < p / q;
    q = qn;
    pos = j;
    return true;
  }
};

__global__ void __launch_bounds__(kWalkWarps * 32) walk_kernel(WalkParams P) {
  extern __shared__ int32_t slots[];
  const Net& g = P.g;
  Ctrl* ctrl = P.ctrl;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int32_t* my_slot = slots + (warp * 32 + lane) * kSlotStride;
  const bool fp64_only = (g.flags & MH_FP64_ONLY) != 0;

  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;
  const unsigned long long total = static_cast<unsigned long long>(S) * P.c.chunk_samples;
  const unsigned lt = lanemask_lt();

  SegWalker wk;
  bool active = false;
  long long item = 0;
  unsigned long long next = 0, end = 0;  // warp-uniform chunk cursor
  bool work_left = total > 0;
  unsigned long long n_draws = 0, n_edges = 0, n_segs = 0, n_fallback = 0;

  while (true) {
    if (work_left) {
      unsigned idle = __ballot_sync(0xffffffffu, !active);
      while (idle && work_left) {
        if (next >= end) {
          unsigned long long t0 = 0;
          if (lane == 0) t0 = atomicAdd(&ctrl->ticket, static_cast<unsigned long long>(kWalkChunk));
          t0 = __shfl_sync(0xffffffffu, t0, 0);
          if (t0 >= total) {
            work_left = false;
            break;
          }
          next = t0;
          end = t0 + kWalkChunk < total ? t0 + kWalkChunk : total;
        }
        const unsigned long long avail = end - next;
        const unsigned rank = __popc(idle & lt);
        if (!active && rank < avail) {
          item = static_cast<long long>(next + rank);
          wk.init(g, item, S, P.c.sample0);
          active = true;
          n_segs += 1;
        }
        const unsigned take = __popc(idle);
        next += take < avail ? take : avail;
        idle = __ballot_sync(0xffffffffu, !active);
      }
    }
    if (__ballot_sync(0xffffffffu, active) == 0u) break;

    bool ended = false;
    if (active) {
      bool acc;
      int32_t j;
      if (wk.step(g, P.c.key0, P.c.key1, fp64_only, n_fallback, acc, j)) {
        if (acc) {
          if (wk.cnt < kSlot) my_slot[wk.cnt] = j;
          wk.cnt += 1;
        }
      } else {
        n_draws += wk.d;  // every Philox draw of the segment, the ending one included
        ended = true;
      }
    }

    const unsigned ended_mask = __ballot_sync(0xffffffffu, ended);
    if (ended_mask) {
      const bool direct = ended && wk.cnt <= kSlot;
      unsigned long long need = direct ? wk.cnt : 0;
      // warp-exclusive prefix of the staging need
      unsigned long long incl = need;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += o;
      }
      const unsigned long long warp_need = __shfl_sync(0xffffffffu, incl, 31);
      unsigned long long base0 = 0;
      if (lane == 0 && warp_need) base0 = atomicAdd(&ctrl->stage_used, warp_need);
      base0 = __shfl_sync(0xffffffffu, base0, 0);
      const unsigned long long my_base = base0 + incl - need;
      if (ended) {
        n_edges += wk.cnt;
        P.c.item_cnt[item] = wk.cnt;
        if (direct) {
          P.c.item_base[item] = static_cast<long long>(my_base);
          if (my_base + wk.cnt > static_cast<unsigned long long>(P.c.staging_cap))
            atomicOr(&ctrl->status, kStCapacity);
        } else {
          P.c.item_base[item] = -1;
          const unsigned long long slot_idx = atomicAdd(&ctrl->overflow_count, 1ull);
          P.c.ovf[slot_idx] = static_cast<int32_t>(item);
        }
      }
      __syncwarp();
      unsigned m = ended_mask;
      while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        const unsigned cnt_l = __shfl_sync(0xffffffffu, wk.cnt, l);
        const unsigned long long base_l = __shfl_sync(0xffffffffu, my_base, l);
        if (cnt_l <= static_cast<unsigned>(kSlot) &&
            base_l + cnt_l <= static_cast<unsigned long long>(P.c.staging_cap)) {
          const int32_t* src_slot = slots + (warp * 32 + l) * kSlotStride;
          for (unsigned e = lane; e < cnt_l; e += 32) P.c.staging[base_l + e] = src_slot[e];
        }
      }
      __syncwarp();
      if (ended) active = false;
    }
  }

  // statistics
#pragma unroll
  for (int dd = 16; dd; dd >>= 1) {
    n_draws += __shfl_xor_sync(0xffffffffu, n_draws, dd);
    n_edges += __shfl_xor_sync(0xffffffffu, n_edges, dd);
    n_segs += __shfl_xor_sync(0xffffffffu, n_segs, dd);
    n_fallback += __shfl_xor_sync(0xffffffffu, n_fallback, dd);
  }
  if (lane == 0) {
    atomicAdd(&ctrl->stats[MH_STAT_PROPOSALS], n_draws);
    atomicAdd(&ctrl->stats[MH_STAT_EDGES], n_edges);
    atomicAdd(&ctrl->stats[MH_STAT_SEGMENTS], n_segs);
    atomicAdd(&ctrl->stats[MH_STAT_FALLBACKS], n_fallback);
  }
}

// Segments with more edges than a shared-memory slot: walk again and write
// the ranks straight into staging.
__global__ void __launch_bounds__(128) overflow_kernel(WalkParams P) {
  const Net& g = P.g;
  Ctrl* ctrl = P.ctrl;
  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;
  const unsigned long long count = ctrl->overflow_count;
  const bool fp64_only = (g.flags & MH_FP64_ONLY) != 0;
  for (unsigned long long t = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; t < count;
       t += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    const long long item = P.c.ovf[t];
    const long long cnt = P.c.item_cnt[item];
    const unsigned long long base = atomicAdd(&ctrl->stage_used, static_cast<unsigned long long>(cnt));
    P.c.item_base[item] = static_cast<long long>(base);
    const bool fits = base + cnt <= static_cast<unsigned long long>(P.c.staging_cap);
    if (!fits) atomicOr(&ctrl->status, kStCapacity);
    SegWalker wk;
    wk.init(g, item, S, P.c.sample0);
    unsigned long long fb = 0;
    long long e = 0;
    bool acc;
    int32_t j;
    while (wk.step(g, P.c.key0, P.c.key1, fp64_only, fb, acc, j)) {
      if (acc) {
        if (fits && e < cnt) P.c.staging[base + e] = j;
        ++e;
      }
    }
  }
}

}  // namespace

cudaError_t launch_walk(const Net& g, const ChunkArgs& c, Ctrl* ctrl, cudaStream_t s) {
  WalkParams P{g, c, ctrl};
  const int threads = kWalkWarps * 32;
  const size_t smem = static_cast<size_t>(threads) * kSlotStride * sizeof(int32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(walk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  walk_kernel<<<static_cast<unsigned>(sm_count() * per_sm), threads, smem, s>>>(P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  overflow_kernel<<<static_cast<unsigned>(sm_count()), 128, 0, s>>>(P);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace mh
