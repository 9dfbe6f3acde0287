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
// Decision arithmetic (walk_math.cuh): each draw is decided from estimates
// with an error bound (pairs of FP32 numbers first, then double-float
// arithmetic) and falls back to the canonical FP64
// expressions only when it lies within that bound of a decision boundary
// (or outside the fast path's range).  The acceptance test compares V with
// the FP64 quotient p/q whenever the FP32 estimate is inconclusive, so the
// decisions reproduce the FP64 definition bit for bit.
//
// Scheduling.  Persistent warps take chunks of work items from a global
// ticket; an idle lane takes the chunk's next item, so lanes stay busy when
// segment lengths differ.  A lane buffers accepted ranks j in its
// shared-memory slot; when its segment ends, the warp reserves staging space
// with one atomic and copies the slot out with coalesced stores.  A segment
// with more than kSlot edges is walked a second time by the same lane (the
// walk is a pure function of the counter), now writing straight into a
// staging range of exactly the counted size.
#include "mh_internal.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

struct WalkParams {
  Net g;
  ChunkArgs c;
  Ctrl* ctrl;
  BatchQueue q;    // batched waves only
  PhiloxKeys rk;   // round keys of (key0, key1); batched waves use rk.k0 and each network's key1
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// One segment's walk state.  A lane's iteration is either the head of a new
// segment (q <- p at the head, no draw consumed) or one candidate; both run
// the same code for the next draw (Philox, -ln U), the product x_i x_j and
// the next q, so a warp whose lanes start segments at different times stays
// converged.  The next draw is computed one iteration ahead: it does not
// depend on this iteration's decisions, so the dependency chains overlap.
//
// Decisions go through three levels: first-level estimates of E, lambda and
// t as pairs of FP32 numbers (walk_math.cuh, within 2^-30.4 t of the
// canonical t) decide almost every draw; draws within that level's margin of
// a boundary recompute t in double-float from the kept product; draws within
// that margin, or with q outside the fast range, use the canonical FP64
// expressions.
struct SegWalker {
  int32_t i, k, a, b, pos, qj;  // qj: the rank whose p (or phat) is the current q
  uint32_t sample, d;           // d: index of the next draw
  bool fresh;                   // the head of the segment is still to be set up
  bool fast;                    // q lies inside the fast levels' range
  int32_t gi;                   // slot of row i in the row arrays
  int32_t ex;                   // directed: the candidate row i skips (its own in-copy)
  uint32_t seg;                 // segment-table row (UECM: its bound constant c)
  df2 xi_df, yi_df, inv1mc;     // double-float x_i (a_i), y_i and 1 / (1 - c)
  float omc_f;                  // 1 - c in FP32
  df2 zq;                       // -ln(1 - q) = log1p(zq): zq = x_i x_j (UBCM) or A / (1 - c) (UECM)
  df2 lam;                      // log1p(zq), first level
  float q_f;                    // q in FP32
  uint4 rnd;                    // Philox words of draw d
  df2 E;                        // -ln U of draw d, first level

  // Canonical FP64 values are read back on the (rare) FP64 paths.
  __device__ __forceinline__ double q64(const Net& g, bool uecm) const {
    if (uecm) return prob_hat(g.as_r[gi], g.as[qj], g.seg_c[seg]);
    return (g.flags & MH_CHUNG_LU) ? prob_cl(g.xs_r[gi], g.xs[qj]) : prob_ubcm(g.xs_r[gi], g.xs[qj]);
  }

  // Loads row segment `seg` of sample `smp`; its head is set up by the next
  // advance().  Segment rows hold ranks local to their network; nb is the
  // network's first slot in the node arrays (0 for a single network), so a,
  // b, pos and j index the node arrays while i stays the local rank that the
  // Philox counter uses.  Directed networks (kExcl): a, b, pos and the
  // walk's positions are virtual, counting the candidates without the
  // excluded one ex; candidate v is rank v below ex and v + 1 from ex on.
  template <bool kExcl = false>
  __device__ __forceinline__ void begin_seg(const Net& g, unsigned sg, uint32_t smp, int nb, bool uecm) {
    const int4 e = g.seg[sg];
    seg = sg;
    i = e.x;
    k = e.y;
    a = nb + e.z;
    b = nb + e.w;
    if (kExcl) {
      ex = g.excl[e.x];
      a -= a > ex;
      b -= b > ex;
    }
    pos = a - 1;
    sample = smp;
    d = 0;
    fresh = true;
    gi = nb + e.x;
    if (!uecm) {
      xi_df = to_df(g.xdf_r[gi]);
    } else {
      xi_df = to_df(g.adf_r[gi]);
      yi_df = to_df(g.ydf_r[gi]);
      const float4 cf = g.seg_cf[sg];
      inv1mc = df2{cf.x, cf.y};
      omc_f = cf.z;
    }
  }

  // Single network: work item = (sample within the chunk, segment).
  template <bool kExcl = false>
  __device__ __forceinline__ void begin(const Net& g, long long item, long long S, uint32_t sample0, bool uecm) {
    // item < 2^31 (the workspace layout bounds the items of a chunk)
    const unsigned s_local = static_cast<unsigned>(item) / static_cast<unsigned>(S);
    const unsigned seg = static_cast<unsigned>(item) - s_local * static_cast<unsigned>(S);
    begin_seg<kExcl>(g, seg, sample0 + s_local, 0, uecm);
  }

  // One iteration.  Returns false when the segment has ended; sets
  // `accepted` / `j` when a candidate was evaluated (never on a head step).
  template <bool kUecm, bool kExcl = false, bool kLaneKey = false>
  __device__ __forceinline__ bool advance(const Net& g, const PhiloxKeys& rk, uint32_t key1, bool fp64_only,
                                          bool init_prev, const LnEntry* tab, unsigned& fallbacks,
                                          unsigned long long& boundary, bool& accepted, int32_t& j) {
    accepted = false;
    const bool head = fresh;
    if (kExcl && head && a >= b) return false;  // the segment held only the excluded candidate
    const bool fast_q = !head && fast && !fp64_only;
    double qc = 0.0;  // canonical q, computed only when a decision needs it
    bool have_qc = false;
    if (!head && !fast_q) {
      qc = q64(g, kUecm);
      have_qc = true;
      if (!(qc > 0.0)) return false;
    }
    const uint4 r = rnd;
    const df2 t1 = quot_df(E, lam);
    if (!head) d += 1;
    // Philox words and -ln U of the next draw (draw 0 on a head step)
    rnd = philox4x32_10_rk<!kLaneKey>(make_uint4(d, static_cast<uint32_t>(k), static_cast<uint32_t>(i), sample), rk,
                                      key1);
    E = neg_ln_u53_m(top53(rnd.y, rnd.x) + 1ull, tab);
    int32_t jv;  // position of the candidate (virtual when kExcl)
    if (head) {
      fresh = false;
      jv = init_prev ? a - 1 : a;
    } else {
      const int room = b - pos - 1;
      unsigned skip = 0;
      bool decided = fast_q && floor_decided_m(t1, room, skip);
      if (!decided && fast_q) {  // double-float level
        const int fl = skip_df(top53(r.y, r.x) + 1ull, zq, room, tab);
        decided = fl >= 0;
        if (decided) skip = static_cast<unsigned>(fl);
      }
      if (!decided) {  // canonical FP64
        if (fast_q) fallbacks += 1;
        if (!have_qc) {
          qc = q64(g, kUecm);
          have_qc = true;
        }
        skip = skip_fp64(top53(r.y, r.x) + 1ull, qc, room, boundary);
      }
      if (skip >= static_cast<unsigned>(room)) return false;
      jv = pos + 1 + static_cast<int32_t>(skip);
    }
    j = kExcl ? jv + (jv >= ex) : jv;  // the candidate's rank
    // product x_i x_j (a_i a_j) for the acceptance test and the next q
    const df2 prod = df_mul(xi_df, to_df(kUecm ? g.adf[j] : g.xdf[j]));
    if (!head) {
      const unsigned long long mV = top53(r.w, r.z);  // V = mV 2^-53
      int verdict = -1;
      if (!kUecm) {
        if (fast_q && prod.hi > 0x1p-100f && prod.hi < 0x1p40f)
          verdict = accept_decided(r.w, __fdividef(prod.hi, 1.0f + prod.hi), q_f);
      } else {
        const df2 yj = to_df(g.ydf[j]);
        const float omr = fmaf(-yi_df.hi, yj.hi, 1.0f) - fmaf(yi_df.hi, yj.lo, yi_df.lo * yj.hi);
        if (fast_q && prod.hi > 0x1p-100f && prod.hi < 0x1p40f && omr > 0x1p-20f)
          verdict = accept_decided(r.w, __fdividef(prod.hi, omr + prod.hi), q_f);
      }
      if (verdict < 0) {
        if (fast_q) fallbacks += 1;
        if (!have_qc) qc = q64(g, kUecm);
        const double p = kUecm                     ? prob_uecm(g.as_r[gi], g.as[j], g.ys_r[gi] * g.ys[j])
                         : (g.flags & MH_CHUNG_LU) ? prob_cl(g.xs_r[gi], g.xs[j])
                                                   : prob_ubcm(g.xs_r[gi], g.xs[j]);
        verdict = (static_cast<double>(mV) * 0x1p-53 < p / qc) ? 1 : 0;
      }
      accepted = verdict != 0;
      pos = jv;
    }
    // q <- p (UBCM) or phat (UECM) of j
    qj = j;
    if (!kUecm) {
      zq = prod;
      fast = prod.hi > 0x1p-100f && prod.hi < kFastZq;
      q_f = __fdividef(prod.hi, 1.0f + prod.hi);
    } else {
      zq = df_mul(prod, inv1mc);
      fast = zq.hi > 0x1p-100f && zq.hi < kFastZq && omc_f >= 0x1p-20f;
      q_f = __fdividef(prod.hi, omc_f + prod.hi);
    }
    lam = fast ? log1p_m(zq, tab) : df2{1.0f, 0.0f};
    return true;
  }
};

// Batched waves: position `qpos` of a model's queue lies in network
// order[p], where p is the last queue entry with mb[p] <= qpos.  Entries of
// networks without work have mb[p] == mb[p + 1] and are passed over.
__device__ __forceinline__ int queue_entry(const BatchQueue& q, unsigned long long qpos) {
  int lo = 0, hi = q.n_order - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (static_cast<unsigned long long>(q.mb[mid]) <= qpos)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Sets up the work item at queue position qpos, starting the network search
// at entry p (a position at or before qpos's entry).  Returns the global
// work item (its slot in item_cnt / item_base) and the network's key word.
template <bool kUecm>
__device__ __forceinline__ long long begin_queued(const Net& g, const BatchQueue& q, unsigned long long qpos, int p,
                                                  SegWalker& wk, uint32_t& key1) {
  while (p + 1 < q.n_order && static_cast<unsigned long long>(q.mb[p + 1]) <= qpos) ++p;
  const int t = q.order[p];
  const WaveNet& w = q.wave[t];
  // a wave holds fewer than 2^31 work items and a network fewer than 2^31 rows
  const unsigned local = static_cast<unsigned>(qpos - static_cast<unsigned long long>(q.mb[p]));
  const unsigned S = static_cast<unsigned>(w.S);
  const unsigned s_local = local / S;
  const unsigned seg = local - s_local * S;
  const BatchNet& bn = q.nets[t];
  key1 = w.key1;
  wk.begin_seg(g, static_cast<unsigned>(bn.seg_base) + seg, w.sample_lo + s_local, static_cast<int>(bn.node_base),
               kUecm);
  if (q.seg_slot)  // CSR wave: the item's slot among its sample's rows in node-id order
    return w.item_begin + static_cast<long long>(s_local) * S + q.seg_slot[bn.seg_base + seg];
  return w.item_begin + local;
}

// kMode: 0 one network, 1 batched waves, 2 one directed network.
template <bool kUecm, int kMode>
__global__ void __launch_bounds__(kWalkWarps * 32, 3) walk_kernel(WalkParams P) {
  constexpr bool kBatch = kMode == 1;
  constexpr bool kExcl = kMode == 2;
  extern __shared__ unsigned char smem_raw[];
  LnEntry* tab = reinterpret_cast<LnEntry*>(smem_raw);
  int32_t* slots = reinterpret_cast<int32_t*>(smem_raw + sizeof(LnEntry) * kLnTable);
  ln_table_to_shared(tab, P.g.lntab);
  __syncthreads();

  const Net& g = P.g;
  Ctrl* ctrl = P.ctrl;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int32_t* my_slot = slots + (warp * 32 + lane) * kSlotStride;
  // the Chung-Lu law (MH_CHUNG_LU) has no fast levels: every draw is FP64
  const bool fp64_only = (g.flags & (MH_FP64_ONLY | MH_CHUNG_LU)) != 0;
  const bool init_prev = (g.flags & MH_INIT_PREV) != 0;
  const unsigned long long cap = static_cast<unsigned long long>(P.c.staging_cap);
  const uint32_t key1 = P.c.key1;

  long long S = ctrl->num_segments;
  if (S > g.max_segments) S = g.max_segments;
  // single network: a truncated segment table (more rows than max_segments)
  // fails the call with MH_ERR_WORKSPACE, so it is not walked
  const bool truncated = !kBatch && ctrl->num_segments > g.max_segments;
  const unsigned long long total = kBatch      ? static_cast<unsigned long long>(*P.q.total)
                                   : truncated ? 0ull
                                               : static_cast<unsigned long long>(S) * P.c.chunk_samples;
  unsigned long long* const ticket = kBatch ? P.q.ticket : &ctrl->ticket;
  // work items per ticket: about 1/8 of an even share, within [32, 1024]
  const unsigned long long warps = static_cast<unsigned long long>(gridDim.x) * kWalkWarps;
  unsigned long long chunk = total / (warps * 8ull);
  chunk = chunk < 32ull ? 32ull : (chunk > 1024ull ? 1024ull : chunk);
  const unsigned lt = lanemask_lt();

  SegWalker wk;
  bool active = false;
  bool rewalk = false;           // second pass of an overflowing segment
  unsigned cnt = 0;              // edges of the current pass
  unsigned long long rbase = 0;  // staging base of a second pass
  unsigned item = 0;  // a chunk or a wave holds fewer than 2^31 work items
  unsigned qpos = 0;        // batched: the lane's queue position (< 2^31)
  uint32_t lane_key1 = key1;
  int qcur = 0;             // batched: queue entry at or before the chunk's first position
  unsigned long long next = 0, end = 0;     // warp-uniform work cursor
  unsigned long long wbase = 0;  // warp-uniform staging chunk: next free entry
  unsigned wleft = 0;            // and entries left (at most kStageChunk)
  bool work_left = total > 0;
  // Per-lane statistics in 32 bits (registers are the walk's occupancy limit),
  // added to the call's 64-bit totals at the end and whenever n_draws passes
  // 2^28: a segment adds fewer than 2^31 draws, at most two fallbacks per draw
  // and pass, and at least one draw, so no counter wraps.
  unsigned n_draws = 0, n_edges = 0, n_segs = 0, n_fallback = 0;
  unsigned long long n_boundary = 0;
  auto flush_stats = [&]() {
    atomicAdd(&ctrl->stats[MH_STAT_PROPOSALS], static_cast<unsigned long long>(n_draws));
    atomicAdd(&ctrl->stats[MH_STAT_EDGES], static_cast<unsigned long long>(n_edges));
    atomicAdd(&ctrl->stats[MH_STAT_SEGMENTS], static_cast<unsigned long long>(n_segs));
    atomicAdd(&ctrl->stats[MH_STAT_FALLBACKS], static_cast<unsigned long long>(n_fallback));
    n_draws = n_edges = n_segs = n_fallback = 0;
  };

  // A lane whose segment ended keeps its run in its slot (pending) until
  // the warp flushes: when kFlushMin runs are pending, or when no lane is
  // walking.  Flushed lanes are then refilled together, so the warp-wide
  // placement, copy and refill steps run once per several finished segments.
  bool pending = false;
  while (true) {
    const unsigned act_mask = __ballot_sync(0xffffffffu, active);
    const unsigned pend_mask = __ballot_sync(0xffffffffu, pending);
    if (pend_mask && (__popc(pend_mask) >= kFlushMin || act_mask == 0u)) {
      // Place the pending lanes' runs in the warp's staging chunk, in lane
      // order; lanes that do not fit go to a fresh chunk (a run never spans
      // two chunks, so each segment stays contiguous).
      const unsigned need = pending ? cnt : 0u;  // a pending run holds at most kSlot ranks
      unsigned incl = need;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += o;
      }
      const unsigned excl = incl - need;
      const unsigned warp_need = __shfl_sync(0xffffffffu, incl, 31);
      const bool fits = incl <= wleft;
      const unsigned spill_mask = __ballot_sync(0xffffffffu, pending && !fits);
      unsigned long long my_base = wbase + excl;
      if (spill_mask) {
        const int first = __ffs(spill_mask) - 1;  // lanes from `first` on move to the new chunk
        const unsigned moved_excl = __shfl_sync(0xffffffffu, excl, first);
        const unsigned long long rest = warp_need - moved_excl;
        const unsigned long long want = rest > static_cast<unsigned long long>(kStageChunk) ? rest : kStageChunk;
        unsigned long long nb = 0;
        if (lane == 0) nb = atomicAdd(&ctrl->stage_used, want);
        nb = __shfl_sync(0xffffffffu, nb, 0);
        if (lane >= first) my_base = nb + (excl - moved_excl);
        wbase = nb + rest;
        wleft = static_cast<unsigned>(want - rest);
      } else {
        wbase += warp_need;
        wleft -= warp_need;
      }
      if (pending) {
        P.c.item_cnt[item] = cnt;
        P.c.item_base[item] = static_cast<long long>(my_base);
        if (my_base + cnt > cap) atomicOr(&ctrl->status, kStCapacity);
      }
      __syncwarp();
      // Copy all pending runs in one pass: element idx of the concatenated
      // runs belongs to the last lane whose exclusive prefix is <= idx.
      const int32_t* wslots = slots + warp * 32 * kSlotStride;
      for (unsigned r0 = 0; r0 < warp_need; r0 += 32) {
        const unsigned idx = r0 + lane;
        int l = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const unsigned v = __shfl_sync(0xffffffffu, excl, l + step);
          if (v <= idx) l += step;
        }
        const unsigned ex_l = __shfl_sync(0xffffffffu, excl, l);
        const unsigned long long base_l = __shfl_sync(0xffffffffu, my_base, l);
        if (idx < warp_need) {
          const unsigned e = idx - ex_l;
          if (base_l + e < cap) P.c.staging[base_l + e] = wslots[l * kSlotStride + e];
        }
      }
      __syncwarp();
      pending = false;
    }
    if (work_left) {
      unsigned idle = __ballot_sync(0xffffffffu, !active && !pending);
      if (idle && (__popc(idle) >= kFlushMin || act_mask == 0u)) {
        while (idle && work_left) {
          if (next >= end) {
            unsigned long long t0 = 0;
            if (lane == 0) t0 = atomicAdd(ticket, chunk);
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            if (t0 >= total) {
              work_left = false;
              break;
            }
            if (kBatch) qcur = queue_entry(P.q, t0);  // the same on every lane
            next = t0;
            end = t0 + chunk < total ? t0 + chunk : total;
          }
          const unsigned long long avail = end - next;
          const unsigned rank = __popc(idle & lt);
          if (!active && !pending && rank < avail) {
            if (kBatch) {
              qpos = static_cast<unsigned>(next + rank);
              item = static_cast<unsigned>(begin_queued<kUecm>(g, P.q, next + rank, qcur, wk, lane_key1));
            } else {
              item = static_cast<unsigned>(next + rank);
              wk.begin<kExcl>(g, item, S, P.c.sample0, kUecm);
              // node-order CSR: the record goes to the segment's slot among its sample's rows
              if (P.c.seg_slot)
                item = (wk.sample - P.c.sample0) * static_cast<unsigned>(S) + static_cast<unsigned>(P.c.seg_slot[wk.seg]);
            }
            active = true;
            rewalk = false;
            cnt = 0;
            n_segs += 1;
          }
          const unsigned take = __popc(idle);
          next += take < avail ? take : avail;
          idle = __ballot_sync(0xffffffffu, !active && !pending);
        }
      }
    }
    if (__ballot_sync(0xffffffffu, active || pending) == 0u) break;

    if (active) {
      bool acc;
      int32_t j;
      if (wk.advance<kUecm, kExcl, kBatch>(g, P.rk, kBatch ? lane_key1 : key1, fp64_only, init_prev, tab,
                                           n_fallback, n_boundary, acc, j)) {
        if (acc) {
          if (!rewalk) {
            if (cnt < static_cast<unsigned>(kSlot)) my_slot[cnt] = j;
          } else if (rbase + cnt < cap) {
            P.c.staging[rbase + cnt] = j;
          }
          cnt += 1;
        }
      } else if (rewalk) {
        active = false;  // second pass done; count and base were recorded
      } else {
        n_draws += wk.d;
        n_edges += cnt;
        if (n_draws >= (1u << 28)) flush_stats();
        if (cnt == 0) {
          active = false;  // nothing to place: the lane is free at once
          P.c.item_cnt[item] = 0;
          P.c.item_base[item] = 0;
        } else if (cnt <= static_cast<unsigned>(kSlot)) {
          active = false;
          pending = true;  // the run waits in the slot for the next flush
        } else {
          // too many edges for the slot: reserve exactly cnt entries and walk again
          rbase = atomicAdd(&ctrl->stage_used, static_cast<unsigned long long>(cnt));
          if (rbase + cnt > cap) atomicOr(&ctrl->status, kStCapacity);
          P.c.item_cnt[item] = cnt;
          P.c.item_base[item] = static_cast<long long>(rbase);
          if (kBatch)
            begin_queued<kUecm>(g, P.q, qpos, queue_entry(P.q, qpos), wk, lane_key1);
          else  // the item's queue position: (sample in the chunk, segment)
            wk.begin<kExcl>(g, static_cast<long long>(wk.sample - P.c.sample0) * S + wk.seg, S, P.c.sample0,
                            kUecm);
          rewalk = true;
          cnt = 0;
        }
      }
    }
  }

  unsigned long long t_draws = n_draws, t_edges = n_edges, t_segs = n_segs, t_fallback = n_fallback;
#pragma unroll
  for (int dd = 16; dd; dd >>= 1) {
    t_draws += __shfl_xor_sync(0xffffffffu, t_draws, dd);
    t_edges += __shfl_xor_sync(0xffffffffu, t_edges, dd);
    t_segs += __shfl_xor_sync(0xffffffffu, t_segs, dd);
    t_fallback += __shfl_xor_sync(0xffffffffu, t_fallback, dd);
    n_boundary += __shfl_xor_sync(0xffffffffu, n_boundary, dd);
  }
  if (lane == 0) {
    atomicAdd(&ctrl->stats[MH_STAT_PROPOSALS], t_draws);
    atomicAdd(&ctrl->stats[MH_STAT_EDGES], t_edges);
    atomicAdd(&ctrl->stats[MH_STAT_SEGMENTS], t_segs);
    atomicAdd(&ctrl->stats[MH_STAT_FALLBACKS], t_fallback);
    if (n_boundary) atomicAdd(&ctrl->stats[MH_STAT_BOUNDARY], n_boundary);
  }
}

// The walk's first decision level on given inputs (mh_debug_first_level).
__global__ void first_level_probe_kernel(const unsigned long long* N, const double* z, const int32_t* room,
                                         long long n, const LnEntry* tab, float2* E_out, float2* lam_out,
                                         int32_t* fl_out) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const df2 E = neg_ln_u53_m(N[i], tab);
    const df2 lam = log1p_m(df_from_double(z[i]), tab);
    unsigned fl = 0;
    const int decided = floor_decided_m(quot_df(E, lam), room[i], fl);
    E_out[i] = make_float2(E.hi, E.lo);
    lam_out[i] = make_float2(lam.hi, lam.lo);
    fl_out[i] = decided ? static_cast<int32_t>(fl) : -1;
  }
}

}  // namespace

cudaError_t launch_first_level_probe(const unsigned long long* N, const double* z, const int32_t* room, long long n,
                                     float* E_out, float* lam_out, int32_t* fl_out, cudaStream_t s) {
  const LnEntry* tab = ln_table_ptr(s);
  if (!tab) return cudaErrorLaunchFailure;
  const long long want = (n + 255) / 256;
  const unsigned grid = static_cast<unsigned>(want < 1024 ? (want < 1 ? 1 : want) : 1024);
  first_level_probe_kernel<<<grid, 256, 0, s>>>(N, z, room, n, tab, reinterpret_cast<float2*>(E_out),
                                                reinterpret_cast<float2*>(lam_out), fl_out);
  note_launches(1);
  return cudaGetLastError();
}

size_t walk_smem_bytes() {
  return sizeof(LnEntry) * kLnTable + static_cast<size_t>(kWalkWarps) * 32 * kSlotStride * sizeof(int32_t);
}

// Shared-memory opt-in and occupancy of the walk kernels, per device (done
// before a call is captured into a graph).
static int g_per_sm[64][2][3] = {};

template <bool kUecm, int kMode>
static cudaError_t walk_attributes(int dev) {
  if (g_per_sm[dev][kUecm][kMode]) return cudaSuccess;
  auto kernel = walk_kernel<kUecm, kMode>;
  const size_t smem = walk_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWalkWarps * 32, smem);
  if (e != cudaSuccess) return e;
  g_per_sm[dev][kUecm][kMode] = per_sm < 1 ? 1 : per_sm;
  return cudaSuccess;
}

cudaError_t prepare_kernel_attributes(int model) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if ((e = sort_kernel_attributes(dev)) != cudaSuccess) return e;
  if (!ln_table_ptr()) return cudaErrorLaunchFailure;  // built here, before any capture
  if (model == MH_UECM) {
    if ((e = walk_attributes<true, 0>(dev)) != cudaSuccess) return e;
    if ((e = walk_attributes<true, 1>(dev)) != cudaSuccess) return e;
    return walk_attributes<true, 2>(dev);
  }
  if ((e = walk_attributes<false, 0>(dev)) != cudaSuccess) return e;
  if ((e = walk_attributes<false, 1>(dev)) != cudaSuccess) return e;
  return walk_attributes<false, 2>(dev);
}

static unsigned walk_blocks(int dev, bool uecm, int mode, int ctas_per_sm) {
  int per_sm = g_per_sm[dev][uecm][mode];
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  int blocks = sm_count() * per_sm;
  if (blocks * kWalkWarps > kMaxWalkWarps) blocks = kMaxWalkWarps / kWalkWarps;
  return static_cast<unsigned>(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_walk(const Net& g, const ChunkArgs& c, Ctrl* ctrl, cudaStream_t s) {
  WalkParams P{g, c, ctrl, BatchQueue{}, philox_round_keys(c.key0, c.key1)};
  const bool uecm = g.model == MH_UECM;
  const int mode = g.excl ? 2 : 0;
  cudaError_t e = prepare_kernel_attributes(g.model);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  auto kernel = uecm ? (mode ? walk_kernel<true, 2> : walk_kernel<true, 0>)
                     : (mode ? walk_kernel<false, 2> : walk_kernel<false, 0>);
  kernel<<<walk_blocks(dev, uecm, mode, c.walk_ctas_per_sm), kWalkWarps * 32, walk_smem_bytes(), s>>>(P);
  note_launches(1);
  return cudaGetLastError();
}

// One persistent launch over the queue of one model's networks in a wave;
// g holds the concatenated arrays of all networks.
cudaError_t launch_walk_batched(const Net& g, const ChunkArgs& c, const BatchQueue& q, Ctrl* ctrl, int model,
                                cudaStream_t s) {
  WalkParams P{g, c, ctrl, q, philox_round_keys(c.key0, c.key1)};
  const bool uecm = model == MH_UECM;
  cudaError_t e = prepare_kernel_attributes(model);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  auto kernel = uecm ? walk_kernel<true, 1> : walk_kernel<false, 1>;
  kernel<<<walk_blocks(dev, uecm, 1, c.walk_ctas_per_sm), kWalkWarps * 32, walk_smem_bytes(), s>>>(P);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mh
