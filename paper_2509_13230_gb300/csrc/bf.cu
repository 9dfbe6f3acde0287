// Brute-force sampler (Sec. 2.2; the comparison baseline of Sec. 3): every
// pair u < v of original ids is an independent Bernoulli(p_uv), and a UECM
// edge draws its weight w ~ Geometric(1 - r_uv) on {1, 2, ...} (Eqs. 2-4).
// O(N^2) evaluations, against the walk's O(N + M): the comparison the paper's
// Fig. 3A and Fig. 4A make, here on the GPU.
//
// Random words: pair (u, v) of sample s takes Philox4x32-10 of the counter
// {u, v, 0xB0F0B0F0, s}; words (1,0) give the acceptance draw V on [0, 1),
// words (3,2) the weight draw U_w on (0, 1].  Edge kept when V < p_uv (FP64,
// p = z / (1 + z), z = x_u x_v; or A / ((1 - r) + A), A = (x_u y_u)(x_v y_v),
// r = y_u y_v); w = 1 + floor(log(U_w) / log(r)), w = 1 when r = 0.
//
// Decisions.  An FP32 estimate of p (per-node FP32 copies of x, y and x y)
// decides V < p when V lies more than p 2^-18 (UECM: 2^-17) from it; anything
// closer, and operands outside the FP32 ranges below, take the FP64
// expressions, so every edge is the FP64 decision.  Weights are FP64.
//
// Order and placement.  Pairs are numbered row-major over the upper
// triangle; blocks take chunks of kBfChunk consecutive pairs.  A count pass
// totals each chunk, an exclusive scan places the chunks, and a write pass
// evaluates the same pairs again and writes the kept ones in pair order, so
// the edges of a sample come out by (u, v), samples one after another.
#include "mh_internal.cuh"
#include "scan.cuh"
#include "walk_math.cuh"

namespace mh {

namespace {

constexpr int kBfThreads = 256;
constexpr int kBfWarps = kBfThreads / 32;
constexpr long long kBfChunk = 1ll << 16;  // pairs per block chunk
constexpr uint32_t kBfCounterWord = 0xB0F0B0F0u;

struct BfLayout {
  size_t ctrl = 0, chunk = 0, sample_counts = 0, xf = 0, yf = 0, af = 0, scan_counters = 0, scan_flags = 0,
         scan_values = 0, zero_begin = 0, zero_end = 0, total = 0;
  int64_t chunks = 0, scan_tiles = 0;
};

BfLayout bf_layout(int64_t n, const mh_params& p) {
  BfLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~static_cast<size_t>(255);
    return at;
  };
  const int64_t pairs = n * (n - 1) / 2;
  L.chunks = (pairs + kBfChunk - 1) / kBfChunk;
  L.ctrl = take(sizeof(Ctrl));
  L.chunk = take(8 * static_cast<size_t>(L.chunks + 1));
  L.sample_counts = take(8 * static_cast<size_t>(p.num_samples));
  L.xf = take(4 * static_cast<size_t>(n));
  L.yf = take(4 * static_cast<size_t>(n));
  L.af = take(4 * static_cast<size_t>(n));
  L.scan_tiles = (L.chunks + 1) / kScanTile + 2;
  L.zero_begin = off;
  L.scan_counters = take(16);
  L.scan_flags = take(4 * static_cast<size_t>(L.scan_tiles));
  L.zero_end = off;
  L.scan_values = take(2 * 8 * static_cast<size_t>(L.scan_tiles));
  L.total = off;
  return L;
}

struct BfArgs {
  const double* x;
  const double* y;
  const float* xf;  // FP32 copies (0 where the node's operands leave the FP32 ranges)
  const float* yf;
  const float* af;  // FP32 x y (UECM)
  long long n, pairs;
  uint32_t key0, key1, sample;
  long long* chunk;  // count pass: edges per chunk; write pass: exclusive edge offsets
  Ctrl* ctrl;
  long long* sample_count;  // this sample's edge count (write pass)
  int32_t *src, *dst, *w;
  long long capacity;
  bool fp64_only;
  bool chung_lu;  // p = min(1, x_u x_v) (MH_CHUNG_LU)
};

// Per-node operands and their validation (the domain of the sampling calls):
// x finite, >= 0 and <= 1e150; y in [0, 1).  FP32 copies are 0 for nodes
// whose pairs must take FP64 (x outside {0} and [2^-60, 2^60]; a = x y likewise;
// y above 7/8, where 1 - r loses too many FP32 bits).
__global__ void bf_prepare_kernel(int model, const double* __restrict__ x, const double* __restrict__ y, long long n,
                                  float* xf, float* yf, float* af, Ctrl* ctrl) {
  bool bad = false;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double xi = x[i];
    bad |= !(xi >= 0.0 && xi <= 1e150);
    const bool x_ok = xi == 0.0 || (xi >= 0x1p-60 && xi <= 0x1p60);
    xf[i] = x_ok ? __double2float_rn(xi) : 0.0f;
    if (model == MH_UECM) {
      const double yi = y[i];
      bad |= !(yi >= 0.0 && yi < 1.0);
      const double ai = xi * yi;
      const bool a_ok = ai == 0.0 || (ai >= 0x1p-60 && ai <= 0x1p60);
      yf[i] = (a_ok && yi <= 0.875) ? __double2float_rn(yi) : -1.0f;  // -1: FP64 pairs
      af[i] = a_ok ? __double2float_rn(ai) : 0.0f;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctrl->status, kStDomain);
}

// (u, v) of pair P: row u holds pairs [b(u), b(u + 1)), b(u) = u (2n - u - 1) / 2.
__device__ __forceinline__ void pair_of(long long P, long long n, long long& u, long long& v) {
  const double nn = static_cast<double>(n) - 0.5;
  long long uu = static_cast<long long>(nn - sqrt(nn * nn - 2.0 * static_cast<double>(P)));
  if (uu < 0) uu = 0;
  if (uu > n - 2) uu = n - 2;
  auto base = [n](long long r) { return r * (2 * n - r - 1) / 2; };
  while (uu > 0 && base(uu) > P) --uu;
  while (uu < n - 2 && base(uu + 1) <= P) ++uu;
  u = uu;
  v = P - base(uu) + uu + 1;
}

// The next pair of this thread: stride pairs further in row-major order.
__device__ __forceinline__ void advance_pair(long long stride, long long n, long long& u, long long& v) {
  v += stride;
  while (v >= n && u < n - 2) {
    const long long over = v - n;
    u += 1;
    v = u + 1 + over;
  }
}

// V < p_uv for the draw words r: FP32 filter, FP64 where it cannot decide.
template <bool kUecm>
__device__ __forceinline__ bool bf_keep(const BfArgs& A, long long u, long long v, uint4 r,
                                        unsigned long long& fallbacks) {
  const float vlo = __uint2float_rn(r.y >> 8) * 0x1p-24f;  // V in [vlo, vlo + 2^-24)
  const float vhi = vlo + 0x1p-24f;
  if (!A.fp64_only) {
    if (!kUecm) {
      const float xu = A.xf[u], xv = A.xf[v];
      if (xu == 0.0f || xv == 0.0f) {
        if (A.x[u] == 0.0 || A.x[v] == 0.0) return false;  // p = 0
      } else {
        const float z = xu * xv;
        const float pf = A.chung_lu ? fminf(z, 1.0f) : __fdividef(z, 1.0f + z);
        if (vhi <= pf * (1.0f - 0x1p-18f)) return true;
        if (vlo >= pf * (1.0f + 0x1p-18f)) return false;
      }
    } else {
      const float yu = A.yf[u], yv = A.yf[v];
      if (yu >= 0.0f && yv >= 0.0f) {
        const float au = A.af[u], av = A.af[v];
        if (au == 0.0f || av == 0.0f) {
          if (A.x[u] * A.y[u] == 0.0 || A.x[v] * A.y[v] == 0.0) return false;  // A = 0: p = 0
        } else {
          const float Af = au * av;
          const float omr = fmaf(-yu, yv, 1.0f);
          const float pf = __fdividef(Af, omr + Af);
          if (vhi <= pf * (1.0f - 0x1p-17f)) return true;
          if (vlo >= pf * (1.0f + 0x1p-17f)) return false;
        }
      }
    }
  }
  fallbacks += 1;
  double p;
  if (!kUecm) {
    const double z = A.x[u] * A.x[v];
    p = A.chung_lu ? (z >= 1.0 ? 1.0 : z) : z / (1.0 + z);
  } else {
    const double Ad = (A.x[u] * A.y[u]) * (A.x[v] * A.y[v]);
    const double rr = A.y[u] * A.y[v];
    p = Ad / ((1.0 - rr) + Ad);
  }
  return static_cast<double>(top53(r.y, r.x)) * 0x1p-53 < p;
}

template <bool kUecm>
__global__ void __launch_bounds__(kBfThreads) bf_count_kernel(BfArgs A) {
  __shared__ unsigned long long warp_tot[kBfWarps];
  if (A.ctrl->status & kStDomain) return;
  const long long c = blockIdx.x;
  const long long p0 = c * kBfChunk, p1 = p0 + kBfChunk < A.pairs ? p0 + kBfChunk : A.pairs;
  unsigned long long kept = 0, fallbacks = 0;
  if (p0 + threadIdx.x < p1) {
    long long u, v;
    pair_of(p0 + threadIdx.x, A.n, u, v);
    for (long long P = p0 + threadIdx.x; P < p1; P += kBfThreads) {
      const uint4 r = philox4x32_10(make_uint4(static_cast<uint32_t>(u), static_cast<uint32_t>(v), kBfCounterWord,
                                               A.sample), A.key0, A.key1);
      kept += bf_keep<kUecm>(A, u, v, r, fallbacks) ? 1u : 0u;
      advance_pair(kBfThreads, A.n, u, v);
    }
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    kept += __shfl_xor_sync(0xffffffffu, kept, d);
    fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, d);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_tot[warp] = kept;
  if (lane == 0 && fallbacks) atomicAdd(&A.ctrl->stats[MH_STAT_FALLBACKS], fallbacks);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kBfWarps; ++w) t += warp_tot[w];
    A.chunk[c] = static_cast<long long>(t);
  }
}

template <bool kUecm>
__global__ void __launch_bounds__(kBfThreads) bf_write_kernel(BfArgs A) {
  __shared__ unsigned warp_cnt[kBfWarps];
  __shared__ unsigned warp_off[kBfWarps];
  __shared__ unsigned step_total;
  if (A.ctrl->status & kStDomain) return;
  const long long c = blockIdx.x;
  if (c == 0 && threadIdx.x == 0) *A.sample_count = A.ctrl->out_end - A.ctrl->out_base;
  const long long p0 = c * kBfChunk, p1 = p0 + kBfChunk < A.pairs ? p0 + kBfChunk : A.pairs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  long long at = A.chunk[c];  // first edge of the chunk (global position)
  unsigned long long fallbacks = 0, boundary = 0, evals = 0;
  bool overflow = false;
  long long u = 0, v = 0;
  if (p0 + threadIdx.x < p1) pair_of(p0 + threadIdx.x, A.n, u, v);
  for (long long S0 = p0; S0 < p1; S0 += kBfThreads) {  // block-uniform steps
    const long long P = S0 + threadIdx.x;
    bool keep = false;
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (P < p1) {
      r = philox4x32_10(make_uint4(static_cast<uint32_t>(u), static_cast<uint32_t>(v), kBfCounterWord, A.sample),
                        A.key0, A.key1);
      keep = bf_keep<kUecm>(A, u, v, r, fallbacks);
      evals += 1;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_cnt[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned t = 0;
      for (int w = 0; w < kBfWarps; ++w) {
        warp_off[w] = t;
        t += warp_cnt[w];
      }
      step_total = t;
    }
    __syncthreads();
    if (keep) {
      const long long pos = at + warp_off[warp] + __popc(m & lt);
      int32_t wt = 1;
      if (kUecm) {
        const double rr = A.y[u] * A.y[v];
        if (rr > 0.0) {
          const double tw = log(static_cast<double>(top53(r.w, r.z) + 1ull) * 0x1p-53) / log(rr);
          if (near_integer(tw)) boundary += 1;
          if (tw >= 2147483646.0) {
            overflow = true;
            wt = 2147483647;
          } else {
            wt = 1 + static_cast<int32_t>(floor(tw));
          }
        }
      }
      if (pos < A.capacity) {
        A.src[pos] = static_cast<int32_t>(u);
        A.dst[pos] = static_cast<int32_t>(v);
        if (kUecm && A.w) A.w[pos] = wt;
      }
    }
    at += step_total;
    __syncthreads();  // step_total and the warp offsets are rewritten next step
    if (P < p1) advance_pair(kBfThreads, A.n, u, v);
  }
  (void)fallbacks;
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    evals += __shfl_xor_sync(0xffffffffu, evals, d);
    boundary += __shfl_xor_sync(0xffffffffu, boundary, d);
  }
  if (lane == 0) {
    atomicAdd(&A.ctrl->stats[MH_STAT_PROPOSALS], evals);
    if (boundary) atomicAdd(&A.ctrl->stats[MH_STAT_BOUNDARY], boundary);
  }
  if (overflow) atomicOr(&A.ctrl->status, kStOverflow);
}

}  // namespace

int run_bf(int model, const double* x, const double* y, int64_t n, const mh_params* p, void* workspace,
           size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w, int64_t capacity, int64_t* h_counts,
           uint64_t* h_stats, cudaStream_t s) {
  if (model != MH_UBCM && model != MH_UECM) {
    set_error("model must be MH_UBCM or MH_UECM");
    return MH_ERR_ARG;
  }
  int rc = check_sample_params(model, n, p);
  if (rc != MH_OK) return rc;
  if (n > 0x7FFFFFFFll) {
    set_error("n must be below 2^31");
    return MH_ERR_ARG;
  }
  if (!x || (model == MH_UECM && !y) || !workspace || !h_counts || capacity < 0 ||
      (capacity > 0 && (!src || !dst || (model == MH_UECM && !w)))) {
    set_error("x%s, workspace, h_edges_per_sample and (with capacity_edges > 0) src, dst%s must be non-NULL",
              model == MH_UECM ? ", y" : "", model == MH_UECM ? ", w" : "");
    return MH_ERR_ARG;
  }
  const BfLayout L = bf_layout(n, *p);
  if (workspace_bytes < L.total) {
    set_error("workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
    return MH_ERR_WORKSPACE;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    set_error("sampling calls read results back and cannot be captured into a caller's graph");
    return MH_ERR_ARG;
  }
  char* ws = static_cast<char*>(workspace);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  take_launch_count();
#define BF_CUDA(expr)                                                          \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      set_error("%s failed: %s", #expr, cudaGetErrorString(e_));               \
      cudaStreamSynchronize(s);                                                \
      return MH_ERR_CUDA;                                                      \
    }                                                                          \
  } while (0)
  BF_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
  BF_CUDA(cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_end - L.zero_begin, s));
  BfArgs A;
  A.x = x;
  A.y = model == MH_UECM ? y : nullptr;
  A.xf = reinterpret_cast<float*>(ws + L.xf);
  A.yf = reinterpret_cast<float*>(ws + L.yf);
  A.af = reinterpret_cast<float*>(ws + L.af);
  A.n = n;
  A.pairs = n * (n - 1) / 2;
  A.key0 = static_cast<uint32_t>(p->seed);
  A.key1 = static_cast<uint32_t>(p->seed >> 32) + p->network_id;
  A.chunk = reinterpret_cast<long long*>(ws + L.chunk);
  A.ctrl = ctrl;
  A.src = src;
  A.dst = dst;
  A.w = model == MH_UECM ? w : nullptr;
  A.capacity = capacity;
  A.fp64_only = (p->flags & MH_FP64_ONLY) != 0;
  A.chung_lu = (p->flags & MH_CHUNG_LU) != 0;
  auto* counts = reinterpret_cast<long long*>(ws + L.sample_counts);
  bf_prepare_kernel<<<grid_for(n, 256, static_cast<unsigned>(sm_count()) * 4u), 256, 0, s>>>(
      model, x, A.y, n, const_cast<float*>(A.xf), const_cast<float*>(A.yf), const_cast<float*>(A.af), ctrl);
  note_launches(1);
  BF_CUDA(cudaGetLastError());
  const ScanState st{reinterpret_cast<unsigned*>(ws + L.scan_flags), ws + L.scan_values,
                     reinterpret_cast<unsigned*>(ws + L.scan_counters), ctrl, L.scan_tiles};
  const unsigned grid = static_cast<unsigned>(L.chunks > 0 ? L.chunks : 1);
  for (uint32_t k = 0; k < p->num_samples; ++k) {
    A.sample = p->sample_begin + k;
    A.sample_count = counts + k;
    // this sample's edges follow those of the samples before it
    BF_CUDA(cudaMemcpyAsync(&ctrl->out_base, &ctrl->out_end, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    if (A.pairs > 0) {
      if (model == MH_UECM)
        bf_count_kernel<true><<<grid, kBfThreads, 0, s>>>(A);
      else
        bf_count_kernel<false><<<grid, kBfThreads, 0, s>>>(A);
      note_launches(1);
      BF_CUDA(cudaGetLastError());
    }
    BF_CUDA((scan_any<long long, SumOp<long long>>(A.chunk, A.chunk, ScanLen{L.chunks, nullptr, 1}, true,
                                                   &ctrl->out_base, &ctrl->out_end, false, st, s)));
    if (model == MH_UECM)
      bf_write_kernel<true><<<grid, kBfThreads, 0, s>>>(A);
    else
      bf_write_kernel<false><<<grid, kBfThreads, 0, s>>>(A);
    note_launches(1);
    BF_CUDA(cudaGetLastError());
  }
  Ctrl hc;
  BF_CUDA(cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  BF_CUDA(cudaMemcpyAsync(h_counts, counts, 8 * static_cast<size_t>(p->num_samples), cudaMemcpyDeviceToHost, s));
  BF_CUDA(cudaStreamSynchronize(s));
#undef BF_CUDA
  mh_call_info info{0, 0, 0, 0.0, 0.0, 0.0, 0.0};
  info.kernel_launches = take_launch_count();
  record_call_info(info);
  if (h_stats) {
    for (int t = 0; t < MH_NUM_STATS; ++t) h_stats[t] = hc.stats[t];
    h_stats[MH_STAT_EDGES] = 0;
    for (uint32_t k = 0; k < p->num_samples; ++k) h_stats[MH_STAT_EDGES] += static_cast<uint64_t>(h_counts[k]);
  }
  if (hc.status & kStDomain) {
    set_error("x must be finite, >= 0 and <= 1e150; y must be in [0, 1)");
    return MH_ERR_DOMAIN;
  }
  if (hc.status & kStTimeout) {
    set_error("a bounded device wait gave up");
    return MH_ERR_DEVICE_TIMEOUT;
  }
  if (hc.status & kStOverflow) {
    set_error("a sampled weight exceeds INT32_MAX");
    return MH_ERR_OVERFLOW;
  }
  if (hc.out_end > capacity) {
    set_error("the samples have %lld edges, capacity_edges is %lld", static_cast<long long>(hc.out_end),
              static_cast<long long>(capacity));
    return MH_ERR_CAPACITY;
  }
  return MH_OK;
}

size_t bf_workspace_bytes(int64_t n, const mh_params& p) { return bf_layout(n, p).total; }

}  // namespace mh

using namespace mh;

extern "C" {

int mh_bf_workspace_size(int model, int64_t n, const mh_params* params, size_t* h_bytes) {
  if (model != MH_UBCM && model != MH_UECM) {
    set_error("model must be MH_UBCM or MH_UECM");
    return MH_ERR_ARG;
  }
  const int rc = check_sample_params(model, n, params);
  if (rc != MH_OK) return rc;
  if (!h_bytes) {
    set_error("h_bytes must be non-NULL");
    return MH_ERR_ARG;
  }
  *h_bytes = bf_workspace_bytes(n, *params);
  return MH_OK;
}

int mh_sample_bf(int model, const double* x, const double* y, int64_t n, const mh_params* params, void* workspace,
                 size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w, int64_t capacity_edges,
                 int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream) {
  record_call_info(mh_call_info{0, 0, 0, 0.0, 0.0, 0.0, 0.0});
  return run_bf(model, x, y, n, params, workspace, workspace_bytes, src, dst, w, capacity_edges, h_edges_per_sample,
                h_stats, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
