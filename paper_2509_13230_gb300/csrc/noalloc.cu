// mh_sample_ubcm_noalloc: the UBCM sampler on a fixed scratch area instead of
// a caller-allocated workspace.
//
// Some callers cannot allocate device memory when they sample: code running
// under another framework's memory budget (its caching allocator owns the
// device memory, and a cudaMalloc / cudaFree here would bypass it, fragment
// it, or synchronise the device), runtimes that allow allocation only during
// initialisation, and plug-ins whose host forbids it.  This entry point lets
// them sample small networks with nothing but their inputs and outputs.
//
// Scratch.  A file-scope __device__ array of kNoAllocScratchBytes (64 MiB),
// which every GPU that loads the library holds until the process exits.  The
// first call on a device looks up its device address (cudaGetSymbolAddress)
// with that device current and, if no other call has yet, builds the
// library's logarithm table with one kernel on the caller's stream; make that
// first call before any stream capture (a call inside a capture is refused).
// Calls share the array: a process-wide lock serialises them and each call
// returns only after its device work is done, so calls through this entry
// point never overlap on a GPU; any other writer of the array would race.
// The sampling steps clear everything they read before writing it (the
// control block and the bound arrays), so leftovers of an earlier call do not
// matter.  No device or pinned host memory is allocated: kernels are launched
// directly (no graph) and results are read back into a static host buffer.
#include <cstring>
#include <mutex>

#include "mh_internal.cuh"

namespace mh {
namespace {

constexpr size_t kNoAllocScratchBytes = static_cast<size_t>(64) << 20;
constexpr uint32_t kNoAllocMaxSamples = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_lock;
void* g_noalloc_ptr[64] = {};
alignas(64) char g_noalloc_host[sizeof(Ctrl) + 8 * kNoAllocMaxSamples];

}  // namespace
}  // namespace mh

namespace mh {
int64_t take_launch_count();
void record_call_info(const mh_call_info& info);
}  // namespace mh

using namespace mh;

extern "C" int mh_sample_ubcm_noalloc(const double* x, int64_t n, const mh_params* params, int32_t* src,
                                      int32_t* dst, int64_t* csr_offsets, int32_t* csr_indices,
                                      int64_t capacity_edges, int64_t* h_edges_per_sample, uint64_t* h_stats,
                                      mh_stream_t stream) {
  std::lock_guard<std::mutex> guard(g_noalloc_lock);
  record_call_info(mh_call_info{0, 0, 0, 0.0, 0.0, 0.0, 0.0});  // this call's info, filled below
  int rc = check_sample_params(MH_UBCM, n, params);
  if (rc != MH_OK) return rc;
  if (!x || !h_edges_per_sample || capacity_edges < 0) {
    set_error("x and h_edges_per_sample must be non-NULL and capacity_edges >= 0");
    return MH_ERR_ARG;
  }
  if (params->num_samples > kNoAllocMaxSamples || (params->flags & (MH_TIMING | MH_CSR_SYMMETRIC))) {
    set_error("the fixed-scratch sampler takes at most %u samples per call, no MH_TIMING and no MH_CSR_SYMMETRIC",
              kNoAllocMaxSamples);
    return MH_ERR_ARG;
  }
  if ((params->flags & MH_OUT_COO) && capacity_edges > 0 && (!src || !dst)) {
    set_error("MH_OUT_COO needs src and dst");
    return MH_ERR_ARG;
  }
  if ((params->flags & MH_OUT_CSR) && (!csr_offsets || (capacity_edges > 0 && !csr_indices))) {
    set_error("MH_OUT_CSR needs csr_offsets and csr_indices");
    return MH_ERR_ARG;
  }
  const Layout L = make_layout(MH_UBCM, n, *params, capacity_edges);
  if (L.total > kNoAllocScratchBytes) {
    set_error("this call needs %zu bytes of scratch; the fixed scratch holds %zu (use mh_sample_ubcm)", L.total,
              kNoAllocScratchBytes);
    return MH_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    set_error("the fixed-scratch sampler reads results back and cannot run inside a stream capture");
    return e != cudaSuccess ? MH_ERR_CUDA : MH_ERR_ARG;
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_error("cudaGetDevice failed or device index out of range");
    return MH_ERR_CUDA;
  }
  if (!g_noalloc_ptr[dev]) {  // set-up, once per device, with that device current
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error("cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
      return MH_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  char* ws = static_cast<char*>(g_noalloc_ptr[dev]);
  // the device's logarithm table, built on the caller's stream the first time
  // (no stream of the library's own is created here)
  if (!ln_table_ptr(s)) {
    set_error("the logarithm table could not be built on this device");
    return MH_ERR_CUDA;
  }
  const Net g = net_view(MH_UBCM, *params, x, nullptr, n, L, ws);
  const Outputs o{src, dst, nullptr, reinterpret_cast<long long*>(csr_offsets), csr_indices, nullptr,
                  capacity_edges};
  take_launch_count();
  rc = enqueue_sample_direct(g, L, ws, params, o, g_noalloc_host, s);
  if (rc != MH_OK) {
    // kernels already queued may still write the shared scratch: let them
    // finish before the lock is released, so calls never overlap
    cudaStreamSynchronize(s);
    return rc;
  }
  mh_call_info info{0, 0, 0, 0.0, 0.0, 0.0, 0.0};
  info.kernel_launches = take_launch_count();
  info.sample_chunks = (params->num_samples + L.spc - 1) / L.spc;
  info.walk_launches = info.sample_chunks;
  record_call_info(info);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("cudaStreamSynchronize failed: %s", cudaGetErrorString(e));
    return MH_ERR_CUDA;
  }
  Ctrl hc;
  memcpy(&hc, g_noalloc_host, sizeof(Ctrl));
  const size_t counts_bytes = 8 * static_cast<size_t>(params->num_samples);
  memcpy(h_edges_per_sample, g_noalloc_host + sizeof(Ctrl), counts_bytes);
  if (h_stats)
    for (int t = 0; t < MH_NUM_STATS; ++t) h_stats[t] = hc.stats[t];
  rc = status_code(hc.status, hc.num_segments, L.max_segments);
  if (rc != MH_OK) return rc;
  int64_t total = 0;
  for (uint32_t t = 0; t < params->num_samples; ++t) total += h_edges_per_sample[t];
  if (total > capacity_edges || (hc.status & kStCapacity)) {
    set_error("the sample has %lld edges, capacity_edges is %lld", static_cast<long long>(total),
              static_cast<long long>(capacity_edges));
    return MH_ERR_CAPACITY;
  }
  return MH_OK;
}
