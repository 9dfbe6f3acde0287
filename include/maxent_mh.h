/*
 * maxent_mh.h — C ABI of the GB300 sampler for maximum-entropy network
 * models (Li, Wang, Kojaku, "Fast unbiased sampling of networks with given
 * expected degrees and strengths", arXiv 2509.13230).
 *
 * Parameters.  The paper writes node parameters as alpha_i (degree) and
 * beta_i (strength).  This ABI takes x_i = exp(-alpha_i) >= 0 and
 * y_i = exp(-beta_i) in [0, 1), as FP64 arrays indexed by original node id.
 *
 *   UBCM edge probability (Sec. 2.2, Eq. 1):  p_ij = x_i x_j / (1 + x_i x_j)
 *   UECM edge probability (Sec. 2.5, Eq. 3):  p_ij = A / (1 - r + A),
 *        A = x_i y_i x_j y_j,  r = y_i y_j
 *   UECM weight given an edge (Eq. 4):         P(w) = r^(w-1) (1 - r), w >= 1
 *
 * Memory.  Every pointer is a DEVICE pointer unless its name starts with
 * h_ (host memory).  The caller owns all memory, including the workspace,
 * whose size mh_workspace_size() returns.  Nothing here allocates device
 * memory; the library keeps one small pinned host buffer per thread for the
 * final read-back of counts.
 *
 * Streams.  All device work is ordered on the given stream (NULL = the
 * legacy default stream).  The sampling calls read back the edge counts and
 * a status word at the end, so they return only after their device work is
 * done; the maxent_expected_* calls (sums, gradient, row ranges, Jacobian
 * diagonal) return without synchronising.
 *
 * Errors.  Every call returns MH_OK (0) or a negative MH_ERR_* code; no C++
 * exception crosses the ABI.  mh_error_string() names a code and
 * mh_last_error_detail() gives the calling thread's last message.
 *
 * Sampled bits.  A sample is a pure function of (x, y, seed, network_id,
 * sample index, seg_target, flags): re-running a call reproduces it bit for
 * bit, and sample s of a batch equals the same sample drawn alone.
 */
#ifndef MAXENT_MH_H
#define MAXENT_MH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mh_stream_t; /* the same handle as cudaStream_t */

/* models */
#define MH_UBCM 0 /* unweighted binary configuration model, Eq. 1          */
#define MH_UECM 1 /* weighted enhanced configuration model, Eqs. 2-4       */

/* return codes */
#define MH_OK 0
#define MH_ERR_ARG -1            /* bad size, null required pointer, bad flag        */
#define MH_ERR_DOMAIN -2         /* x not finite / < 0 / > 1e150, or y outside [0,1) */
#define MH_ERR_CAPACITY -3       /* output shorter than the sample; counts returned  */
#define MH_ERR_WORKSPACE -4      /* workspace too small or segment table overflow    */
#define MH_ERR_OVERFLOW -5       /* a weight above INT32_MAX                         */
#define MH_ERR_DEVICE_TIMEOUT -6 /* a bounded device wait gave up                    */
#define MH_ERR_CUDA -7           /* a CUDA runtime call failed                       */

/* flags */
#define MH_OUT_COO 0x01u     /* write src/dst (and w) edge arrays                  */
#define MH_OUT_CSR 0x02u     /* write CSR offsets/indices (and weights)            */
#define MH_BOUND_PAPER 0x10u /* UECM: c = product of the two largest y among the   */
                             /* nodes not yet processed (Sec. 2.5); default is     */
                             /* c = y_i * max_{j >= segment head} y_j              */
#define MH_INIT_PREV 0x20u   /* first proposal q = p at the rank before the        */
                             /* segment head (p_ii for a row's first segment,      */
                             /* Sec. 2.4 step (ii)); default: q = p at the head    */
#define MH_DIRECTED 0x40u    /* mh_sample_bipartite: a directed network (Sec. 2.6) */
#define MH_CSR_SYMMETRIC 0x80u /* with MH_OUT_CSR, mh_sample_ubcm / _weighted only:  */
                               /* every edge in both endpoint rows, each row's      */
                               /* neighbours in node order (descending key, ties by */
                               /* ascending id); csr_indices and csr_weights then   */
                               /* hold 2 x capacity_edges entries                   */
#define MH_FP64_ONLY 0x100u  /* decide every draw with the plain FP64 path         */
#define MH_TIMING 0x200u     /* time the call's phases with CUDA events on the     */
                             /* caller's stream (see mh_last_call_info); calls of  */
                             /* more than 1024 sample chunks are not timed         */
#define MH_CHUNG_LU 0x800u   /* mh_sample_ubcm, mh_sample_bf (MH_UBCM), the        */
                             /* fixed-scratch call: the Chung-Lu law              */
                             /* p_ij = min(1, x_i x_j) instead of Eq. 1 (Sec. 2.1: */
                             /* the expected multiplicity k_i k_j / 2M read as a  */
                             /* probability), sampled by the same walk (the       */
                             /* Miller-Hagberg original, Sec. 2.3) with every     */
                             /* draw decided by the FP64 expressions; for         */
                             /* comparisons with the UBCM                          */
#define MH_TEST_WAIT_TIMEOUT 0x400u /* test hook for the bounded device waits: in    */
                             /* every single-pass scan of the call, tile 1 first    */
                             /* waits on a device flag that nothing sets; the wait  */
                             /* gives up after 4096 polls (well under a            */
                             /* millisecond) exactly as a real look-back wait that  */
                             /* ran out would, and the scan then finishes normally. */
                             /* The call returns MH_ERR_DEVICE_TIMEOUT; the device  */
                             /* stays usable and the next call is unaffected.       */
                             /* Needs at least 2 scan tiles (2,049 values) to fire. */

/* stats slots (h_stats, MH_NUM_STATS x uint64) */
#define MH_STAT_PROPOSALS 0 /* candidate draws                                     */
#define MH_STAT_EDGES 1     /* accepted edges                                      */
#define MH_STAT_SEGMENTS 2  /* segments walked (samples x table rows)              */
#define MH_STAT_FALLBACKS 3 /* skip draws the fast levels left to the FP64 path    */
#define MH_STAT_BOUNDARY 4  /* boundary draws: a skip draw whose FP64 t =           */
                            /* log(U)/log1p(-q) lies within 8 ulp of an integer m  */
                            /* with 1 <= m <= b - pos - 1 (the integers that decide */
                            /* the candidate), or a weight draw whose FP64         */
                            /* log(U_w)/log(r) >= 0.5 lies within 8 ulp of an      */
                            /* integer.  Only these draws may decide differently   */
                            /* from a host FP64 evaluation (the device and host    */
                            /* log/log1p may differ by an ulp); every other draw   */
                            /* is decided as in FP64 (Sec. 2.3 skip, Eq. 4)        */
#define MH_NUM_STATS 5

typedef struct mh_params {
    uint64_t seed;         /* Philox key: (seed lo32, seed hi32 + network_id)       */
    uint32_t network_id;   /* 0 for single-network calls                            */
    uint32_t sample_begin; /* first sample index (Philox counter word 3)            */
    uint32_t num_samples;  /* samples drawn by this call, >= 1                      */
    uint32_t seg_target;   /* T: expected proposals per row segment, >= 2;          */
                           /* 0 selects 32.  Part of a sample's identity.           */
    uint32_t flags;        /* MH_OUT_*, MH_BOUND_PAPER, MH_INIT_PREV, MH_FP64_ONLY  */
    uint32_t walk_ctas_per_sm; /* proposal-walk blocks per SM, 0 = as many as fit;   */
                               /* a schedule choice only: samples do not change    */
    int64_t max_segments;  /* row-segment table capacity; 0 selects 4 n + 1024      */
} mh_params;

/* Per-call record of the calling thread's last sampling call. */
typedef struct mh_call_info {
    int64_t kernel_launches; /* kernels this library launched in the call          */
    int64_t walk_launches;   /* launches of the proposal-walk kernel                */
    int64_t sample_chunks;   /* sample chunks the call was split into               */
    double prepare_ms;       /* MH_TIMING: sort + bound prep + segment table        */
    double walk_ms;          /* MH_TIMING: proposal walk (all chunks)               */
    double emit_ms;          /* MH_TIMING: scans + edge output (all chunks)         */
    double total_ms;         /* MH_TIMING: whole call, device time                  */
} mh_call_info;

/* Name of a return code (static string). */
const char* mh_error_string(int code);

/* Last error message of the calling thread (static per-thread buffer). */
const char* mh_last_error_detail(void);

/* Copies the calling thread's last mh_call_info (zeros before any call). */
int mh_last_call_info(mh_call_info* h_info);

/*
 * Workspace bytes for a sampling call on a network of n nodes whose output
 * holds up to capacity_edges edges (all samples of the call together).
 * Returns MH_ERR_ARG for n < 1, capacity_edges < 0 or a bad params struct.
 */
int mh_workspace_size(int model, int64_t n, const mh_params* params, int64_t capacity_edges, size_t* h_bytes);

/*
 * mh_sample_ubcm — Miller-Hagberg rejection sampling of the UBCM (Sec. 2.3,
 * Sec. 2.4 steps (i)-(iv)).  Nodes are sorted by descending x (ascending
 * alpha), each row i's candidates j > i are cut into segments of about
 * seg_target expected proposals, and each segment is walked with geometric
 * skips of parameter q, acceptance with probability p_ij / q and q <- p_ij.
 *
 *   x                 FP64[n], original node order
 *   src, dst          COO output, int32[capacity_edges] each (MH_OUT_COO),
 *                     original node ids; edge (u, v) has u the endpoint of
 *                     higher x.  Samples are concatenated in sample order,
 *                     edges of a sample in (rank of u, rank of v) order.
 *   csr_offsets       int64[num_samples * (n + 1)] (MH_OUT_CSR): sample s,
 *                     node u owns csr_indices[off[s(n+1)+u] .. off[s(n+1)+u+1]),
 *                     the edges whose higher-ranked endpoint is u; offsets are
 *                     global positions in csr_indices.
 *   csr_indices       int32[capacity_edges] (MH_OUT_CSR)
 *                     With MH_CSR_SYMMETRIC every edge is listed in both
 *                     endpoint rows (row u: all neighbours of u in node
 *                     order), offsets are global positions in a
 *                     csr_indices of int32[2 * capacity_edges], and sample
 *                     s starts at twice the edges of the samples before it.
 *                     This is a layout of the same sample: the edges, their
 *                     weights and the counts are unchanged.
 *   capacity_edges    length of each edge output array (< 2^31 with
 *                     MH_CSR_SYMMETRIC)
 *   h_edges_per_sample host int64[num_samples]: edges of each sample
 *   h_stats           host uint64[MH_NUM_STATS] (MH_STAT_*), or NULL
 *
 * On MH_ERR_CAPACITY the exact counts are in h_edges_per_sample and nothing
 * past capacity_edges was written; re-calling with more room reproduces the
 * same sample.
 */
int mh_sample_ubcm(const double* x, int64_t n, const mh_params* params, void* workspace, size_t workspace_bytes,
                   int32_t* src, int32_t* dst, int64_t* csr_offsets, int32_t* csr_indices, int64_t capacity_edges,
                   int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream);

/*
 * mh_sample_weighted — the UECM sampler of Algorithm 1 (Sec. 2.5).  Nodes are
 * sorted by descending a = x y (ascending alpha + beta); proposals use the
 * bound phat_ij = A / (1 - c + A) of Eq. 5 with q <- phat_ij, and each
 * accepted edge draws its weight w ~ Geometric(1 - r_ij) on {1, 2, ...}.
 * Arguments as mh_sample_ubcm, plus
 *   y                 FP64[n] in [0, 1)
 *   w, csr_weights    int32[capacity_edges] weights aligned with src/dst and
 *                     csr_indices (either may be NULL when its layout is off)
 */
int mh_sample_weighted(const double* x, const double* y, int64_t n, const mh_params* params, void* workspace,
                       size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w, int64_t* csr_offsets,
                       int32_t* csr_indices, int32_t* csr_weights, int64_t capacity_edges,
                       int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream);

/*
 * mh_sample_range — the share of mh_sample_ubcm / mh_sample_weighted that
 * lies in rows [seg_begin, seg_end) of the segment table (the table
 * mh_segment_table exports for the same arguments).  The walk of a segment
 * depends only on the segment, the sample and the key (Sec. 2.3: each
 * segment head restarts the proposal bound; the Philox counter names the
 * segment), so ranges that tile [0, S) and are concatenated in range order
 * give exactly the whole call's edges, for every sample.  This is how one
 * large sample is split across GPUs: each rank draws a contiguous range and
 * an exclusive scan of the ranks' edge counts places its edges.
 *   model             MH_UBCM (y ignored) or MH_UECM
 *   seg_begin/_end    0 <= seg_begin <= seg_end; rows past the table's end
 *                     are empty
 *   src, dst, w       COO int32[capacity_edges] (w: MH_UECM); sample s's
 *                     edges of the range follow those of sample s - 1
 *   other arguments   as mh_sample_weighted; params->flags must not ask for
 *                     MH_OUT_CSR or MH_CSR_SYMMETRIC (MH_ERR_ARG)
 *   h_edges_per_sample, h_stats: of the range only
 * Workspace: mh_workspace_size of the whole call.  Errors as
 * mh_sample_weighted (a truncated table: MH_ERR_WORKSPACE).
 */
int mh_sample_range(int model, const double* x, const double* y, int64_t n, const mh_params* params,
                    int64_t seg_begin, int64_t seg_end, void* workspace, size_t workspace_bytes, int32_t* src,
                    int32_t* dst, int32_t* w, int64_t capacity_edges, int64_t* h_edges_per_sample,
                    uint64_t* h_stats, mh_stream_t stream);

/*
 * Bipartite and directed networks (Sec. 2.6).  The + set's nodes are the
 * rows, each walked over every node of the - set; each set is sorted by its
 * own key (descending x, or a = x y for MH_UECM), so
 *   UBCM form  p_ij = x+_i x-_j / (1 + x+_i x-_j)
 *   UECM form  p_ij = A / (1 - r + A),  A = x+_i y+_i x-_j y-_j,  r = y+_i y-_j
 * with the proposal bound c = y+_i max_{j >= segment head} y-_j.  With
 * MH_DIRECTED the + set holds every node's out-parameters and the - set
 * its in-parameters (n_plus == n_minus, the same ids): edge (u, v) is u -> v
 * and the pairs (i, i) are never proposed.
 *
 * Workspace bytes for mh_sample_bipartite (as mh_workspace_size).
 */
int mh_bipartite_workspace_size(int model, int64_t n_plus, int64_t n_minus, const mh_params* params,
                                int64_t capacity_edges, size_t* h_bytes);

/*
 * mh_sample_bipartite — samples of a bipartite (or, with MH_DIRECTED, a
 * directed) network.  Arguments as mh_sample_weighted with
 *   x_plus, y_plus      FP64[n_plus]  (y only for MH_UECM, else NULL)
 *   x_minus, y_minus    FP64[n_minus]
 *   src, dst            + id and - id of each edge (out and in node when
 *                       directed); a sample's edges in (+ rank, - rank) order
 *   w, csr_weights      MH_UECM weights (else NULL)
 *   csr_offsets         int64[num_samples * (n_plus + 1)]: rows are + ids
 * MH_BOUND_PAPER and MH_INIT_PREV do not apply (MH_ERR_ARG); MH_DIRECTED
 * needs n_plus == n_minus.  max_segments (0: 4 n_plus + 1024) must be at
 * least n_plus.  Errors as mh_sample_weighted.
 */
int mh_sample_bipartite(int model, const double* x_plus, const double* y_plus, int64_t n_plus,
                        const double* x_minus, const double* y_minus, int64_t n_minus, const mh_params* params,
                        void* workspace, size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w,
                        int64_t* csr_offsets, int32_t* csr_indices, int32_t* csr_weights, int64_t capacity_edges,
                        int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream);

/*
 * Batched ensembles: many networks of uneven size, UBCM and UECM mixed, each
 * sampled num_samples times.  The paper samples one network at a time
 * (Sec. 2.4, Algorithm 1); batching only schedules those same samples, so
 * sample s of network t is bit-identical to mh_sample_ubcm / _weighted on
 * that network alone with network_id = nets[t].network_id and
 * sample_begin = params->sample_begin + s.
 *
 * Work is split into (network, sample) PAIRS, numbered network-major:
 * pair p is network t = p / num_samples, sample params->sample_begin +
 * p % num_samples.  One mh_sample_batched call draws a contiguous range of
 * pairs (a wave) with one persistent walk launch per model over all of the
 * wave's (network, sample, row segment) work items, then writes the wave's
 * edges in pair order.  The caller sizes waves so their work items fit
 * max_wave_items and their edges fit capacity_edges; the segment counts
 * from mh_batch_prepare give the items of a pair exactly.
 */
typedef struct mh_network_desc {
    int32_t model;        /* MH_UBCM or MH_UECM                                   */
    uint32_t network_id;  /* Philox key word 1 = hi32(seed) + network_id         */
    int64_t n;            /* nodes, >= 1                                          */
    const double* x;      /* FP64[n], >= 0                                        */
    const double* y;      /* FP64[n] in [0, 1) for MH_UECM; NULL for MH_UBCM     */
    int64_t max_segments; /* this network's segment-table rows; 0 = the params   */
                          /* value (0 there: 4 n + 1024); else >= n - 1         */
} mh_network_desc;

/*
 * Workspace bytes for a batch: the prepared networks (about 112 bytes per
 * node plus 52 bytes per segment-table row, the node-order slot maps of CSR
 * waves included) and the larger of the sort scratch and a wave's buffers
 * (20 bytes per work item, staging for capacity_edges edges).
 *   h_nets           host array of n_nets descriptors (1 <= n_nets <= 65536,
 *                    sum of n < 2^31 - 2^20)
 *   params           seed, sample_begin, num_samples (per network),
 *                    seg_target, flags, max_segments (the default of every
 *                    network's segment-table rows); network_id must be 0
 *   max_wave_items   work items one wave may hold, in [1, 2^30]; 0 selects 2^26
 *   capacity_edges   edges one wave may write
 */
int mh_batch_workspace_size(const mh_network_desc* h_nets, int32_t n_nets, const mh_params* params,
                            int64_t max_wave_items, int64_t capacity_edges, size_t* h_bytes);

/*
 * mh_batch_prepare — sort, bound prep and segment table of every network
 * (Sec. 2.4 step (i), Algorithm 1's ordering and bound, row segments), kept
 * in the workspace for any number of mh_sample_batched calls.  Networks are
 * prepared on several internal streams joined back to `stream`.
 *   h_num_segments   host int64[n_nets]: segment-table rows of each network;
 *                    a pair of network t is h_num_segments[t] work items
 * Errors: MH_ERR_DOMAIN (a bad x or y; the detail names the network),
 * MH_ERR_WORKSPACE (workspace too small, or a network's segment table above
 * its max_segments: h_num_segments holds every network's needed rows).
 */
int mh_batch_prepare(const mh_network_desc* h_nets, int32_t n_nets, const mh_params* params, void* workspace,
                     size_t workspace_bytes, int64_t* h_num_segments, mh_stream_t stream);

/*
 * mh_sample_batched — one wave: pairs [pair_begin, pair_begin + pair_count).
 * The workspace must hold mh_batch_prepare's result for the same h_nets and
 * params (same n, model, x and y pointers, seg_target, MH_BOUND_PAPER and
 * max_segments; the seed, sample_begin, network ids and the other flags may
 * differ).  A workspace prepared for other networks gives MH_ERR_ARG.
 *   src, dst, w      COO (MH_OUT_COO), int32[capacity_edges]; the wave's
 *                    edges in pair order, each pair's edges in the order of
 *                    the single-network call; ids are node ids within the
 *                    pair's network; w only when the wave has UECM networks
 *   csr_offsets      int64 (MH_OUT_CSR): for each pair of the wave in order,
 *                    n_t + 1 offsets into csr_indices (as mh_sample_ubcm's
 *                    per-sample offsets); sum over the wave's pairs of n_t + 1
 *                    entries
 *   csr_indices, csr_weights  int32[capacity_edges]
 *   h_edges_per_pair host int64[pair_count]: edges of each pair
 *   h_stats          host uint64[MH_NUM_STATS] (MH_STAT_*) of the wave, or NULL
 * pair_count must be >= 1 and at most 2^20.  MH_ERR_WORKSPACE when the
 * wave has more than max_wave_items work items or the workspace is too
 * small; MH_ERR_CAPACITY as for the single-network calls (exact counts are
 * returned and a larger capacity_edges reproduces the wave).
 */
int mh_sample_batched(const mh_network_desc* h_nets, int32_t n_nets, const mh_params* params,
                      int64_t max_wave_items, void* workspace, size_t workspace_bytes, int64_t pair_begin,
                      int64_t pair_count, int32_t* src, int32_t* dst, int32_t* w, int64_t* csr_offsets,
                      int32_t* csr_indices, int32_t* csr_weights, int64_t capacity_edges,
                      int64_t* h_edges_per_pair, uint64_t* h_stats, mh_stream_t stream);

/*
 * mh_bf_workspace_size / mh_sample_bf — the brute-force sampler (Sec. 2.2;
 * the comparison baseline of Sec. 3): every pair u < v of original ids is an
 * independent Bernoulli(p_uv) (Eq. 1, or Eq. 3 for MH_UECM), and a UECM edge
 * draws its weight w ~ Geometric(1 - r_uv) on {1, 2, ...} (Eq. 4).  N (N - 1)
 * / 2 pair evaluations per sample, against the walk's O(N + M).
 *   Random words of pair (u, v) in sample s: Philox4x32-10 of the counter
 *   {u, v, 0xB0F0B0F0, s}, key (seed lo32, seed hi32 + network_id); words
 *   (1,0) give V on [0, 1), kept when V < p_uv (FP64); words (3,2) give
 *   U_w on (0, 1], w = 1 + floor(log(U_w) / log(r)) (w = 1 when r = 0).
 *   Samples [sample_begin, sample_begin + num_samples) one after another,
 *   each sample's edges by (u, v).  Agrees with the walk in distribution,
 *   not in bits.
 *   model, x, y, n, params   as mh_sample_weighted (num_samples, seed,
 *                           network_id, sample_begin and MH_FP64_ONLY are
 *                           read; segment length and output flags are not)
 *   src, dst, w            COO int32[capacity_edges] (w: MH_UECM)
 *   h_edges_per_sample     host int64[num_samples]
 *   h_stats                host uint64[MH_NUM_STATS] or NULL: pair
 *                          evaluations (MH_STAT_PROPOSALS), edges, FP64
 *                          decisions, weight boundary draws
 * Workspace: mh_bf_workspace_size (about 12 B per node plus 8 B per 2^16
 * pairs).  MH_ERR_CAPACITY keeps the exact counts; re-calling with more room
 * draws the same samples.  Other errors as mh_sample_weighted.
 */
int mh_bf_workspace_size(int model, int64_t n, const mh_params* params, size_t* h_bytes);
int mh_sample_bf(int model, const double* x, const double* y, int64_t n, const mh_params* params, void* workspace,
                 size_t workspace_bytes, int32_t* src, int32_t* dst, int32_t* w, int64_t capacity_edges,
                 int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream);

/*
 * mh_sample_ubcm_noalloc — mh_sample_ubcm without a caller-supplied
 * workspace.  The paper has no counterpart: this is an interface for callers
 * that cannot allocate device memory while they sample, such as code that
 * runs inside another framework's memory budget (a cudaMalloc / cudaFree
 * here would bypass its caching allocator or synchronise the device),
 * runtimes that allow allocation only at start-up, and plug-ins whose host
 * forbids it.  It allocates nothing: its scratch is a fixed 64 MiB device
 * array inside the library, held by every GPU that loads the library until
 * the process exits, and results are read back into a static host buffer.
 *
 * Arguments as mh_sample_ubcm (no workspace).  Limits: the call's
 * mh_workspace_size must fit in the 64 MiB (about n <= 50,000 with a few
 * million edges; otherwise MH_ERR_WORKSPACE, use mh_sample_ubcm),
 * num_samples <= 1024 (otherwise MH_ERR_ARG), no MH_TIMING, no
 * MH_CSR_SYMMETRIC.  The first call on a device looks up the scratch's
 * device address and, unless another call already did, builds the library's
 * logarithm table on the caller's stream; make it before any stream capture.
 * Called inside a capture it returns MH_ERR_ARG and enqueues nothing.  Calls
 * share the scratch: the library serialises them with a process-wide lock
 * and each returns after its device work (also on an error return), so
 * calls through this function never overlap on a GPU; any other kernel
 * that wrote the scratch would race with them.  Each call clears what it
 * reads before it writes it, so calls of any size may follow one another.
 * mh_last_call_info describes the call (launches, sample chunks).
 * Output is bit-identical to mh_sample_ubcm with the same arguments.
 */
int mh_sample_ubcm_noalloc(const double* x, int64_t n, const mh_params* params, int32_t* src, int32_t* dst,
                           int64_t* csr_offsets, int32_t* csr_indices, int64_t capacity_edges,
                           int64_t* h_edges_per_sample, uint64_t* h_stats, mh_stream_t stream);

/*
 * mh_segment_table — the node order and row-segment table a sampling call
 * with the same arguments walks (for inspection and tests).
 *   seg_row, seg_k    int32[cap]: row rank i and segment index k within row i
 *   seg_a, seg_b      int64[cap]: segment candidates are ranks [a, b)
 *   perm              int32[n]: perm[rank] = original node id
 *   h_num_segments    host: number of segments (written even when > cap)
 * Returns MH_ERR_CAPACITY when the table has more than cap rows.
 */
int mh_segment_table(int model, const double* x, const double* y, int64_t n, const mh_params* params,
                     void* workspace, size_t workspace_bytes, int32_t* seg_row, int32_t* seg_k, int64_t* seg_a,
                     int64_t* seg_b, int32_t* perm, int64_t cap, int64_t* h_num_segments, mh_stream_t stream);

/*
 * mh_debug_first_level — the walk's first decision level on given inputs,
 * for tests of its error bound.  The walk's skip is L = 1 + floor(t) with
 * t = E / lambda, E = -ln U, lambda = -ln(1 - q) (Sec. 2.3, Fig. 2); the
 * first level evaluates E and lambda as pairs (hi, lo) of FP32 numbers and
 * decides floor(t) only when t lies farther than t 2^-28 + 2^-22 from every
 * integer.  For i < n:
 *   E_out[2i], E_out[2i+1]      the pair for E = -ln(N[i] 2^-53), N[i] in [1, 2^53]
 *   lam_out[2i], lam_out[2i+1]  the pair for lambda = log1p(z[i]), z[i] in [2^-100, 2^16)
 *                               (z[i] is first rounded to a double-float, as the walk holds it)
 *   fl_out[i]                   floor(t) capped at room[i] (0 <= room[i] < 2^31), or -1 when
 *                               the level leaves the draw to the next one
 * All arrays are device memory owned by the caller (N uint64[n], z FP64[n],
 * room int32[n], E_out and lam_out FP32[2n], fl_out int32[n]); outside the
 * stated ranges the outputs are unspecified.  MH_ERR_ARG for n < 0 or a NULL
 * pointer with n > 0.  Asynchronous on `stream`; builds the library's
 * logarithm table on first use.
 */
int mh_debug_first_level(const uint64_t* N, const double* z, const int32_t* room, int64_t n, float* E_out,
                         float* lam_out, int32_t* fl_out, mh_stream_t stream);

/*
 * maxent_expected_fwd — expected degrees and strengths, the O(N^2) sums
 * behind maximum-likelihood inference (Sec. 2.2, Sec. 2.5, Sec. 4):
 *   k_out[i] = sum_{j != i} p_ij
 *   s_out[i] = sum_{j != i} p_ij / (1 - r_ij)     (UECM; E[w | w > 0] = 1/(1-r))
 * x, y (y NULL for UBCM), k_out, s_out (NULL for UBCM): FP64[n].
 * Each pair term is recomputed tile by tile; no N^2 storage.
 */
int maxent_expected_fwd(int model, const double* x, const double* y, int64_t n, double* k_out, double* s_out,
                        mh_stream_t stream);

/*
 * maxent_expected_bwd — gradient of a loss L(<k>, <s>) with respect to x
 * (and y) given g_k = dL/d<k> and g_s = dL/d<s> (NULL for UBCM):
 *   g_x[i] = sum_{j != i} (g_k[i] + g_k[j]) dp_ij/dx_i + (g_s[i] + g_s[j]) dm_ij/dx_i
 * with m_ij = p_ij / (1 - r_ij); g_y likewise with d/dy_i (UECM; NULL for UBCM).
 */
int maxent_expected_bwd(int model, const double* x, const double* y, int64_t n, const double* g_k,
                        const double* g_s, double* g_x, double* g_y, mh_stream_t stream);

/*
 * maxent_expected_jacobian_diag — the diagonal of the Jacobian of the
 * expected sums: for every node i the derivatives of its own <k_i> (and
 * <s_i>) with respect to its own x_i (and y_i), the other parameters fixed
 * (the per-node blocks a Newton step's preconditioner inverts; Sec. 2.2,
 * Sec. 2.5):
 *   dk_dx[i] = sum_{j != i} dp_ij/dx_i      dk_dy[i] = sum_{j != i} dp_ij/dy_i
 *   ds_dx[i] = sum_{j != i} dm_ij/dx_i      ds_dy[i] = sum_{j != i} dm_ij/dy_i
 * x, y (y NULL for UBCM) and the outputs are FP64[n]; the UBCM returns dk_dx
 * only (dk_dy, ds_dx, ds_dy NULL).  One pass over the pairs, where two
 * maxent_expected_bwd calls with unit upstream gradients would give the same
 * values (each pair term then counted from both of its ends).
 */
int maxent_expected_jacobian_diag(int model, const double* x, const double* y, int64_t n, double* dk_dx,
                                  double* dk_dy, double* ds_dx, double* ds_dy, mh_stream_t stream);

/*
 * maxent_expected_jacobian_diag_rows — the same for rows
 * [row_begin, row_begin + row_count) over all columns: outputs hold
 * row_count entries, entry r being row row_begin + r, bit for bit the value
 * of the whole call (a row's sum does not depend on the rows launched with
 * it).  With the _rows forms of the sums and gradient it lets ranks of a
 * distributed fit each evaluate their own block of rows.  Errors as
 * maxent_expected_fwd_rows.
 */
int maxent_expected_jacobian_diag_rows(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                                       int64_t row_count, double* dk_dx, double* dk_dy, double* ds_dx, double* ds_dy,
                                       mh_stream_t stream);

/*
 * maxent_expected_fwd_rows / maxent_expected_bwd_rows — the sums of
 * maxent_expected_fwd / _bwd (Sec. 2.2, Sec. 2.5, Sec. 4) for the rows i in
 * [row_begin, row_begin + row_count) only (every sum still runs over all
 * j != i), so that ranks can share one call by rows with no reduction:
 * x, y, g_k, g_s are FP64[n] as above (all rows' values are needed); k_out,
 * s_out, g_x, g_y hold row_count values, entry r for row row_begin + r.  Each
 * value equals, bit for bit, the one the whole call returns for that row.
 * MH_ERR_ARG unless 0 <= row_begin, 0 <= row_count and row_begin + row_count
 * <= n; row_count = 0 returns MH_OK without work (the pointers may then be
 * NULL).  The whole-range calls above keep their order of checks: with
 * n >= 1 a NULL required pointer is MH_ERR_ARG.
 */
int maxent_expected_fwd_rows(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                             int64_t row_count, double* k_out, double* s_out, mh_stream_t stream);
int maxent_expected_bwd_rows(int model, const double* x, const double* y, int64_t n, int64_t row_begin,
                             int64_t row_count, const double* g_k, const double* g_s, double* g_x, double* g_y,
                             mh_stream_t stream);

/*
 * maxent_expected_fwd_sym / maxent_expected_jacobian_diag_sym /
 * maxent_expected_bwd_sym — the whole-range sums of maxent_expected_fwd,
 * maxent_expected_jacobian_diag and maxent_expected_bwd (same arguments,
 * same outputs, Sec. 2.2, Sec. 2.5, Sec. 4), with every unordered pair
 * {i, j} evaluated once for both of its rows: p_ij = p_ji, and each
 * derivative term is a factor symmetric in i and j times a_j (row i) or a_i
 * (row j), a = x (UBCM) or x y (UECM).  Half the pair terms of the row forms.
 *
 * Results are deterministic (fixed order of additions, independent of the
 * grid and timing) and within the error bound of the row forms (about 1e-11
 * of the sum of the terms' magnitudes), but not bit for bit equal to them:
 * the additions run in another order.  The _rows forms above stay the ones
 * whose rows equal the whole call bit for bit.
 *
 * workspace: device memory of at least maxent_expected_sym_workspace_size()
 * bytes, 256-byte aligned, owned by the caller, not kept after the call's
 * work; it holds the double-float copies of the operands and one partial
 * sum per (quantity, band of columns, node): 8 q ceil(n / L) n bytes with
 * L = max(2048, n / 128 rounded up to a multiple of 512) and q = 1 (UBCM),
 * 3 (UECM).  Calls on one stream may share it; concurrent calls may not.
 * Errors: MH_ERR_ARG (model, n < 1 or n > 2^31, a NULL required pointer,
 * misaligned workspace), MH_ERR_WORKSPACE (NULL or too small), MH_ERR_CUDA.
 * The calls return without synchronising.
 */
int maxent_expected_sym_workspace_size(int model, int64_t n, size_t* h_bytes);
int maxent_expected_fwd_sym(int model, const double* x, const double* y, int64_t n, double* k_out, double* s_out,
                            void* workspace, size_t workspace_bytes, mh_stream_t stream);
int maxent_expected_jacobian_diag_sym(int model, const double* x, const double* y, int64_t n, double* dk_dx,
                                      double* dk_dy, double* ds_dx, double* ds_dy, void* workspace,
                                      size_t workspace_bytes, mh_stream_t stream);
int maxent_expected_bwd_sym(int model, const double* x, const double* y, int64_t n, const double* g_k,
                            const double* g_s, double* g_x, double* g_y, void* workspace, size_t workspace_bytes,
                            mh_stream_t stream);

/*
 * maxent_expected_jacobian_diag_sym_f32 / maxent_expected_bwd_sym_f32 — the
 * sums of maxent_expected_jacobian_diag_sym and maxent_expected_bwd_sym
 * (same arguments, workspace and outputs, FP64 outputs) with FP32 pair terms,
 * summed in FP32 over tiles of 32 and 64 terms and in double-float across
 * tiles: within about 1e-5 of the sum of the terms' magnitudes, for Newton
 * directions (the derivatives of Sec. 2.2 and Sec. 2.5 that an inexact
 * Newton step solves with; the residual it drives to zero keeps the
 * double-float forms).  Operands outside the double-float range (see above)
 * take FP64 terms as there.  Deterministic, as the other symmetric forms.
 */
int maxent_expected_jacobian_diag_sym_f32(int model, const double* x, const double* y, int64_t n, double* dk_dx,
                                          double* dk_dy, double* ds_dx, double* ds_dy, void* workspace,
                                          size_t workspace_bytes, mh_stream_t stream);
int maxent_expected_bwd_sym_f32(int model, const double* x, const double* y, int64_t n, const double* g_k,
                                const double* g_s, double* g_x, double* g_y, void* workspace, size_t workspace_bytes,
                                mh_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MAXENT_MH_H */
