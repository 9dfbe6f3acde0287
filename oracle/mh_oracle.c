/*
 * CPU oracle for maximum-entropy network sampling (arXiv 2509.13230).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Plain, serial, FP64, no FMA contraction (build with -ffp-contract=off).
 * Every floating-point expression below is written in the one order that
 * defines the sampled bits; the C library log/log1p are used as-is.
 *
 * Notation.  The paper parametrises nodes by alpha_i (degree) and beta_i
 * (strength).  Here x_i = exp(-alpha_i) and y_i = exp(-beta_i), so
 *   UBCM (Eq. 1):  p_ij = x_i x_j / (1 + x_i x_j)
 *   UECM (Eq. 3):  p_ij = A / (1 - r + A),  A = x_i y_i x_j y_j,  r = y_i y_j
 *   UECM (Eq. 4):  P(w | w > 0) = r^(w-1) (1 - r),  w = 1, 2, ...
 *   Bound (Eq. 5): phat_ij = A / (1 - c + A),  c >= r over the pairs proposed
 *
 * Contents
 *   orc_philox4x32_10   counter-based generator (Salmon et al., SC'11)
 *   orc_sort_desc       node order of Sec. 2.4 step (i) / Algorithm 1 sort
 *   orc_partition       row-segment table (restart of the proposal bound)
 *   orc_mh_sample       serial Miller-Hagberg walk, Sec. 2.3-2.5, Algorithm 1
 *   orc_mh_sample_segments  the same over a range of segment-table rows
 *   orc_bf_sample       brute-force Bernoulli sampler, Sec. 2.2 / Sec. 3
 *   orc_bip_partition   row-segment table of a bipartite network, Sec. 2.6
 *   orc_bip_sample      serial walk of bipartite and directed networks, Sec. 2.6
 *   orc_bip_bf_sample   brute-force sampler of bipartite and directed networks
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_UBCM 0
#define ORC_UECM 1
#define ORC_CL 2 /* Chung-Lu: p_ij = min(1, x_i x_j), Sec. 2.1 and the MH algorithm of Sec. 2.3 */

/* flags */
#define ORC_BOUND_PAPER 0x1u /* c = product of the two largest y among ranks >= i */
#define ORC_INIT_PREV 0x2u   /* first q taken at the position before the segment head */

/* stats slots */
#define ORC_ST_DRAWS 0
#define ORC_ST_EDGES 1
#define ORC_ST_SEGMENTS 2
#define ORC_ST_BOUNDARY 3

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds of a multiply/xor bijection on a    */
/* 128-bit counter, with a Weyl sequence on the 64-bit key between rounds.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t prod0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* 53 random bits -> (0, 1]: the skip and weight draws take a log of it. */
static double unit_open0(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((((uint64_t)hi) << 32) | lo) >> 11;
    return (double)(m + 1u) * 0x1p-53;
}

/* 53 random bits -> [0, 1): the acceptance draw is compared with p/q. */
static double unit_open1(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((((uint64_t)hi) << 32) | lo) >> 11;
    return (double)m * 0x1p-53;
}

/* A draw lands on an integer boundary when it is within 8 ulp of one.  The
 * CUDA and C library logarithms may differ there by an ulp or two, so these
 * draws are counted (they are the only ones allowed to decide differently).
 * A skip draw counts only when the integer is one that decides the
 * candidate, m in [1, b - pos - 1]: beyond that every t ends the segment. */
static int near_integer(double t)
{
    if (!(t >= 0.5) || !isfinite(t)) return 0;
    double m = nearbyint(t);
    double ulp = nextafter(t, INFINITY) - t;
    return fabs(t - m) <= 8.0 * ulp;
}

/* Optional log of the boundary draws, for tests that trace a difference
 * between two samplers to the segment it came from.  Entry: sample, row
 * rank i, segment k, kind (0 skip draw, 1 weight draw), draw or edge index. */
static uint32_t* boundary_log = NULL;
static int64_t boundary_log_cap = 0, boundary_log_len = 0;

void orc_boundary_log(uint32_t* buf, int64_t cap_entries)
{
    boundary_log = buf;
    boundary_log_cap = buf ? cap_entries : 0;
    boundary_log_len = 0;
}

int64_t orc_boundary_log_len(void) { return boundary_log_len; }

static void boundary_hit(uint64_t* stats, uint32_t sample, int64_t i, int32_t k, uint32_t kind, uint32_t index)
{
    stats[ORC_ST_BOUNDARY] += 1;
    if (boundary_log_len < boundary_log_cap) {
        uint32_t* e = boundary_log + 5 * boundary_log_len;
        e[0] = sample;
        e[1] = (uint32_t)i;
        e[2] = (uint32_t)k;
        e[3] = kind;
        e[4] = index;
    }
    boundary_log_len += 1;
}

/* ------------------------------------------------------------------------ */
/* Node order (Sec. 2.4 step (i); Algorithm 1, sort by alpha + beta).        */
/* Ascending alpha == descending x; ascending alpha+beta == descending x*y.  */
/* Stable: equal keys keep ascending original id.                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double key;
    int32_t id;
} keyed_node;

static int cmp_desc(const void* pa, const void* pb)
{
    const keyed_node* a = (const keyed_node*)pa;
    const keyed_node* b = (const keyed_node*)pb;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* key[i] -> perm[rank] = original id, ranks in descending key order. */
void orc_sort_desc(const double* key, int64_t n, int32_t* perm)
{
    keyed_node* tmp = (keyed_node*)malloc(sizeof(keyed_node) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        tmp[i].key = key[i];
        tmp[i].id = (int32_t)i;
    }
    qsort(tmp, (size_t)n, sizeof(keyed_node), cmp_desc);
    for (int64_t i = 0; i < n; ++i) perm[i] = tmp[i].id;
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* One network in sorted order.                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int model;
    int64_t n;
    uint32_t flags;
    int32_t* perm;   /* rank -> original id                                 */
    double* xs;      /* x in rank order                                     */
    double* ys;      /* y in rank order (UECM)                              */
    double* as;      /* a = x*y in rank order (UECM sort key)               */
    double* ymax;    /* ymax[a] = max_{j >= a} ys[j]                        */
    double* top1;    /* largest y among ranks >= i                          */
    double* top2;    /* second largest y among ranks >= i                   */
} net_t;

static void net_free(net_t* g)
{
    free(g->perm);
    free(g->xs);
    free(g->ys);
    free(g->as);
    free(g->ymax);
    free(g->top1);
    free(g->top2);
}

static void net_build(net_t* g, int model, const double* x, const double* y, int64_t n, uint32_t flags)
{
    size_t cnt = (size_t)(n > 0 ? n : 1);
    memset(g, 0, sizeof(*g));
    g->model = model;
    g->n = n;
    g->flags = flags;
    g->perm = (int32_t*)malloc(sizeof(int32_t) * cnt);
    g->xs = (double*)malloc(sizeof(double) * cnt);
    g->ys = (double*)malloc(sizeof(double) * cnt);
    g->as = (double*)malloc(sizeof(double) * cnt);
    g->ymax = (double*)malloc(sizeof(double) * (cnt + 1));
    g->top1 = (double*)malloc(sizeof(double) * (cnt + 1));
    g->top2 = (double*)malloc(sizeof(double) * (cnt + 1));

    double* key = (double*)malloc(sizeof(double) * cnt);
    for (int64_t u = 0; u < n; ++u) key[u] = (model != ORC_UECM) ? x[u] : x[u] * y[u];
    orc_sort_desc(key, n, g->perm);
    free(key);

    for (int64_t i = 0; i < n; ++i) {
        int32_t u = g->perm[i];
        g->xs[i] = x[u];
        g->ys[i] = (model == ORC_UECM) ? y[u] : 0.0;
        g->as[i] = (model == ORC_UECM) ? x[u] * y[u] : x[u];
    }
    /* Suffix bounds on y over the ranks not processed yet (Sec. 2.5). */
    g->ymax[n] = 0.0;
    g->top1[n] = 0.0;
    g->top2[n] = 0.0;
    for (int64_t i = n - 1; i >= 0; --i) {
        double v = g->ys[i];
        g->ymax[i] = (v > g->ymax[i + 1]) ? v : g->ymax[i + 1];
        if (v > g->top1[i + 1]) {
            g->top1[i] = v;
            g->top2[i] = g->top1[i + 1];
        } else {
            g->top1[i] = g->top1[i + 1];
            g->top2[i] = (v > g->top2[i + 1]) ? v : g->top2[i + 1];
        }
    }
}

/* Edge probability (Eq. 1 / Eq. 3) between ranks i and j. */
static double prob(const net_t* g, int64_t i, int64_t j)
{
    if (g->model == ORC_UBCM) {
        double z = g->xs[i] * g->xs[j];
        return z / (1.0 + z);
    }
    if (g->model == ORC_CL) {
        double z = g->xs[i] * g->xs[j];
        return z >= 1.0 ? 1.0 : z;
    }
    double A = g->as[i] * g->as[j];
    double r = g->ys[i] * g->ys[j];
    return A / ((1.0 - r) + A);
}

/* Upper bound (Eq. 5) with the constant c = exp(-beta_min). */
static double prob_hat(const net_t* g, int64_t i, int64_t j, double c)
{
    double A = g->as[i] * g->as[j];
    return A / ((1.0 - c) + A);
}

/* exp(-beta_min) for a segment of row i starting at rank a.  The paper takes
 * the two largest y among unprocessed nodes (Sec. 2.5); the default takes
 * y_i times the largest y from the segment head on, which is also >= r_ij for
 * every candidate j >= a and never larger. */
static double bound_c(const net_t* g, int64_t i, int64_t a)
{
    if (g->flags & ORC_BOUND_PAPER) return g->top1[i] * g->top2[i];
    return g->ys[i] * g->ymax[a];
}

/* ------------------------------------------------------------------------ */
/* Row-segment table.  Row i's candidates [i+1, n) are cut into segments     */
/* [a, b) of about T expected proposals each.  The proposal bound q restarts */
/* at every segment head, which keeps the walk exact (q only has to bound    */
/* p over the candidates it proposes).  The cut points come from a monotone  */
/* cost function evaluated with a fixed sequence of IEEE operations and      */
/* integer prefix sums, so they are reproducible bit for bit.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int F;               /* fixed-point fraction bits of the prefix sums   */
    uint64_t* Q;         /* Q[j] = sum_{l<j} floor(min(v_l, 2^20) * 2^F)   */
} proxy_t;

static int bitlen_u64(uint64_t v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

static void proxy_build(proxy_t* P, const net_t* g)
{
    int64_t n = g->n;
    const double* v = (g->model != ORC_UECM) ? g->xs : g->as;
    double vmax = (n > 0) ? v[0] : 0.0;
    if (vmax > 0x1p20) vmax = 0x1p20;
    uint64_t bits;
    memcpy(&bits, &vmax, sizeof(bits));
    int E = (int)((bits >> 52) & 0x7FF) - 1022; /* vmax = m 2^E, m in [0.5, 1) */
    if (E < 1) E = 1;
    int F = 62 - bitlen_u64((uint64_t)n) - E;
    if (F < 0) F = 0;
    P->F = F;
    P->Q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    P->Q[0] = 0;
    for (int64_t j = 0; j < n; ++j) {
        double vj = v[j] > 0x1p20 ? 0x1p20 : v[j];
        P->Q[j + 1] = P->Q[j] + (uint64_t)ldexp(vj, F);
    }
}

/* Per-row weight w_i: the cost of candidate j is min(1, w_i v_j). */
static double row_weight(const net_t* g, int64_t i)
{
    if (g->model != ORC_UECM) return g->xs[i];
    double c;
    if (g->flags & ORC_BOUND_PAPER)
        c = g->top1[i] * g->top2[i];
    else
        c = g->ys[i] * g->ymax[i + 1];
    return g->as[i] / (1.0 - c);
}

/* First j in [i+1, n) with w v_j < 1, else n (products are non-increasing). */
static int64_t unit_cut(const net_t* g, int64_t i, double w)
{
    const double* v = (g->model != ORC_UECM) ? g->xs : g->as;
    int64_t lo = i + 1, hi = g->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (w * v[mid] < 1.0)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* Per-row weight in fixed point: floor(w * 2^40), saturated at 2^64 - 1. */
static uint64_t weight_fixed(double w)
{
    double wq = ldexp(w, 40);
    if (!(wq < 0x1p64)) return UINT64_MAX;
    return (uint64_t)wq;
}

/* Cumulative cost of candidates [i+1, b) in units of 2^-F.  The first part
 * counts candidates with w v_j >= 1 as one proposal each; the rest is
 * floor(qw (Q[b] - Q[J]) / 2^40), an exact 128-bit product.  Each candidate
 * adds at most 2^F + 1, so cut points at multiples of Tc >= 2^(F+1) are
 * strictly increasing. */
static uint64_t row_cost(const proxy_t* P, int64_t i, int64_t J, uint64_t qw, int64_t b)
{
    int64_t units = (b < J ? b : J) - (i + 1);
    uint64_t c = (uint64_t)units << P->F;
    if (b > J) {
        unsigned __int128 prod = (unsigned __int128)qw * (unsigned __int128)(P->Q[b] - P->Q[J]);
        c += (uint64_t)(prod >> 40);
    }
    return c;
}

/* Segments of row i: writes up to `cap` entries, returns the count.
 * nseg = max(1, floor(total / 2^F) / T); cut k (k = 1 .. nseg-1) is the first
 * b with cost(b) >= k * floor(total / nseg).  Requires T >= 2. */
static int64_t row_segments(const net_t* g, const proxy_t* P, int64_t i, int64_t T, int64_t* seg_a,
                            int64_t* seg_b, int64_t cap)
{
    int64_t n = g->n;
    if (i + 1 >= n) return 0;
    double w = row_weight(g, i);
    int64_t J = unit_cut(g, i, w);
    uint64_t qw = weight_fixed(w);
    uint64_t total = row_cost(P, i, J, qw, n);
    uint64_t nseg = (total >> P->F) / (uint64_t)T;
    if (nseg < 1) nseg = 1;
    uint64_t Tc = total / nseg;
    int64_t prev = i + 1;
    for (uint64_t k = 0; k < nseg; ++k) {
        int64_t b = n;
        if (k + 1 < nseg) {
            uint64_t target = Tc * (k + 1);
            int64_t lo = i + 2, hi = n; /* first b with cost >= target */
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (row_cost(P, i, J, qw, mid) >= target)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            b = lo;
        }
        if ((int64_t)k < cap) {
            seg_a[k] = prev;
            seg_b[k] = b;
        }
        prev = b;
    }
    return (int64_t)nseg;
}

/* Whole table in canonical (row, k) order.  Returns the segment count; when
 * it exceeds `cap` only the first `cap` entries are written. */
int64_t orc_partition(int model, const double* x, const double* y, int64_t n, int64_t T, uint32_t flags,
                      int32_t* seg_row, int32_t* seg_k, int64_t* seg_a, int64_t* seg_b, int64_t cap,
                      int32_t* perm_out)
{
    net_t g;
    proxy_t P;
    net_build(&g, model, x, y, n, flags);
    proxy_build(&P, &g);
    if (perm_out) memcpy(perm_out, g.perm, sizeof(int32_t) * (size_t)n);
    int64_t total = 0;
    int64_t* ta = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i + 1 < n; ++i) {
        int64_t ns = row_segments(&g, &P, i, T, ta, tb, n);
        for (int64_t k = 0; k < ns; ++k, ++total) {
            if (total < cap) {
                seg_row[total] = (int32_t)i;
                seg_k[total] = (int32_t)k;
                seg_a[total] = ta[k];
                seg_b[total] = tb[k];
            }
        }
    }
    free(ta);
    free(tb);
    free(P.Q);
    net_free(&g);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Serial Miller-Hagberg walk over one segment (Sec. 2.3, Sec. 2.4 steps     */
/* (ii)-(iv), Algorithm 1).                                                  */
/*                                                                           */
/*  q    proposal probability; bounds p_ij for every candidate still ahead  */
/*  L    skip to the next candidate, Geometric(q) on {1, 2, ...} (Fig. 2):   */
/*       L = 1 + floor(t), t = ln U / ln(1 - q), U uniform on (0, 1]         */
/*  V    acceptance draw on [0, 1): candidate j is kept when V < p_ij / q    */
/*  q <- p_ij (UBCM, Sec. 2.4 step (iii)) or phat_ij (UECM, Algorithm 1)     */
/*  w    UECM weight given an edge, Geometric(1 - r) on {1, 2, ...} (Eq. 4)  */
/*       w = 1 + floor(ln U_w / ln r)                                        */
/*                                                                           */
/* Random words: candidate d of segment k of row i in sample s uses          */
/* Philox(ctr = {d, k, i, s}); U from words (1,0), V from words (3,2).       */
/* Edge e of that segment takes its weight from ctr = {2^31 | e/2, k, i, s}, */
/* words (1,0) for even e and (3,2) for odd e.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t* src;
    int32_t* dst;
    int32_t* w;
    int64_t cap;
    int64_t count;
    uint64_t* stats;
    int weight_overflow;
} sink_t;

static void walk_segment(const net_t* g, const uint32_t key[2], uint32_t sample, int64_t i, int32_t k,
                         int64_t a, int64_t b, sink_t* out)
{
    const int uecm = (g->model == ORC_UECM);
    const double c = uecm ? bound_c(g, i, a) : 0.0;
    int64_t head = (g->flags & ORC_INIT_PREV) ? a - 1 : a;
    double q = uecm ? prob_hat(g, i, head, c) : prob(g, i, head);
    int64_t pos = a - 1;
    uint32_t d = 0, e = 0;
    out->stats[ORC_ST_SEGMENTS] += 1;
    for (;;) {
        if (!(q > 0.0)) break;
        uint32_t ctr[4] = {d, (uint32_t)k, (uint32_t)i, sample};
        uint32_t rnd[4];
        orc_philox4x32_10(ctr, key, rnd);
        d += 1;
        out->stats[ORC_ST_DRAWS] += 1;
        double U = unit_open0(rnd[1], rnd[0]);
        double V = unit_open1(rnd[3], rnd[2]);
        double R = (double)(b - pos - 1);
        double t = (q >= 1.0) ? 0.0 : log(U) / log1p(-q);
        if (near_integer(t) && nearbyint(t) <= R) boundary_hit(out->stats, sample, i, k, 0, d - 1);
        if (t >= R) break;
        int64_t j = pos + 1 + (int64_t)floor(t);
        double p = prob(g, i, j);
        if (V < p / q) {
            int32_t wt = 1;
            if (uecm) {
                uint32_t wctr[4] = {0x80000000u | (e >> 1), (uint32_t)k, (uint32_t)i, sample};
                uint32_t wr[4];
                orc_philox4x32_10(wctr, key, wr);
                double Uw = (e & 1u) ? unit_open0(wr[3], wr[2]) : unit_open0(wr[1], wr[0]);
                double r = g->ys[i] * g->ys[j];
                if (r > 0.0) {
                    double tw = log(Uw) / log(r);
                    if (near_integer(tw)) boundary_hit(out->stats, sample, i, k, 1, e);
                    if (tw >= 2147483646.0) {
                        wt = 2147483647;
                        out->weight_overflow = 1;
                    } else {
                        wt = 1 + (int32_t)floor(tw);
                    }
                }
            }
            if (out->count < out->cap) {
                out->src[out->count] = g->perm[i];
                out->dst[out->count] = g->perm[j];
                if (out->w) out->w[out->count] = wt;
            }
            out->count += 1;
            out->stats[ORC_ST_EDGES] += 1;
            e += 1;
        }
        q = uecm ? prob_hat(g, i, j, c) : p;
        pos = j;
    }
}

/* Samples [sample_begin, sample_begin + num_samples) of one network.  Edges
 * of all samples are concatenated in sample order, each sample in canonical
 * (row rank, segment, candidate) order; counts[s] receives the edge count of
 * sample s.  Returns the total edge count (which may exceed cap: then only
 * the first cap edges are written), or -1 on a weight above INT32_MAX. */
int64_t orc_mh_sample(int model, const double* x, const double* y, int64_t n, uint64_t seed, uint32_t network_id,
                      uint32_t sample_begin, uint32_t num_samples, int64_t T, uint32_t flags, int32_t* src,
                      int32_t* dst, int32_t* w, int64_t cap, int64_t* counts, uint64_t* stats)
{
    net_t g;
    proxy_t P;
    net_build(&g, model, x, y, n, flags);
    proxy_build(&P, &g);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) + network_id};
    uint64_t local_stats[4] = {0, 0, 0, 0};
    sink_t out = {src, dst, w, cap, 0, stats ? stats : local_stats, 0};
    int64_t* ta = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (uint32_t s = 0; s < num_samples; ++s) {
        int64_t before = out.count;
        for (int64_t i = 0; i + 1 < n; ++i) {
            int64_t ns = row_segments(&g, &P, i, T, ta, tb, n);
            for (int64_t kk = 0; kk < ns; ++kk)
                walk_segment(&g, key, sample_begin + s, i, (int32_t)kk, ta[kk], tb[kk], &out);
        }
        if (counts) counts[s] = out.count - before;
    }
    free(ta);
    free(tb);
    free(P.Q);
    net_free(&g);
    return out.weight_overflow ? -1 : out.count;
}

/* The same samples restricted to rows [seg_begin, seg_end) of the segment
 * table (canonical (row, k) order): the share of one sample that a rank draws
 * when the table is split into contiguous ranges.  The walk of a segment
 * depends only on the segment and the sample, so the ranges' edge lists,
 * concatenated in range order, are the whole sample's.  counts[s] receives
 * the edges of sample s within the range. */
int64_t orc_mh_sample_segments(int model, const double* x, const double* y, int64_t n, uint64_t seed,
                               uint32_t network_id, uint32_t sample_begin, uint32_t num_samples, int64_t T,
                               uint32_t flags, int64_t seg_begin, int64_t seg_end, int32_t* src, int32_t* dst,
                               int32_t* w, int64_t cap, int64_t* counts, uint64_t* stats)
{
    net_t g;
    proxy_t P;
    net_build(&g, model, x, y, n, flags);
    proxy_build(&P, &g);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) + network_id};
    uint64_t local_stats[4] = {0, 0, 0, 0};
    sink_t out = {src, dst, w, cap, 0, stats ? stats : local_stats, 0};
    int64_t* ta = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (uint32_t s = 0; s < num_samples; ++s) {
        int64_t before = out.count;
        int64_t row_of_table = 0; /* index of the table row of (i, kk) */
        for (int64_t i = 0; i + 1 < n && row_of_table < seg_end; ++i) {
            int64_t ns = row_segments(&g, &P, i, T, ta, tb, n);
            for (int64_t kk = 0; kk < ns; ++kk, ++row_of_table)
                if (row_of_table >= seg_begin && row_of_table < seg_end)
                    walk_segment(&g, key, sample_begin + s, i, (int32_t)kk, ta[kk], tb[kk], &out);
        }
        if (counts) counts[s] = out.count - before;
    }
    free(ta);
    free(tb);
    free(P.Q);
    net_free(&g);
    return out.weight_overflow ? -1 : out.count;
}

/* ------------------------------------------------------------------------ */
/* Brute force (Sec. 2.2; the BF baseline of Sec. 3): every pair u < v of    */
/* original ids is an independent Bernoulli(p_uv); a UECM edge then draws    */
/* w ~ Geometric(1 - r_uv) on {1, 2, ...} (Eqs. 2-4).  Random words come     */
/* from Philox(ctr = {u, v, 0xB0F0B0F0, s}): words (1,0) give the [0, 1)     */
/* Bernoulli draw, words (3,2) the (0, 1] weight draw.  Agrees with the      */
/* walk in distribution, not in bits.                                        */
/* ------------------------------------------------------------------------ */
int64_t orc_bf_sample(int model, const double* x, const double* y, int64_t n, uint64_t seed, uint32_t sample,
                      int32_t* src, int32_t* dst, int32_t* w, int64_t cap, uint64_t* evaluations)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t count = 0;
    uint64_t evals = 0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t v = u + 1; v < n; ++v) {
            double p, r = 0.0;
            if (model == ORC_UBCM) {
                double z = x[u] * x[v];
                p = z / (1.0 + z);
            } else if (model == ORC_CL) {
                double z = x[u] * x[v];
                p = z >= 1.0 ? 1.0 : z;
            } else {
                double A = (x[u] * y[u]) * (x[v] * y[v]);
                r = y[u] * y[v];
                p = A / ((1.0 - r) + A);
            }
            evals += 1;
            uint32_t ctr[4] = {(uint32_t)u, (uint32_t)v, 0xB0F0B0F0u, sample};
            uint32_t rnd[4];
            orc_philox4x32_10(ctr, key, rnd);
            double V = unit_open1(rnd[1], rnd[0]);
            if (V < p) {
                int32_t wt = 1;
                if (model == ORC_UECM && r > 0.0) {
                    double Uw = unit_open0(rnd[3], rnd[2]);
                    double tw = log(Uw) / log(r);
                    wt = (tw >= 2147483646.0) ? 2147483647 : 1 + (int32_t)floor(tw);
                }
                if (count < cap) {
                    src[count] = (int32_t)u;
                    dst[count] = (int32_t)v;
                    if (w) w[count] = wt;
                }
                count += 1;
            }
        }
    }
    if (evaluations) *evaluations = evals;
    return count;
}

/* ------------------------------------------------------------------------ */
/* Bipartite and directed networks (Sec. 2.6).  The rows are the nodes of    */
/* the + set, each walked over all nodes of the - set; each set is sorted by */
/* its own key (descending x, or a = x*y for the UECM form), so p_ij is      */
/* non-increasing along a row and the same geometric skipping applies:       */
/*   UBCM form  p_ij = x+_i x-_j / (1 + x+_i x-_j)                           */
/*   UECM form  p_ij = A / (1 - r + A),  A = a+_i a-_j,  r = y+_i y-_j        */
/*   bound c of a segment [a, b) of row i: y+_i max_{j >= a} y-_j (>= r_ij)  */
/* A directed network is the bipartite one with the out-parameters of every  */
/* node as the + set and its in-parameters as the - set (the same ids), and  */
/* without the pairs (i, i): the walk of row i skips the - rank e_i of node  */
/* i.  Candidates are then counted in "virtual" positions that leave e_i     */
/* out: virtual v is - rank v for v < e_i and v + 1 from e_i on; p stays     */
/* non-increasing along virtual positions.  The segment table is the        */
/* bipartite one in - ranks (a segment that holds only e_i has no candidate).*/
/* Random words as in the one-set walk, with i the + rank of the row.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    net_t R;         /* + set (rows)                                        */
    net_t C;         /* - set (candidates)                                  */
    int32_t* rank_c; /* - id -> - rank                                      */
    int directed;
} bip_t;

static void bip_build(bip_t* B, int model, const double* xp, const double* yp, int64_t np, const double* xm,
                      const double* ym, int64_t nm, int directed)
{
    net_build(&B->R, model, xp, yp, np, 0u);
    net_build(&B->C, model, xm, ym, nm, 0u);
    B->directed = directed;
    B->rank_c = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nm > 0 ? nm : 1));
    for (int64_t j = 0; j < nm; ++j) B->rank_c[B->C.perm[j]] = (int32_t)j;
}

static void bip_free(bip_t* B)
{
    net_free(&B->R);
    net_free(&B->C);
    free(B->rank_c);
}

static double bip_prob(const bip_t* B, int64_t i, int64_t j)
{
    if (B->R.model == ORC_UBCM) {
        double z = B->R.xs[i] * B->C.xs[j];
        return z / (1.0 + z);
    }
    double A = B->R.as[i] * B->C.as[j];
    double r = B->R.ys[i] * B->C.ys[j];
    return A / ((1.0 - r) + A);
}

static double bip_prob_hat(const bip_t* B, int64_t i, int64_t j, double c)
{
    double A = B->R.as[i] * B->C.as[j];
    return A / ((1.0 - c) + A);
}

static double bip_bound_c(const bip_t* B, int64_t i, int64_t a)
{
    return B->R.ys[i] * B->C.ymax[a];
}

/* Cost weight of row i over the whole - set (bound at a = 0). */
static double bip_row_weight(const bip_t* B, int64_t i)
{
    if (B->R.model == ORC_UBCM) return B->R.xs[i];
    return B->R.as[i] / (1.0 - bip_bound_c(B, i, 0));
}

/* First - rank j with w v_j < 1, else m. */
static int64_t bip_unit_cut(const bip_t* B, double w)
{
    const double* v = (B->C.model == ORC_UBCM) ? B->C.xs : B->C.as;
    int64_t lo = 0, hi = B->C.n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (w * v[mid] < 1.0)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* Cumulative cost of - ranks [0, b), as row_cost with the row starting at 0. */
static uint64_t bip_row_cost(const proxy_t* P, int64_t J, uint64_t qw, int64_t b)
{
    int64_t units = (b < J ? b : J);
    uint64_t c = (uint64_t)units << P->F;
    if (b > J) {
        unsigned __int128 prod = (unsigned __int128)qw * (unsigned __int128)(P->Q[b] - P->Q[J]);
        c += (uint64_t)(prod >> 40);
    }
    return c;
}

/* Segments of row i over - ranks [0, m), as row_segments. */
static int64_t bip_row_segments(const bip_t* B, const proxy_t* P, int64_t i, int64_t T, int64_t* seg_a,
                                int64_t* seg_b, int64_t cap)
{
    int64_t m = B->C.n;
    if (m < 1) return 0;
    double w = bip_row_weight(B, i);
    int64_t J = bip_unit_cut(B, w);
    uint64_t qw = weight_fixed(w);
    uint64_t total = bip_row_cost(P, J, qw, m);
    uint64_t nseg = (total >> P->F) / (uint64_t)T;
    if (nseg < 1) nseg = 1;
    uint64_t Tc = total / nseg;
    int64_t prev = 0;
    for (uint64_t k = 0; k < nseg; ++k) {
        int64_t b = m;
        if (k + 1 < nseg) {
            uint64_t target = Tc * (k + 1);
            int64_t lo = 1, hi = m; /* first b with cost >= target */
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (bip_row_cost(P, J, qw, mid) >= target)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            b = lo;
        }
        if ((int64_t)k < cap) {
            seg_a[k] = prev;
            seg_b[k] = b;
        }
        prev = b;
    }
    return (int64_t)nseg;
}

/* Whole bipartite table in (+ rank, k) order; segment bounds are - ranks. */
int64_t orc_bip_partition(int model, const double* xp, const double* yp, int64_t np, const double* xm,
                          const double* ym, int64_t nm, int64_t T, int32_t* seg_row, int32_t* seg_k,
                          int64_t* seg_a, int64_t* seg_b, int64_t cap, int32_t* perm_plus, int32_t* perm_minus)
{
    bip_t B;
    proxy_t P;
    bip_build(&B, model, xp, yp, np, xm, ym, nm, 0);
    proxy_build(&P, &B.C);
    if (perm_plus) memcpy(perm_plus, B.R.perm, sizeof(int32_t) * (size_t)np);
    if (perm_minus) memcpy(perm_minus, B.C.perm, sizeof(int32_t) * (size_t)nm);
    int64_t total = 0;
    int64_t* ta = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm > 0 ? nm : 1));
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm > 0 ? nm : 1));
    for (int64_t i = 0; i < np; ++i) {
        int64_t ns = bip_row_segments(&B, &P, i, T, ta, tb, nm);
        for (int64_t k = 0; k < ns; ++k, ++total) {
            if (total < cap) {
                seg_row[total] = (int32_t)i;
                seg_k[total] = (int32_t)k;
                seg_a[total] = ta[k];
                seg_b[total] = tb[k];
            }
        }
    }
    free(ta);
    free(tb);
    free(P.Q);
    bip_free(&B);
    return total;
}

/* - rank of virtual position v of a row whose excluded - rank is ex (-1: none). */
static int64_t bip_actual(int64_t v, int64_t ex)
{
    return (ex >= 0 && v >= ex) ? v + 1 : v;
}

static void bip_walk_segment(const bip_t* B, const uint32_t key[2], uint32_t sample, int64_t i, int32_t k,
                             int64_t a, int64_t b, int64_t ex, sink_t* out)
{
    const int uecm = (B->R.model == ORC_UECM);
    const int64_t va = (ex >= 0 && a > ex) ? a - 1 : a;
    const int64_t vb = (ex >= 0 && b > ex) ? b - 1 : b;
    out->stats[ORC_ST_SEGMENTS] += 1;
    if (va >= vb) return; /* the segment holds only the excluded candidate */
    const double c = uecm ? bip_bound_c(B, i, a) : 0.0;
    int64_t head = bip_actual(va, ex);
    double q = uecm ? bip_prob_hat(B, i, head, c) : bip_prob(B, i, head);
    int64_t pos = va - 1;
    uint32_t d = 0, e = 0;
    for (;;) {
        if (!(q > 0.0)) break;
        uint32_t ctr[4] = {d, (uint32_t)k, (uint32_t)i, sample};
        uint32_t rnd[4];
        orc_philox4x32_10(ctr, key, rnd);
        d += 1;
        out->stats[ORC_ST_DRAWS] += 1;
        double U = unit_open0(rnd[1], rnd[0]);
        double V = unit_open1(rnd[3], rnd[2]);
        double R = (double)(vb - pos - 1);
        double t = (q >= 1.0) ? 0.0 : log(U) / log1p(-q);
        if (near_integer(t) && nearbyint(t) <= R) boundary_hit(out->stats, sample, i, k, 0, d - 1);
        if (t >= R) break;
        int64_t jv = pos + 1 + (int64_t)floor(t);
        int64_t j = bip_actual(jv, ex);
        double p = bip_prob(B, i, j);
        if (V < p / q) {
            int32_t wt = 1;
            if (uecm) {
                uint32_t wctr[4] = {0x80000000u | (e >> 1), (uint32_t)k, (uint32_t)i, sample};
                uint32_t wr[4];
                orc_philox4x32_10(wctr, key, wr);
                double Uw = (e & 1u) ? unit_open0(wr[3], wr[2]) : unit_open0(wr[1], wr[0]);
                double r = B->R.ys[i] * B->C.ys[j];
                if (r > 0.0) {
                    double tw = log(Uw) / log(r);
                    if (near_integer(tw)) boundary_hit(out->stats, sample, i, k, 1, e);
                    if (tw >= 2147483646.0) {
                        wt = 2147483647;
                        out->weight_overflow = 1;
                    } else {
                        wt = 1 + (int32_t)floor(tw);
                    }
                }
            }
            if (out->count < out->cap) {
                out->src[out->count] = B->R.perm[i];
                out->dst[out->count] = B->C.perm[j];
                if (out->w) out->w[out->count] = wt;
            }
            out->count += 1;
            out->stats[ORC_ST_EDGES] += 1;
            e += 1;
        }
        q = uecm ? bip_prob_hat(B, i, j, c) : p;
        pos = jv;
    }
}

/* Samples of a bipartite (directed = 0) or directed (directed = 1, np == nm)
 * network.  Edges (+ id, - id) of all samples concatenated in sample order,
 * each sample in (+ rank, segment, candidate) order.  Returns the total
 * edge count, or -1 on a weight above INT32_MAX or np != nm when directed. */
int64_t orc_bip_sample(int model, const double* xp, const double* yp, int64_t np, const double* xm,
                       const double* ym, int64_t nm, int directed, uint64_t seed, uint32_t network_id,
                       uint32_t sample_begin, uint32_t num_samples, int64_t T, int32_t* src, int32_t* dst,
                       int32_t* w, int64_t cap, int64_t* counts, uint64_t* stats)
{
    if (directed && np != nm) return -1;
    bip_t B;
    proxy_t P;
    bip_build(&B, model, xp, yp, np, xm, ym, nm, directed);
    proxy_build(&P, &B.C);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) + network_id};
    uint64_t local_stats[4] = {0, 0, 0, 0};
    sink_t out = {src, dst, w, cap, 0, stats ? stats : local_stats, 0};
    int64_t* ta = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm > 0 ? nm : 1));
    int64_t* tb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nm > 0 ? nm : 1));
    for (uint32_t s = 0; s < num_samples; ++s) {
        int64_t before = out.count;
        for (int64_t i = 0; i < np; ++i) {
            int64_t ex = directed ? (int64_t)B.rank_c[B.R.perm[i]] : -1;
            int64_t ns = bip_row_segments(&B, &P, i, T, ta, tb, nm);
            for (int64_t kk = 0; kk < ns; ++kk)
                bip_walk_segment(&B, key, sample_begin + s, i, (int32_t)kk, ta[kk], tb[kk], ex, &out);
        }
        if (counts) counts[s] = out.count - before;
    }
    free(ta);
    free(tb);
    free(P.Q);
    bip_free(&B);
    return out.weight_overflow ? -1 : out.count;
}

/* Brute force for bipartite / directed networks: every pair (u, v), u a +
 * id and v a - id (u != v when directed), is an independent Bernoulli(p_uv)
 * with a UECM weight as in orc_bf_sample; Philox(ctr = {u, v, 0xB1B1B1B1,
 * s}).  Edges in (u, v) order. */
int64_t orc_bip_bf_sample(int model, const double* xp, const double* yp, int64_t np, const double* xm,
                          const double* ym, int64_t nm, int directed, uint64_t seed, uint32_t sample,
                          int32_t* src, int32_t* dst, int32_t* w, int64_t cap, uint64_t* evaluations)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t count = 0;
    uint64_t evals = 0;
    for (int64_t u = 0; u < np; ++u) {
        for (int64_t v = 0; v < nm; ++v) {
            if (directed && u == v) continue;
            double p, r = 0.0;
            if (model == ORC_UBCM) {
                double z = xp[u] * xm[v];
                p = z / (1.0 + z);
            } else {
                double A = (xp[u] * yp[u]) * (xm[v] * ym[v]);
                r = yp[u] * ym[v];
                p = A / ((1.0 - r) + A);
            }
            evals += 1;
            uint32_t ctr[4] = {(uint32_t)u, (uint32_t)v, 0xB1B1B1B1u, sample};
            uint32_t rnd[4];
            orc_philox4x32_10(ctr, key, rnd);
            double V = unit_open1(rnd[1], rnd[0]);
            if (V < p) {
                int32_t wt = 1;
                if (model == ORC_UECM && r > 0.0) {
                    double Uw = unit_open0(rnd[3], rnd[2]);
                    double tw = log(Uw) / log(r);
                    wt = (tw >= 2147483646.0) ? 2147483647 : 1 + (int32_t)floor(tw);
                }
                if (count < cap) {
                    src[count] = (int32_t)u;
                    dst[count] = (int32_t)v;
                    if (w) w[count] = wt;
                }
                count += 1;
            }
        }
    }
    if (evaluations) *evaluations = evals;
    return count;
}
