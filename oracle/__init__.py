"""CPU oracle for maximum-entropy network sampling (arXiv 2509.13230).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the library under
``paper_2509_13230_gb300`` never does, and the two share no code.

Everything here is plain and slow on purpose:

* ``mh_sample`` / ``bf_sample`` / ``partition`` / ``philox`` call the serial C
  file ``mh_oracle.c`` (FP64, no FMA contraction, C library ``log``/``log1p``).
* ``expected_fwd`` / ``expected_bwd`` / ``expected_jacobian_diag``
  evaluate the O(N^2) sums of the maximum-likelihood conditions (Sec. 2.2,
  Sec. 2.5, Sec. 4), their gradient and the diagonal of their Jacobian pair
  by pair in FP64 with correctly rounded summation (``math.fsum``).
* ``graph_probabilities`` enumerates every simple graph of a tiny network
  and multiplies the independent pair probabilities (Eq. 1 / Eq. 3).
* ``symmetric_csr`` lists every sampled edge in both endpoint rows, in the
  sample's edge order.
* ``bip_*`` are the same for bipartite and directed networks (Sec. 2.6): the
  rows are the + set, the candidates the - set; a directed network uses the
  out-parameters as the + set and the in-parameters as the - set, without
  the pairs (i, i).

Notation: x_i = exp(-alpha_i), y_i = exp(-beta_i) (the paper's alpha, beta).
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading

import numpy as np

UBCM = 0
UECM = 1
CL = 2  # Chung-Lu: p_ij = min(1, x_i x_j) (Sec. 2.1; the Miller-Hagberg original, Sec. 2.3)
BOUND_PAPER = 0x1
INIT_PREV = 0x2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None


def build(extra_flags: tuple[str, ...] = (), name: str = "libmh_oracle.so") -> str:
    """Compile the C oracle (gcc, -O2, no FP contraction) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, name)
    if (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               *extra_flags, "-o", out + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)
    return out


def _declare(lib):
    i64, u64, u32, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    vp = ctypes.c_void_p
    lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
    lib.orc_philox4x32_10.restype = None
    lib.orc_sort_desc.argtypes = [vp, i64, vp]
    lib.orc_sort_desc.restype = None
    lib.orc_partition.argtypes = [i32, vp, vp, i64, i64, u32, vp, vp, vp, vp, i64, vp]
    lib.orc_partition.restype = i64
    lib.orc_mh_sample.argtypes = [i32, vp, vp, i64, u64, u32, u32, u32, i64, u32, vp, vp, vp, i64, vp, vp]
    lib.orc_mh_sample.restype = i64
    lib.orc_mh_sample_segments.argtypes = [i32, vp, vp, i64, u64, u32, u32, u32, i64, u32, i64, i64, vp, vp, vp,
                                           i64, vp, vp]
    lib.orc_mh_sample_segments.restype = i64
    lib.orc_bf_sample.argtypes = [i32, vp, vp, i64, u64, u32, vp, vp, vp, i64, vp]
    lib.orc_bf_sample.restype = i64
    lib.orc_bip_partition.argtypes = [i32, vp, vp, i64, vp, vp, i64, i64, vp, vp, vp, vp, i64, vp, vp]
    lib.orc_bip_partition.restype = i64
    lib.orc_bip_sample.argtypes = [i32, vp, vp, i64, vp, vp, i64, i32, u64, u32, u32, u32, i64, vp, vp, vp, i64,
                                   vp, vp]
    lib.orc_bip_sample.restype = i64
    lib.orc_bip_bf_sample.argtypes = [i32, vp, vp, i64, vp, vp, i64, i32, u64, u32, vp, vp, vp, i64, vp]
    lib.orc_bip_bf_sample.restype = i64
    lib.orc_boundary_log.argtypes = [vp, i64]
    lib.orc_boundary_log.restype = None
    lib.orc_boundary_log_len.argtypes = []
    lib.orc_boundary_log_len.restype = i64
    return lib


def load(path: str | None = None):
    """Load (building if needed) the C oracle.  ``path`` selects another build."""
    global _LIB
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _LOCK:
        if _LIB is None:
            _LIB = _declare(ctypes.CDLL(build()))
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Philox4x32-10 and node order
# --------------------------------------------------------------------------
def philox(ctr, key, lib=None) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) of one 128-bit counter, 64-bit key."""
    lib = lib or load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sort_desc(key, lib=None) -> np.ndarray:
    """Ranks in descending key order, ties by ascending id (Sec. 2.4 step (i))."""
    lib = lib or load()
    k = _f64(key)
    perm = np.zeros(len(k), dtype=np.int32)
    lib.orc_sort_desc(_ptr(k), len(k), _ptr(perm))
    return perm


# --------------------------------------------------------------------------
# Segment table, MH walk, brute force
# --------------------------------------------------------------------------
def partition(model, x, y=None, seg_target=32, flags=0, lib=None):
    """Row-segment table (row rank, k, a, b) in canonical order, plus the node order."""
    lib = lib or load()
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    n = len(x)
    cap = max(4 * n + 1024, 16)
    while True:
        row = np.zeros(cap, np.int32)
        k = np.zeros(cap, np.int32)
        a = np.zeros(cap, np.int64)
        b = np.zeros(cap, np.int64)
        perm = np.zeros(max(n, 1), np.int32)
        total = lib.orc_partition(model, _ptr(x), _ptr(y), n, int(seg_target), flags, _ptr(row), _ptr(k),
                                  _ptr(a), _ptr(b), cap, _ptr(perm))
        if total <= cap:
            return dict(row=row[:total], k=k[:total], a=a[:total], b=b[:total], perm=perm[:n])
        cap = int(total)


def mh_sample(model, x, y=None, *, seed=0, network_id=0, sample_begin=0, num_samples=1, seg_target=32,
              flags=0, lib=None):
    """Serial Miller-Hagberg samples.  Returns (src, dst, w or None, counts, stats).

    stats = [proposals drawn, edges, segments walked, boundary draws]: a
    boundary draw is a skip draw whose t lies within 8 ulp of an integer m in
    [1, b - pos - 1], or a weight draw whose t >= 0.5 lies within 8 ulp of an
    integer (``boundary_draws`` lists them).
    """
    lib = lib or load()
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    n = len(x)
    cap = 1024
    while True:
        src = np.zeros(cap, np.int32)
        dst = np.zeros(cap, np.int32)
        w = np.zeros(cap, np.int32) if model == UECM else None
        counts = np.zeros(max(num_samples, 1), np.int64)
        stats = np.zeros(4, np.uint64)
        total = lib.orc_mh_sample(model, _ptr(x), _ptr(y), n, int(seed), int(network_id), int(sample_begin),
                                  int(num_samples), int(seg_target), int(flags), _ptr(src), _ptr(dst), _ptr(w),
                                  cap, _ptr(counts), _ptr(stats))
        if total < 0:
            raise OverflowError("a sampled weight exceeds INT32_MAX")
        if total <= cap:
            return (src[:total], dst[:total], None if w is None else w[:total], counts[:num_samples], stats)
        cap = int(total)


def mh_sample_segments(model, x, y=None, *, seg_begin, seg_end, seed=0, network_id=0, sample_begin=0,
                       num_samples=1, seg_target=32, flags=0, lib=None):
    """mh_sample restricted to rows [seg_begin, seg_end) of the segment table
    (``partition``'s canonical order), each sample's edges in that range."""
    lib = lib or load()
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    n = len(x)
    cap = 1024
    while True:
        src = np.zeros(cap, np.int32)
        dst = np.zeros(cap, np.int32)
        w = np.zeros(cap, np.int32) if model == UECM else None
        counts = np.zeros(max(num_samples, 1), np.int64)
        stats = np.zeros(4, np.uint64)
        total = lib.orc_mh_sample_segments(model, _ptr(x), _ptr(y), n, int(seed), int(network_id),
                                           int(sample_begin), int(num_samples), int(seg_target), int(flags),
                                           int(seg_begin), int(seg_end), _ptr(src), _ptr(dst), _ptr(w), cap,
                                           _ptr(counts), _ptr(stats))
        if total < 0:
            raise OverflowError("a sampled weight exceeds INT32_MAX")
        if total <= cap:
            return (src[:total], dst[:total], None if w is None else w[:total], counts[:num_samples], stats)
        cap = int(total)


def boundary_draws(sample_fn, *args, max_entries=1 << 16, **kw):
    """Runs ``sample_fn(*args, **kw)`` (``mh_sample`` or ``bip_sample``) with
    the oracle's boundary-draw log on.  Returns (its result, log) where log is
    an int64 array of rows (sample, row rank i, segment k, kind, index):
    kind 0 is the skip draw ``index`` of that segment, kind 1 the weight draw
    of its edge ``index``."""
    lib = kw.get("lib") or load()
    buf = np.zeros(5 * max_entries, np.uint32)
    lib.orc_boundary_log(_ptr(buf), max_entries)
    try:
        res = sample_fn(*args, **kw)
        m = int(lib.orc_boundary_log_len())
    finally:
        lib.orc_boundary_log(None, 0)
    if m > max_entries:
        raise RuntimeError(f"{m} boundary draws, more than the log's {max_entries} entries")
    return res, buf[:5 * m].reshape(m, 5).astype(np.int64)


def bf_sample(model, x, y=None, *, seed=0, sample=0, lib=None):
    """Brute-force sample: every pair an independent Bernoulli (Sec. 2.2).

    Returns (src, dst, w or None, pair evaluations)."""
    lib = lib or load()
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    n = len(x)
    cap = max(1024, n * 8)
    while True:
        src = np.zeros(cap, np.int32)
        dst = np.zeros(cap, np.int32)
        w = np.zeros(cap, np.int32) if model == UECM else None
        ev = np.zeros(1, np.uint64)
        total = lib.orc_bf_sample(model, _ptr(x), _ptr(y), n, int(seed), int(sample), _ptr(src), _ptr(dst),
                                  _ptr(w), cap, _ptr(ev))
        if total <= cap:
            return src[:total], dst[:total], None if w is None else w[:total], int(ev[0])
        cap = int(total)


# --------------------------------------------------------------------------
# Expected degrees and strengths (the O(N^2) evaluation behind parameter
# inference, Sec. 2.2 and Sec. 4) and their gradients.
# --------------------------------------------------------------------------
def _pair_terms(model, x, y, i, rows=None):
    """p_ij and m_ij = p_ij / (1 - r_ij) for all j != i (FP64)."""
    n = len(x)
    j = np.arange(n) if rows is None else rows
    j = j[j != i]
    if model == UBCM:
        z = x[i] * x[j]
        p = z / (1.0 + z)
        return j, p, None, None
    a = x * y
    A = a[i] * a[j]
    r = y[i] * y[j]
    p = A / ((1.0 - r) + A)
    return j, p, p / (1.0 - r), r


def expected_fwd(model, x, y=None, rows=None):
    """<k_i> = sum_{j!=i} p_ij and (UECM) <s_i> = sum_{j!=i} p_ij / (1 - r_ij).

    The strength uses E[w | w > 0] = 1 / (1 - r) of Eq. 4.  ``rows`` limits
    the output to those i (full sums over j)."""
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    idx = np.arange(len(x)) if rows is None else np.asarray(rows)
    k = np.zeros(len(idx))
    s = np.zeros(len(idx)) if model == UECM else None
    for t, i in enumerate(idx):
        _, p, m, _ = _pair_terms(model, x, y, int(i))
        k[t] = math.fsum(p.tolist())
        if model == UECM:
            s[t] = math.fsum(m.tolist())
    return k, s


def expected_bwd(model, x, y, g_k, g_s=None, rows=None):
    """Gradient of L(<k>, <s>) with respect to x (and y) given dL/d<k>, dL/d<s>.

    With p symmetric, d L / d x_i = sum_{j!=i} (g_k,i + g_k,j) dp_ij/dx_i
    + (g_s,i + g_s,j) dm_ij/dx_i, and likewise for y_i, where (D = 1 - r + A)
      dp/dx_i = p (1 - p) / x_i            dp/dy_i = p / (y_i D)
      dm/dx_i = p (1 - p) / (x_i (1 - r))  dm/dy_i = p / (y_i D (1 - r)) + p r / (y_i (1 - r)^2)
    """
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    g_k = _f64(g_k)
    g_s = _f64(g_s) if model == UECM else None
    idx = np.arange(len(x)) if rows is None else np.asarray(rows)
    gx = np.zeros(len(idx))
    gy = np.zeros(len(idx)) if model == UECM else None
    for t, i in enumerate(idx):
        i = int(i)
        j, p, m, r = _pair_terms(model, x, y, i)
        gk = g_k[i] + g_k[j]
        dp_dx = p * (1.0 - p) / x[i]
        if model == UBCM:
            gx[t] = math.fsum((gk * dp_dx).tolist())
            continue
        gs = g_s[i] + g_s[j]
        a = x * y
        A = a[i] * a[j]
        D = (1.0 - r) + A
        dm_dx = dp_dx / (1.0 - r)
        dp_dy = p / (y[i] * D)
        dm_dy = p / (y[i] * D * (1.0 - r)) + p * r / (y[i] * (1.0 - r) ** 2)
        gx[t] = math.fsum((gk * dp_dx).tolist() + (gs * dm_dx).tolist())
        gy[t] = math.fsum((gk * dp_dy).tolist() + (gs * dm_dy).tolist())
    return gx, gy


def expected_jacobian_diag(model, x, y=None, rows=None):
    """Diagonal of the Jacobian of the expected degrees (and strengths) of the
    maximum-likelihood conditions (Sec. 2.2, Sec. 2.5): for each row i the
    partial derivatives of <k_i> (and <s_i>) with respect to the node's own
    x_i (and y_i), every other parameter held fixed.  With D = 1 - r + A,
      d<k_i>/dx_i = sum_j p (1 - p) / x_i
      d<k_i>/dy_i = sum_j p / (y_i D)
      d<s_i>/dx_i = sum_j p (1 - p) / (x_i (1 - r))
      d<s_i>/dy_i = sum_j p / (y_i D (1 - r)) + p r / (y_i (1 - r)^2)
    Returns (dk_dx,) for the UBCM and (dk_dx, dk_dy, ds_dx, ds_dy) for the
    UECM; x_i (and y_i) must be positive."""
    x = _f64(x)
    y = _f64(y) if model == UECM else None
    idx = np.arange(len(x)) if rows is None else np.asarray(rows)
    out = [np.zeros(len(idx)) for _ in range(1 if model == UBCM else 4)]
    for t, i in enumerate(idx):
        i = int(i)
        j, p, m, r = _pair_terms(model, x, y, i)
        dp_dx = p * (1.0 - p) / x[i]
        out[0][t] = math.fsum(dp_dx.tolist())
        if model == UBCM:
            continue
        a = x * y
        D = (1.0 - r) + a[i] * a[j]
        out[1][t] = math.fsum((p / (y[i] * D)).tolist())
        out[2][t] = math.fsum((dp_dx / (1.0 - r)).tolist())
        out[3][t] = math.fsum((p / (y[i] * D * (1.0 - r)) + p * r / (y[i] * (1.0 - r) ** 2)).tolist())
    return tuple(out)


# --------------------------------------------------------------------------
# Exact law of a tiny network: all 2^(N(N-1)/2) simple graphs.
# --------------------------------------------------------------------------
def pair_list(n):
    return [(u, v) for u in range(n) for v in range(u + 1, n)]


def graph_probabilities(model, alpha, beta=None):
    """Probability of every simple graph (pairs independent, Eq. 1 / Eq. 3).

    Written in the paper's alpha/beta notation, independent of the x/y form
    the samplers use.  Graph g has bit t set when pair t of ``pair_list`` is
    an edge."""
    n = len(alpha)
    pairs = pair_list(n)
    probs = []
    for (u, v) in pairs:
        if model == UBCM:
            e = math.exp(-alpha[u] - alpha[v])
            probs.append(e / (1.0 + e))
        elif model == CL:  # expected multiplicity k_u k_v / 2M taken as a probability, capped at 1
            probs.append(min(1.0, math.exp(-alpha[u] - alpha[v])))
        else:
            num = math.exp(-alpha[u] - alpha[v] - beta[u] - beta[v])
            probs.append(num / (1.0 - math.exp(-beta[u] - beta[v]) + num))
    out = np.zeros(1 << len(pairs))
    for g, bits in enumerate(itertools.product((0, 1), repeat=len(pairs))):
        pr = 1.0
        for t, b in enumerate(reversed(bits)):
            pr *= probs[t] if b else (1.0 - probs[t])
        out[g] = pr
    return out, np.array(probs)


def graph_codes(src, dst, counts, n):
    """Encode each sample's edge list as its graph bit pattern (see graph_probabilities)."""
    index = {pq: t for t, pq in enumerate(pair_list(n))}
    codes = np.zeros(len(counts), dtype=np.int64)
    pos = 0
    for s, c in enumerate(counts):
        code = 0
        for e in range(pos, pos + int(c)):
            u, v = int(src[e]), int(dst[e])
            code |= 1 << index[(min(u, v), max(u, v))]
        codes[s] = code
        pos += int(c)
    return codes


def symmetric_csr(src, dst, w, counts, n):
    """Every edge of every sample in both endpoint rows.

    Sample s's rows follow the samples before it; each edge, taken in the
    sample's output order, appends v to row u and u to row v (weights
    alongside).  Returns (offsets int64[S (n + 1)] as global positions,
    indices int32[2 M], weights int32[2 M] or None)."""
    S = len(counts)
    offsets = np.zeros(S * (n + 1), dtype=np.int64)
    indices, weights = [], []
    pos = 0
    for s in range(S):
        rows = [[] for _ in range(n)]
        for e in range(pos, pos + int(counts[s])):
            u, v = int(src[e]), int(dst[e])
            we = None if w is None else int(w[e])
            rows[u].append((v, we))
            rows[v].append((u, we))
        base = len(indices)
        for u in range(n):
            offsets[s * (n + 1) + u] = base
            for v, we in rows[u]:
                indices.append(v)
                weights.append(we)
            base = len(indices)
        offsets[s * (n + 1) + n] = base
        pos += int(counts[s])
    idx = np.array(indices, dtype=np.int32)
    wts = None if w is None else np.array(weights, dtype=np.int32)
    return offsets, idx, wts


# --------------------------------------------------------------------------
# Bipartite and directed networks (Sec. 2.6)
# --------------------------------------------------------------------------
def bip_partition(model, xp, yp, xm, ym, seg_target=32, lib=None):
    """Row-segment table of a bipartite network: (+ rank, k, a, b) with a, b
    in - ranks, plus both node orders."""
    lib = lib or load()
    xp, xm = _f64(xp), _f64(xm)
    yp = _f64(yp) if model == UECM else None
    ym = _f64(ym) if model == UECM else None
    np_, nm = len(xp), len(xm)
    cap = max(4 * np_ + 1024, 16)
    while True:
        row = np.zeros(cap, np.int32)
        k = np.zeros(cap, np.int32)
        a = np.zeros(cap, np.int64)
        b = np.zeros(cap, np.int64)
        pp = np.zeros(max(np_, 1), np.int32)
        pm = np.zeros(max(nm, 1), np.int32)
        total = lib.orc_bip_partition(model, _ptr(xp), _ptr(yp), np_, _ptr(xm), _ptr(ym), nm, int(seg_target),
                                      _ptr(row), _ptr(k), _ptr(a), _ptr(b), cap, _ptr(pp), _ptr(pm))
        if total <= cap:
            return dict(row=row[:total], k=k[:total], a=a[:total], b=b[:total], perm_plus=pp[:np_],
                        perm_minus=pm[:nm])
        cap = int(total)


def bip_sample(model, xp, yp, xm, ym, *, directed=False, seed=0, network_id=0, sample_begin=0, num_samples=1,
               seg_target=32, lib=None):
    """Serial walk of a bipartite (or directed) network.  Returns (src, dst, w
    or None, counts, stats) with src a + id and dst a - id (out / in ids when
    directed); stats as in mh_sample."""
    lib = lib or load()
    xp, xm = _f64(xp), _f64(xm)
    yp = _f64(yp) if model == UECM else None
    ym = _f64(ym) if model == UECM else None
    cap = 1024
    while True:
        src = np.zeros(cap, np.int32)
        dst = np.zeros(cap, np.int32)
        w = np.zeros(cap, np.int32) if model == UECM else None
        counts = np.zeros(max(num_samples, 1), np.int64)
        st = np.zeros(4, np.uint64)
        total = lib.orc_bip_sample(model, _ptr(xp), _ptr(yp), len(xp), _ptr(xm), _ptr(ym), len(xm), int(directed),
                                   int(seed), int(network_id), int(sample_begin), int(num_samples), int(seg_target),
                                   _ptr(src), _ptr(dst), _ptr(w), cap, _ptr(counts), _ptr(st))
        if total < 0:
            raise ValueError("weight above INT32_MAX, or a directed network with unequal sets")
        if total <= cap:
            return src[:total], dst[:total], None if w is None else w[:total], counts[:num_samples], st
        cap = int(total)


def bip_bf_sample(model, xp, yp, xm, ym, *, directed=False, seed=0, sample=0, lib=None):
    """Brute-force sample of a bipartite (or directed) network: (src, dst, w or None, evaluations)."""
    lib = lib or load()
    xp, xm = _f64(xp), _f64(xm)
    yp = _f64(yp) if model == UECM else None
    ym = _f64(ym) if model == UECM else None
    cap = len(xp) * len(xm) + 1
    src = np.zeros(cap, np.int32)
    dst = np.zeros(cap, np.int32)
    w = np.zeros(cap, np.int32) if model == UECM else None
    ev = ctypes.c_uint64(0)
    total = lib.orc_bip_bf_sample(model, _ptr(xp), _ptr(yp), len(xp), _ptr(xm), _ptr(ym), len(xm), int(directed),
                                  int(seed), int(sample), _ptr(src), _ptr(dst), _ptr(w), cap, ctypes.byref(ev))
    return src[:total], dst[:total], None if w is None else w[:total], int(ev.value)


def bip_pair_list(n_plus, n_minus, directed=False):
    return [(u, v) for u in range(n_plus) for v in range(n_minus) if not (directed and u == v)]


def bip_graph_probabilities(model, alpha_p, alpha_m, beta_p=None, beta_m=None, directed=False):
    """Probability of every graph on the pairs of bip_pair_list (independent
    pairs, Eq. 1 / Eq. 3 with one endpoint in each set), in the paper's
    alpha/beta notation.  Graph g has bit t set when pair t is an edge."""
    pairs = bip_pair_list(len(alpha_p), len(alpha_m), directed)
    probs = []
    for (u, v) in pairs:
        if model == UBCM:
            e = math.exp(-alpha_p[u] - alpha_m[v])
            probs.append(e / (1.0 + e))
        else:
            num = math.exp(-alpha_p[u] - alpha_m[v] - beta_p[u] - beta_m[v])
            probs.append(num / (1.0 - math.exp(-beta_p[u] - beta_m[v]) + num))
    out = np.zeros(1 << len(pairs))
    for g, bits in enumerate(itertools.product((0, 1), repeat=len(pairs))):
        pr = 1.0
        for t, b in enumerate(reversed(bits)):
            pr *= probs[t] if b else (1.0 - probs[t])
        out[g] = pr
    return out, np.array(probs)
