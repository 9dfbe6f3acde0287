"""The parity rule between a sampler's output and the oracle's (test helper).

Edge lists, weights and per-sample counts must equal the oracle's bit for
bit.  The one allowed exception is a boundary draw: a skip draw whose FP64
t = log(U) / log1p(-q) lies within 8 ulp of an integer that decides the
candidate, or a weight draw whose log(U_w) / log(r) lies within 8 ulp of an
integer (Sec. 2.3 skip law; Eq. 4).  There the device and host logarithms may
round differently.  So a difference is accepted only when every segment
whose edges or weights differ holds a boundary draw that the oracle logged
(its (sample, row rank, segment) is in the oracle's boundary log).

Every edge of a one-set sample belongs to one segment: its row is the rank
of its higher-ranked endpoint u, its candidate the rank j of the other
endpoint, and its segment the table row of that row with a <= j < b.
"""
import numpy as np

import oracle


def _locate(tab_row, tab_k, tab_a, tab_b, i, j, ncol, counts, nedges):
    key_tab = tab_row.astype(np.int64) * (ncol + 1) + tab_a
    at = np.searchsorted(key_tab, i * (ncol + 1) + j, side="right") - 1
    if len(at) and (at.min() < 0 or np.any(tab_row[at] != i) or np.any(j >= tab_b[at])):
        raise AssertionError("an edge lies in no segment of its row")
    sample = np.repeat(np.arange(len(counts)), np.asarray(counts, np.int64))
    if len(sample) != nedges:
        raise AssertionError("per-sample counts do not add up to the edge count")
    return sample, i, tab_k[at].astype(np.int64)


def _rank(perm):
    r = np.empty(len(perm), np.int64)
    r[perm] = np.arange(len(perm))
    return r


def edge_segments(model, x, y, src, dst, counts, *, seg_target, flags):
    """(sample, row rank, segment k) of every edge of a one-set sample list."""
    tab = oracle.partition(model, x, y, seg_target=seg_target, flags=flags)
    rank = _rank(tab["perm"])
    i, j = rank[np.asarray(src, np.int64)], rank[np.asarray(dst, np.int64)]
    return _locate(tab["row"], tab["k"], tab["a"], tab["b"], i, j, len(x), counts, len(src))


def bip_edge_segments(model, xp, yp, xm, ym, src, dst, counts, *, seg_target):
    """The same for a bipartite or directed sample (src a + id, dst a - id;
    segments in - ranks, cut over the actual candidates, Sec. 2.6)."""
    tab = oracle.bip_partition(model, xp, yp, xm, ym, seg_target=seg_target)
    i = _rank(tab["perm_plus"])[np.asarray(src, np.int64)]
    j = _rank(tab["perm_minus"])[np.asarray(dst, np.int64)]
    return _locate(tab["row"], tab["k"], tab["a"], tab["b"], i, j, len(xm), counts, len(src))


def _groups(seg, dst, w):
    s, i, k = seg
    out = {}
    for e in range(len(s)):
        out.setdefault((int(s[e]), int(i[e]), int(k[e])), []).append(
            (int(dst[e]), None if w is None else int(w[e])))
    return out


def _differing(segs, got, ref):
    gg = _groups(segs(got[0], got[1], got[3]), got[1], got[2])
    rg = _groups(segs(ref[0], ref[1], ref[3]), ref[1], ref[2])
    return {key for key in set(gg) | set(rg) if gg.get(key) != rg.get(key)}


def differing_segments(model, x, y, got, ref, *, seg_target, flags):
    """Segments (sample, row rank, k) whose edge runs differ between two sample
    lists; got and ref are (src, dst, w or None, counts)."""
    return _differing(lambda s, d, c: edge_segments(model, x, y, s, d, c, seg_target=seg_target, flags=flags),
                      got, ref)


def _assert_subset(diff, log, sample_begin):
    flagged = {(int(e[0]) - sample_begin, int(e[1]), int(e[2])) for e in log}
    untraced = sorted(diff - flagged)
    assert not untraced, (f"{len(untraced)} segment(s) differ from the oracle without a boundary draw, "
                          f"first (sample, row, segment) = {untraced[:3]}; oracle boundary draws: {len(log)}")


def oracle_sample(model, x, y=None, **kw):
    """The oracle's sample with its boundary log: ((src, dst, w or None, counts), stats, log)."""
    (src, dst, w, counts, stats), log = oracle.boundary_draws(oracle.mh_sample, model, x, y, **kw)
    return (src, dst, w, counts), stats, log


def same_sample(got, ref):
    g_src, g_dst, g_w, g_counts = got
    src, dst, w, counts = ref
    return (np.array_equal(np.asarray(g_counts), counts) and np.array_equal(np.asarray(g_src), src)
            and np.array_equal(np.asarray(g_dst), dst) and (w is None or np.array_equal(np.asarray(g_w), w)))


def assert_traced(model, x, y, got, ref, log, *, seg_target, flags, sample_begin=0):
    """Every segment whose runs differ between got and ref holds a boundary
    draw of the oracle's log (whose samples are absolute indices)."""
    got = tuple(None if v is None else np.asarray(v) for v in got)
    _assert_subset(differing_segments(model, x, y, got, ref, seg_target=seg_target, flags=flags), log,
                   sample_begin)


def check_sample(got, model, x, y=None, *, num_samples=1, seg_target=32, flags=0, seed=0, sample_begin=0,
                 network_id=0):
    """Compares got = (src, dst, w or None, counts) with the oracle's sample.

    Returns (same, stats): same is True when the lists are identical; when
    they differ, every differing segment must hold a logged boundary draw
    (AssertionError otherwise) and same is False."""
    ref, stats, log = oracle_sample(model, x, y, seed=seed, network_id=network_id, sample_begin=sample_begin,
                                    num_samples=num_samples, seg_target=seg_target, flags=flags)
    if same_sample(got, ref):
        return True, stats
    assert_traced(model, x, y, got, ref, log, seg_target=seg_target, flags=flags, sample_begin=sample_begin)
    return False, stats


def check_bip_sample(got, model, xp, yp, xm, ym, *, directed=False, num_samples=1, seg_target=32, seed=0,
                     sample_begin=0, network_id=0):
    """check_sample for a bipartite or directed network (Sec. 2.6)."""
    (src, dst, w, counts, stats), log = oracle.boundary_draws(
        oracle.bip_sample, model, xp, yp, xm, ym, directed=directed, seed=seed, network_id=network_id,
        sample_begin=sample_begin, num_samples=num_samples, seg_target=seg_target)
    ref = (src, dst, w, counts)
    if same_sample(got, ref):
        return True, ref, stats
    got = tuple(None if v is None else np.asarray(v) for v in got)
    segs = lambda s, d, c: bip_edge_segments(model, xp, yp, xm, ym, s, d, c, seg_target=seg_target)  # noqa: E731
    _assert_subset(_differing(segs, got, ref), log, sample_begin)
    return False, ref, stats
