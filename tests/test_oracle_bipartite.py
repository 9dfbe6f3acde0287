"""Pins of the oracle's bipartite and directed samplers (Sec. 2.6), no GPU.

As for one node set, every check compares sampler output with a law written
in the paper's alpha/beta notation: exact enumeration of every graph on a
tiny network, per-pair closed forms, the weight law of Eq. 4, the
Erdős-Rényi special case and expected degrees.  A directed network is the
bipartite one on (out-copies, in-copies) without the pairs (i, i)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from tests.oracle_pins import alpha_of, chi2_pvalue

UBCM, UECM = oracle.UBCM, oracle.UECM


def bip_code_counts(src, dst, counts, n_plus, n_minus, directed):
    """Histogram of sampled graphs (bit t = pair t of bip_pair_list) plus a
    final cell for samples with an invalid edge (self pair when directed,
    duplicate, bad id)."""
    index = {pq: t for t, pq in enumerate(oracle.bip_pair_list(n_plus, n_minus, directed))}
    hist = np.zeros((1 << len(index)) + 1)
    pos = 0
    for c in counts:
        code, ok = 0, True
        for e in range(pos, pos + int(c)):
            key = (int(src[e]), int(dst[e]))
            if key not in index or (code >> index[key]) & 1:
                ok = False
                break
            code |= 1 << index[key]
        hist[code if ok else -1] += 1
        pos += int(c)
    return hist


def bip_enumeration_pvalue(model, xp, xm, yp=None, ym=None, *, directed=False, samples=40000, seg_target=1 << 30,
                           seed=5, sampler="mh", lib=None):
    exact, _ = oracle.bip_graph_probabilities(model, alpha_of(xp), alpha_of(xm),
                                              None if yp is None else alpha_of(yp),
                                              None if ym is None else alpha_of(ym), directed)
    if sampler == "mh":
        src, dst, _, counts, _ = oracle.bip_sample(model, xp, yp, xm, ym, directed=directed, seed=seed,
                                                   num_samples=samples, seg_target=seg_target, lib=lib)
    else:
        parts = [oracle.bip_bf_sample(model, xp, yp, xm, ym, directed=directed, seed=seed, sample=s, lib=lib)
                 for s in range(samples)]
        src = np.concatenate([p[0] for p in parts])
        dst = np.concatenate([p[1] for p in parts])
        counts = np.array([len(p[0]) for p in parts])
    hist = bip_code_counts(src, dst, counts, len(xp), len(xm), directed)
    assert hist[-1] == 0, "invalid edge in a sample"
    return chi2_pvalue(hist[:-1], exact * samples)


BIP_XP = np.array([2.5, 0.4])
BIP_XM = np.array([1.2, 0.7, 0.15])
BIP_YP = np.array([0.8, 0.35])
BIP_YM = np.array([0.6, 0.9, 0.2])
DIR_XO = np.array([1.5, 0.5, 0.2])
DIR_XI = np.array([0.3, 2.0, 0.8])
DIR_YO = np.array([0.7, 0.3, 0.85])
DIR_YI = np.array([0.5, 0.9, 0.25])


@pytest.mark.parametrize("T", [2, 1 << 30])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_bipartite_walk_matches_exact_enumeration(model, T):
    yp, ym = (BIP_YP, BIP_YM) if model == UECM else (None, None)
    assert bip_enumeration_pvalue(model, BIP_XP, BIP_XM, yp, ym, seg_target=T) > 1e-4


@pytest.mark.parametrize("T", [2, 1 << 30])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_directed_walk_matches_exact_enumeration(model, T):
    yo, yi = (DIR_YO, DIR_YI) if model == UECM else (None, None)
    assert bip_enumeration_pvalue(model, DIR_XO, DIR_XI, yo, yi, directed=True, seg_target=T) > 1e-4


@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_brute_force_matches_exact_enumeration(model, directed):
    if directed:
        xp, xm, yp, ym = DIR_XO, DIR_XI, DIR_YO, DIR_YI
    else:
        xp, xm, yp, ym = BIP_XP, BIP_XM, BIP_YP, BIP_YM
    if model == UBCM:
        yp = ym = None
    assert bip_enumeration_pvalue(model, xp, xm, yp, ym, directed=directed, samples=20000, sampler="bf") > 1e-4


@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_pair_marginals_and_weights(model, directed):
    rng = np.random.default_rng(21 + model + 2 * directed)
    n_plus, n_minus = (5, 5) if directed else (4, 6)
    xp, xm = np.exp(rng.normal(-0.5, 1.2, n_plus)), np.exp(rng.normal(-0.5, 1.2, n_minus))
    xp[0] = 6.0  # a hub: long runs of near-certain candidates
    yp = rng.uniform(0.1, 0.9, n_plus) if model == UECM else None
    ym = rng.uniform(0.1, 0.9, n_minus) if model == UECM else None
    S = 20000
    src, dst, w, counts, _ = oracle.bip_sample(model, xp, yp, xm, ym, directed=directed, num_samples=S,
                                               seg_target=2)
    ap, am = alpha_of(xp), alpha_of(xm)
    zmax = 0.0
    pooled_obs, pooled_exp = [], []
    for (u, v) in oracle.bip_pair_list(n_plus, n_minus, directed):
        if model == UBCM:
            e = math.exp(-ap[u] - am[v])
            p = e / (1.0 + e)
        else:
            bp, bm = alpha_of(yp), alpha_of(ym)
            num = math.exp(-ap[u] - am[v] - bp[u] - bm[v])
            p = num / (1.0 - math.exp(-bp[u] - bm[v]) + num)
        sel = (src == u) & (dst == v)
        f = sel.sum() / S
        zmax = max(zmax, abs(f - p) / math.sqrt(p * (1 - p) / S + 1e-300))
        if model == UECM and sel.sum() > 50:
            r = math.exp(-bp[u] - bm[v])
            ws = w[sel]
            kmax = 6
            obs = np.array([(ws == k).sum() for k in range(1, kmax)] + [(ws >= kmax).sum()])
            exp = np.array([r ** (k - 1) * (1 - r) for k in range(1, kmax)] + [r ** (kmax - 1)]) * len(ws)
            pooled_obs.append(obs)
            pooled_exp.append(exp)
    assert zmax < 4.5
    if model == UECM:
        assert chi2_pvalue(np.concatenate(pooled_obs), np.concatenate(pooled_exp)) > 1e-4
    if directed:
        assert not np.any(src == dst)


def test_bipartite_erdos_renyi_special_case():
    # all x equal within each set: every pair has the same p, so the edge
    # count is Binomial(n+ n-, p) (Eq. 1)
    n_plus, n_minus = 30, 45
    xp, xm = np.full(n_plus, 0.3), np.full(n_minus, 0.5)
    _, _, _, counts, _ = oracle.bip_sample(UBCM, xp, None, xm, None, num_samples=4000, seg_target=3)
    p = 0.15 / 1.15
    n_pairs = n_plus * n_minus
    assert abs(counts.mean() - n_pairs * p) < 4.5 * math.sqrt(n_pairs * p * (1 - p) / 4000)
    assert stats.kstest(counts, stats.binom(n_pairs, p).cdf).pvalue > 1e-4


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_directed_degrees_in_expectation(model):
    rng = np.random.default_rng(31 + model)
    n = 40
    xo, xi = np.exp(rng.normal(-1.0, 1.0, n)), np.exp(rng.normal(-1.0, 1.0, n))
    yo = rng.uniform(0.2, 0.9, n) if model == UECM else None
    yi = rng.uniform(0.2, 0.9, n) if model == UECM else None
    S = 10000
    src, dst, w, counts, _ = oracle.bip_sample(model, xo, yo, xi, yi, directed=True, num_samples=S, seg_target=4)
    ao, ai = alpha_of(xo), alpha_of(xi)
    P = np.zeros((n, n))
    for u in range(n):
        for v in range(n):
            if u == v:
                continue
            if model == UBCM:
                e = math.exp(-ao[u] - ai[v])
                P[u, v] = e / (1.0 + e)
            else:
                bo, bi = alpha_of(yo), alpha_of(yi)
                num = math.exp(-ao[u] - ai[v] - bo[u] - bi[v])
                P[u, v] = num / (1.0 - math.exp(-bo[u] - bi[v]) + num)
    out_deg = np.bincount(src, minlength=n) / S
    in_deg = np.bincount(dst, minlength=n) / S
    sd_out = np.sqrt((P * (1 - P)).sum(axis=1) / S)
    sd_in = np.sqrt((P * (1 - P)).sum(axis=0) / S)
    assert np.max(np.abs(out_deg - P.sum(axis=1)) / sd_out) < 4.5
    assert np.max(np.abs(in_deg - P.sum(axis=0)) / sd_in) < 4.5


@pytest.mark.parametrize("T", [2, 5, 1 << 30])
def test_bipartite_partition_covers_every_row(T):
    rng = np.random.default_rng(T)
    xp, xm = np.exp(rng.normal(0.0, 1.5, 40)), np.exp(rng.normal(-1.0, 1.5, 70))
    part = oracle.bip_partition(UBCM, xp, None, xm, None, seg_target=T)
    row, k, a, b = part["row"], part["k"], part["a"], part["b"]
    assert np.array_equal(np.unique(row), np.arange(40))
    for i in range(40):
        sel = row == i
        assert np.array_equal(k[sel], np.arange(sel.sum()))
        assert a[sel][0] == 0 and b[sel][-1] == 70
        assert np.all(a[sel][1:] == b[sel][:-1]) and np.all(b[sel] > a[sel])
        if T == 1 << 30:
            assert sel.sum() == 1
    assert np.array_equal(np.sort(part["perm_plus"]), np.arange(40))
    assert np.array_equal(part["perm_minus"], oracle.sort_desc(xm))


def test_uecm_bound_with_rising_y_along_the_order():
    # sorted by a = x y, the - set's y rises: the bound must use the largest
    # y ahead of the segment head, not the head's own
    ym = np.array([0.1, 0.3, 0.5, 0.7, 0.9])
    xm = np.array([1.0, 0.8, 0.6, 0.4, 0.2]) / ym
    yp = np.array([0.95, 0.6])
    xp = np.array([1.0, 0.5]) / yp
    S = 20000
    for T in (2, 1 << 30):
        src, dst, _, _, _ = oracle.bip_sample(UECM, xp, yp, xm, ym, num_samples=S, seg_target=T)
        ap, am, bp, bm = alpha_of(xp), alpha_of(xm), alpha_of(yp), alpha_of(ym)
        zmax = 0.0
        for (u, v) in oracle.bip_pair_list(2, 5):
            num = math.exp(-ap[u] - am[v] - bp[u] - bm[v])
            p = num / (1.0 - math.exp(-bp[u] - bm[v]) + num)
            f = ((src == u) & (dst == v)).sum() / S
            zmax = max(zmax, abs(f - p) / math.sqrt(p * (1 - p) / S))
        assert zmax < 4.5
