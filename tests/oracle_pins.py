"""Statistical pins shared by the oracle tests and the planted-mistake tests.

Every check compares sampler output with a law fixed by the paper itself,
written in the paper's alpha/beta notation (Eq. 1, Eq. 3, Eq. 4), never with
another oracle function.  Seeds are fixed, so each check is deterministic.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats

import oracle


def alpha_of(x):
    return -np.log(np.asarray(x, dtype=np.float64))


def p_ubcm_alpha(alpha, u, v):
    """Eq. 1."""
    e = math.exp(-alpha[u] - alpha[v])
    return e / (1.0 + e)


def p_uecm_alpha(alpha, beta, u, v):
    """Eq. 3."""
    num = math.exp(-alpha[u] - alpha[v] - beta[u] - beta[v])
    return num / (1.0 - math.exp(-beta[u] - beta[v]) + num)


def chi2_pvalue(observed, expected, min_expected=5.0):
    """Pearson chi-square after pooling the sparse cells into one."""
    observed = np.asarray(observed, dtype=np.float64)
    expected = np.asarray(expected, dtype=np.float64)
    keep = expected >= min_expected
    obs = list(observed[keep])
    exp = list(expected[keep])
    if (~keep).any():
        obs.append(observed[~keep].sum())
        exp.append(expected[~keep].sum())
    obs, exp = np.array(obs), np.array(exp)
    exp *= obs.sum() / exp.sum()
    return float(stats.chisquare(obs, exp).pvalue)


def graph_code_counts(src, dst, counts, n):
    """Histogram of sampled graphs (bit t = pair t of oracle.pair_list) plus a
    final cell for samples with an invalid edge (self-loop, duplicate, bad id)."""
    index = {pq: t for t, pq in enumerate(oracle.pair_list(n))}
    hist = np.zeros((1 << len(index)) + 1)
    pos = 0
    for c in counts:
        code, ok = 0, True
        for e in range(pos, pos + int(c)):
            u, v = int(src[e]), int(dst[e])
            key = (min(u, v), max(u, v))
            if key not in index or (code >> index[key]) & 1:
                ok = False
                break
            code |= 1 << index[key]
        hist[code if ok else -1] += 1
        pos += int(c)
    return hist


def enumeration_pvalue(model, x, y=None, *, samples=40000, seg_target=1 << 30, flags=0, seed=11, lib=None,
                       sampler="mh"):
    """Chi-square p-value of the sampled graph law against exact enumeration."""
    n = len(x)
    alpha = alpha_of(x)
    beta = None if y is None else alpha_of(y)
    exact, _ = oracle.graph_probabilities(model, alpha, beta)
    if sampler == "mh":
        src, dst, _, counts, _ = oracle.mh_sample(model, x, y, seed=seed, num_samples=samples,
                                                  seg_target=seg_target, flags=flags, lib=lib)
    else:
        parts = [oracle.bf_sample(model, x, y, seed=seed, sample=s, lib=lib) for s in range(samples)]
        src = np.concatenate([p[0] for p in parts])
        dst = np.concatenate([p[1] for p in parts])
        counts = np.array([len(p[0]) for p in parts])
    hist = graph_code_counts(src, dst, counts, n)
    if hist[-1] > 0:
        return 0.0
    return chi2_pvalue(hist[:-1], exact * samples)


def weight_pvalue(x, y, *, samples=40000, seg_target=1 << 30, flags=0, seed=12, lib=None):
    """Smallest chi-square p-value over pairs of the weights given an edge
    against Eq. 4, P(w) = r^(w-1) (1 - r), with r = exp(-beta_u - beta_v)."""
    beta = alpha_of(y)
    src, dst, w, counts, _ = oracle.mh_sample(oracle.UECM, x, y, seed=seed, num_samples=samples,
                                              seg_target=seg_target, flags=flags, lib=lib)
    if np.any(w < 1):
        return 0.0
    worst = 1.0
    n = len(x)
    for (u, v) in oracle.pair_list(n):
        sel = ((src == u) & (dst == v)) | ((src == v) & (dst == u))
        ws = w[sel]
        if len(ws) < 200:
            continue
        r = math.exp(-beta[u] - beta[v])
        kmax = max(2, int(math.log(5.0 / len(ws)) / math.log(r)) if r > 0 else 2)
        obs = [np.sum(ws == k) for k in range(1, kmax + 1)] + [np.sum(ws > kmax)]
        exp = [len(ws) * r ** (k - 1) * (1 - r) for k in range(1, kmax + 1)] + [len(ws) * r ** kmax]
        worst = min(worst, chi2_pvalue(obs, exp))
    return worst


def marginal_zmax(model, x, y=None, *, samples=20000, seg_target=1 << 30, flags=0, seed=13, lib=None,
                  law=None):
    """Largest |z| of per-pair edge frequencies against a closed-form law."""
    n = len(x)
    alpha = alpha_of(x)
    beta = None if y is None else alpha_of(y)
    if law is None:
        law = (lambda u, v: p_ubcm_alpha(alpha, u, v)) if model == oracle.UBCM else \
            (lambda u, v: p_uecm_alpha(alpha, beta, u, v))
    src, dst, _, counts, _ = oracle.mh_sample(model, x, y, seed=seed, num_samples=samples, seg_target=seg_target,
                                              flags=flags, lib=lib)
    lo, hi = np.minimum(src, dst).astype(np.int64), np.maximum(src, dst).astype(np.int64)
    freq = np.bincount(lo * n + hi, minlength=n * n).reshape(n, n)
    zmax = 0.0
    for (u, v) in oracle.pair_list(n):
        p = law(u, v)
        sd = math.sqrt(max(p * (1 - p) / samples, 1e-300))
        zmax = max(zmax, abs(freq[u, v] / samples - p) / sd)
    return zmax
