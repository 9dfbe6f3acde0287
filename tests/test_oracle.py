"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import ctypes
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from tests.oracle_pins import (alpha_of, chi2_pvalue, enumeration_pvalue, marginal_zmax, p_ubcm_alpha,
                               p_uecm_alpha, weight_pvalue)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P_MIN = 1e-4   # chi-square threshold; every seed is fixed, so a pass is reproducible
Z_MAX = 4.5

# ---------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator (an independent library).
# cuRAND's host Philox maps output block B = value_index / 4 to the counter
# {B / 65536 (64-bit across words 0,1), B mod 65536, 0} with key = seed.
# ---------------------------------------------------------------------------
_CURAND = "/usr/local/cuda/lib64/libcurand.so"


def _curand_block(seed, block):
    lib = ctypes.CDLL(_CURAND)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * block)) == 0
        out = np.zeros(4, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.skipif(not os.path.exists(_CURAND), reason="cuRAND not installed")
@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("block", [0, 1, 7, 65535, 65536 * 5 + 3, (1 << 48) + 65536 * 3 + 9,
                                   65536 * 0xFFFFFFFF + 65535])
def test_philox_matches_curand(seed, block):
    hi, w2 = divmod(block, 65536)
    ctr = [hi & 0xFFFFFFFF, hi >> 32, w2, 0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    assert list(oracle.philox(ctr, key)) == list(_curand_block(seed, block))


def test_philox_zero_vector():
    # Philox4x32-10 of the zero counter and key (as cuRAND also returns it).
    assert [hex(v) for v in oracle.philox([0, 0, 0, 0], [0, 0])] == ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c",
                                                                      "0x9b00dbd8"]


# ---------------------------------------------------------------------------
# Node order (Sec. 2.4 step (i)): numpy's stable lexsort is the reference.
# ---------------------------------------------------------------------------
def test_sort_matches_lexsort():
    rng = np.random.default_rng(0)
    for n in [1, 2, 17, 1000, 5000]:
        key = rng.choice(np.exp(rng.normal(-3, 2, max(2, n // 3))), size=n)  # many ties
        perm = oracle.sort_desc(key)
        ref = np.lexsort((np.arange(n), -key))
        assert np.array_equal(perm, ref)


# ---------------------------------------------------------------------------
# Segment table: covers every candidate pair exactly once.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("model", [oracle.UBCM, oracle.UECM])
@pytest.mark.parametrize("T", [2, 5, 32, 1 << 30])
@pytest.mark.parametrize("flags", [0, oracle.BOUND_PAPER])
def test_partition_covers_candidates(model, T, flags):
    rng = np.random.default_rng(1)
    n = 700
    x = np.exp(rng.normal(-1.5, 1.5, n))
    x[:5] = 40.0  # hubs with many unit-cost candidates
    y = rng.uniform(0.2, 0.95, n) if model == oracle.UECM else None
    t = oracle.partition(model, x, y, seg_target=T, flags=flags)
    row, k, a, b = t["row"], t["k"], t["a"], t["b"]
    assert np.all(a < b)
    rows = np.arange(n - 1)
    assert np.array_equal(np.unique(row), rows)
    for i in rows:
        sel = row == i
        assert np.array_equal(k[sel], np.arange(sel.sum()))
        assert a[sel][0] == i + 1 and b[sel][-1] == n
        assert np.array_equal(a[sel][1:], b[sel][:-1])
    if T == 1 << 30:
        assert len(row) == n - 1
    if T == 2:
        assert len(row) > 2 * n


# ---------------------------------------------------------------------------
# Exact law on N = 4: all 2^6 graphs (Eq. 1 / Eq. 3, pairs independent).
# ---------------------------------------------------------------------------
UBCM_CASES = [
    np.array([3.0, 0.8, 0.5, 0.05]),      # x_0 x_1 > 1: unit-probability region
    np.array([0.4, 0.4, 0.4, 0.2]),       # ties in the sort key
    np.array([0.2, 5.0, 0.01, 2.0]),      # input not in sorted order
]


@pytest.mark.parametrize("case", range(len(UBCM_CASES)))
@pytest.mark.parametrize("T,flags", [(1 << 30, 0), (2, 0), (2, oracle.INIT_PREV), (1 << 30, oracle.INIT_PREV)])
def test_ubcm_enumeration(case, T, flags):
    assert enumeration_pvalue(oracle.UBCM, UBCM_CASES[case], seg_target=T, flags=flags) > P_MIN


UECM_X = np.array([2.0, 0.7, 1.3, 0.1])
UECM_Y = np.array([0.3, 0.85, 0.6, 0.9])


@pytest.mark.parametrize("T,flags", [(1 << 30, 0), (2, 0), (1 << 30, oracle.BOUND_PAPER), (2, oracle.BOUND_PAPER),
                                     (2, oracle.INIT_PREV)])
def test_uecm_enumeration_and_weights(T, flags):
    assert enumeration_pvalue(oracle.UECM, UECM_X, UECM_Y, seg_target=T, flags=flags) > P_MIN
    assert weight_pvalue(UECM_X, UECM_Y, seg_target=T, flags=flags) > P_MIN


def test_bruteforce_enumeration():
    assert enumeration_pvalue(oracle.UBCM, UBCM_CASES[0], samples=20000, sampler="bf") > P_MIN
    assert enumeration_pvalue(oracle.UECM, UECM_X, UECM_Y, samples=20000, sampler="bf") > P_MIN


# ---------------------------------------------------------------------------
# Per-pair marginals on a larger network against the closed forms.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T", [1 << 30, 3])
def test_marginals_ubcm(T):
    rng = np.random.default_rng(2)
    x = np.exp(rng.normal(-0.8, 1.3, 12))
    assert marginal_zmax(oracle.UBCM, x, seg_target=T) < Z_MAX


@pytest.mark.parametrize("T,flags", [(1 << 30, 0), (3, 0), (3, oracle.BOUND_PAPER)])
def test_marginals_uecm(T, flags):
    rng = np.random.default_rng(3)
    x = np.exp(rng.normal(-0.5, 1.2, 12))
    y = rng.uniform(0.1, 0.9, 12)
    assert marginal_zmax(oracle.UECM, x, y, seg_target=T, flags=flags) < Z_MAX


# ---------------------------------------------------------------------------
# Special cases that reduce to textbook laws.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T", [1 << 30, 2])
def test_equal_fitness_is_erdos_renyi(T):
    """All x equal: the UBCM is G(N, p) (Sec. 2.3), so the edge count is
    Binomial(N(N-1)/2, p)."""
    n, xv, S = 30, 0.3, 6000
    x = np.full(n, xv)
    _, _, _, counts, _ = oracle.mh_sample(oracle.UBCM, x, seed=5, num_samples=S, seg_target=T)
    m = n * (n - 1) // 2
    p = xv * xv / (1 + xv * xv)
    ks = np.arange(m + 1)
    expected = stats.binom.pmf(ks, m, p) * S
    observed = np.bincount(counts, minlength=m + 1)[: m + 1]
    assert chi2_pvalue(observed, expected) > P_MIN


def test_equal_strength_parameter_reduces_to_ubcm():
    """All y = y0: Eq. 3 becomes Eq. 1 with x' = x y0 / sqrt(1 - y0^2)."""
    rng = np.random.default_rng(4)
    n, y0 = 10, 0.6
    x = np.exp(rng.normal(-0.3, 1.0, n))
    alpha_p = alpha_of(x * y0 / math.sqrt(1 - y0 * y0))
    z = marginal_zmax(oracle.UECM, x, np.full(n, y0), law=lambda u, v: p_ubcm_alpha(alpha_p, u, v))
    assert z < Z_MAX


# ---------------------------------------------------------------------------
# Degree and strength preservation in expectation (Sec. 3, Fig. 3B / 4B).
# ---------------------------------------------------------------------------
def test_expected_degree_and_strength_invariants():
    rng = np.random.default_rng(6)
    n, S = 60, 10000
    x = np.exp(rng.normal(-1.0, 1.5, n))
    y = rng.uniform(0.2, 0.9, n)
    alpha, beta = alpha_of(x), alpha_of(y)
    P = np.zeros((n, n))
    R = np.zeros((n, n))
    for u in range(n):
        for v in range(n):
            if u != v:
                P[u, v] = p_uecm_alpha(alpha, beta, u, v)
                R[u, v] = math.exp(-beta[u] - beta[v])
    src, dst, w, counts, _ = oracle.mh_sample(oracle.UECM, x, y, seed=7, num_samples=S, seg_target=4)
    deg = np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    stren = np.bincount(src, weights=w, minlength=n) + np.bincount(dst, weights=w, minlength=n)
    k_exp = P.sum(1)
    m = P / np.where(R < 1, 1 - R, 1)
    s_exp = m.sum(1)
    k_sd = np.sqrt((P * (1 - P)).sum(1) / S)
    w2 = P * (1 + R) / (1 - R) ** 2          # E[w^2] = p (1 + r) / (1 - r)^2 (Eq. 4)
    s_sd = np.sqrt((w2 - m * m).sum(1) / S)
    assert np.all(np.abs(deg / S - k_exp) <= 4.5 * k_sd)
    assert np.all(np.abs(stren / S - s_exp) <= 4.5 * s_sd)


# ---------------------------------------------------------------------------
# Expected degrees / strengths and their gradient.
# ---------------------------------------------------------------------------
def test_expected_fwd_closed_forms():
    n = 50
    k, _ = oracle.expected_fwd(oracle.UBCM, np.full(n, 0.7))
    assert np.allclose(k, (n - 1) * 0.49 / 1.49, rtol=1e-14)
    # two groups: m nodes at a, n - m at b
    m, a, b = 20, 1.7, 0.03
    x = np.r_[np.full(m, a), np.full(n - m, b)]
    k, _ = oracle.expected_fwd(oracle.UBCM, x)
    ka = (m - 1) * a * a / (1 + a * a) + (n - m) * a * b / (1 + a * b)
    kb = m * a * b / (1 + a * b) + (n - m - 1) * b * b / (1 + b * b)
    assert np.allclose(k[:m], ka, rtol=1e-14) and np.allclose(k[m:], kb, rtol=1e-14)
    # UECM, two groups in (x, y)
    ya, yb = 0.8, 0.35
    y = np.r_[np.full(m, ya), np.full(n - m, yb)]
    k, s = oracle.expected_fwd(oracle.UECM, x, y)
    al, be = alpha_of([a, b]), alpha_of([ya, yb])

    def pr(g, h):
        return p_uecm_alpha(al, be, g, h), math.exp(-be[g] - be[h])

    (paa, raa), (pab, rab), (pbb, rbb) = pr(0, 0), pr(0, 1), pr(1, 1)
    assert np.allclose(k[:m], (m - 1) * paa + (n - m) * pab, rtol=1e-13)
    assert np.allclose(s[:m], (m - 1) * paa / (1 - raa) + (n - m) * pab / (1 - rab), rtol=1e-13)
    assert np.allclose(s[m:], m * pab / (1 - rab) + (n - m - 1) * pbb / (1 - rbb), rtol=1e-13)


@pytest.mark.parametrize("model", [oracle.UBCM, oracle.UECM])
def test_expected_bwd_matches_central_differences(model):
    rng = np.random.default_rng(8)
    n = 24
    x = np.exp(rng.normal(-0.5, 1.0, n))
    y = rng.uniform(0.2, 0.9, n) if model == oracle.UECM else None
    gk = rng.normal(size=n)
    gs = rng.normal(size=n) if model == oracle.UECM else None

    def loss(xx, yy):
        k, s = oracle.expected_fwd(model, xx, yy)
        return float(np.dot(gk, k) + (np.dot(gs, s) if s is not None else 0.0))

    gx, gy = oracle.expected_bwd(model, x, y, gk, gs)
    for i in range(n):
        h = 1e-6 * x[i]
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (loss(xp, y) - loss(xm, y)) / (2 * h)
        assert abs(fd - gx[i]) <= 1e-6 * max(1.0, abs(fd))
        if y is not None:
            h = 1e-6 * y[i]
            yp, ym = y.copy(), y.copy()
            yp[i] += h
            ym[i] -= h
            fd = (loss(x, yp) - loss(x, ym)) / (2 * h)
            assert abs(fd - gy[i]) <= 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------------------
# The paper's brute-force cost example (Sec. 2.2).
# ---------------------------------------------------------------------------
def test_bruteforce_cost_example():
    g = json.load(open(os.path.join(GOLDEN, "paper_bf_cost.json")))
    x = np.full(g["n"], 1e-4)
    _, _, _, evals = oracle.bf_sample(oracle.UBCM, x, seed=1)
    assert abs(evals - g["evaluations_approx"]) <= g["relative_tolerance"] * g["evaluations_approx"]


def test_pareto_scale_matches_calibration():
    from paper_2509_13230_gb300 import workloads
    g = json.load(open(os.path.join(GOLDEN, "pareto_scale.json")))
    assert workloads.PARETO_SCALE_N1M == g["scale"]
    assert abs(g["mean_degree"] - 20.0) < 0.05


def test_pareto_scale_grid_matches_calibration():
    from paper_2509_13230_gb300 import workloads
    g = json.load(open(os.path.join(GOLDEN, "pareto_scale_grid.json")))
    assert list(workloads.PARETO_SCALE_GRID_N) == g["n"]
    assert list(workloads.PARETO_SCALE_GRID) == g["scale"]
    assert max(abs(k - 20.0) for k in g["mean_degree"]) < 0.05
    assert workloads.pareto_scale(1_000_000) == workloads.PARETO_SCALE_N1M
    # between grid points: a fresh oracle sample at an off-grid size lands near 20
    n = 7000
    net = workloads.pareto_ubcm(n, workloads.pareto_scale(n), seed=3)
    _, _, _, counts, _ = oracle.mh_sample(oracle.UBCM, net.x, seed=0, num_samples=1, seg_target=1 << 30)
    assert abs(2.0 * counts[0] / n - 20.0) < 1.5


@pytest.mark.parametrize("model", [oracle.UBCM, oracle.UECM])
def test_jacobian_diagonal_matches_central_differences(model):
    """Each entry against a central difference of the expected sums with only
    node i's own parameter moved (Sec. 2.2, Sec. 2.5)."""
    rng = np.random.default_rng(19)
    n = 24
    x = np.exp(rng.normal(-0.5, 1.0, n))
    y = rng.uniform(0.2, 0.9, n) if model == oracle.UECM else None
    diag = oracle.expected_jacobian_diag(model, x, y)
    for i in range(n):
        h = 1e-6 * x[i]
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        (kp, sp), (km, sm) = (oracle.expected_fwd(model, xx, y, rows=[i]) for xx in (xp, xm))
        fd = [(kp[0] - km[0]) / (2 * h)] + ([(sp[0] - sm[0]) / (2 * h)] if y is not None else [])
        got = [diag[0][i]] + ([diag[2][i]] if y is not None else [])
        for f, g in zip(fd, got):
            assert abs(f - g) <= 1e-6 * max(1.0, abs(f)), (i, f, g)
        if y is None:
            continue
        h = 1e-6 * y[i]
        yp, ym = y.copy(), y.copy()
        yp[i] += h
        ym[i] -= h
        (kp, sp), (km, sm) = (oracle.expected_fwd(model, x, yy, rows=[i]) for yy in (yp, ym))
        for f, g in (((kp[0] - km[0]) / (2 * h), diag[1][i]), ((sp[0] - sm[0]) / (2 * h), diag[3][i])):
            assert abs(f - g) <= 1e-6 * max(1.0, abs(f)), (i, f, g)


def test_jacobian_diagonal_rows_and_ubcm_closed_form():
    # the UBCM entry is sum_j x_j / (1 + x_i x_j)^2; rows= picks the same values
    rng = np.random.default_rng(20)
    x = np.exp(rng.normal(-1.0, 1.0, 40))
    (d,) = oracle.expected_jacobian_diag(oracle.UBCM, x)
    i = 7
    j = np.arange(40) != i
    assert d[i] == pytest.approx(np.sum(x[j] / (1.0 + x[i] * x[j]) ** 2), rel=1e-13)
    (dr,) = oracle.expected_jacobian_diag(oracle.UBCM, x, rows=[3, 7])
    assert dr[1] == d[7] and dr[0] == d[3]
