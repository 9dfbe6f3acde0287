"""Chung-Lu law in the oracle (CPU): p_ij = min(1, x_i x_j), the expected edge
multiplicity k_i k_j / 2M of Sec. 2.1 read as a probability, sampled by the
Miller-Hagberg walk of Sec. 2.3 (q <- p_ij after every candidate) and by brute
force.  Pinned like the other models: exact enumeration of all graphs on four
nodes (including pairs with x_i x_j > 1, whose edge is certain), per-pair
frequencies against the law, and the equal-fitness case, which is G(N, x^2)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle_pins import chi2_pvalue, enumeration_pvalue, marginal_zmax

P_MIN = 1e-4
Z_MAX = 4.5

CL_CASES = [
    np.array([1.8, 0.9, 0.5, 0.05]),   # x_0 x_1 > 1: p = 1 there
    np.array([0.6, 0.6, 0.6, 0.3]),    # ties in the sort key
    np.array([0.2, 3.0, 0.01, 0.4]),   # input not in sorted order
]


@pytest.mark.parametrize("case", range(len(CL_CASES)))
@pytest.mark.parametrize("T", [1 << 30, 2])
def test_chunglu_walk_enumeration(case, T):
    assert enumeration_pvalue(oracle.CL, CL_CASES[case], seg_target=T) > P_MIN


def test_chunglu_bruteforce_enumeration():
    assert enumeration_pvalue(oracle.CL, CL_CASES[0], samples=20000, sampler="bf") > P_MIN


def test_chunglu_enumeration_rejects_the_ubcm_law():
    # the UBCM walk on the same x (p = z / (1 + z)) must fail the Chung-Lu law
    x = CL_CASES[0]
    alpha = -np.log(x)
    exact, _ = oracle.graph_probabilities(oracle.CL, alpha)
    src, dst, _, counts, _ = oracle.mh_sample(oracle.UBCM, x, num_samples=40000, seed=11)
    from oracle_pins import graph_code_counts
    hist = graph_code_counts(src, dst, counts, len(x))
    assert chi2_pvalue(hist[:-1], exact * 40000) < 1e-12


@pytest.mark.parametrize("T", [1 << 30, 3])
def test_chunglu_marginals(T):
    rng = np.random.default_rng(21)
    x = np.exp(rng.normal(-0.8, 1.0, 12))
    assert marginal_zmax(oracle.CL, x, seg_target=T, law=lambda u, v: min(1.0, x[u] * x[v])) < Z_MAX


@pytest.mark.parametrize("T", [1 << 30, 2])
def test_chunglu_equal_fitness_is_erdos_renyi(T):
    n, xv, S = 30, 0.4, 6000
    _, _, _, counts, _ = oracle.mh_sample(oracle.CL, np.full(n, xv), seed=5, num_samples=S, seg_target=T)
    m = n * (n - 1) // 2
    p = xv * xv
    expected = stats.binom.pmf(np.arange(m + 1), m, p) * S
    observed = np.bincount(counts, minlength=m + 1)[: m + 1]
    assert chi2_pvalue(observed, expected) > P_MIN


def test_chunglu_segment_table_equals_the_ubcm_table():
    # the partition's cost min(1, x_i x_j) is the Chung-Lu probability itself
    rng = np.random.default_rng(22)
    x = np.exp(rng.normal(-2.0, 1.5, 500))
    a = oracle.partition(oracle.CL, x, seg_target=8)
    b = oracle.partition(oracle.UBCM, x, seg_target=8)
    for key in ("perm", "row", "k", "a", "b"):
        assert np.array_equal(a[key], b[key])
    assert math.isfinite(float(x.sum()))
