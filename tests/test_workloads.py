"""The seeded input generators follow the recipes they state (no GPU): the
shapes, laws and parameters of the synthetic stand-ins for the paper's
networks, and that every generator is reproducible from its seed."""
import numpy as np
import pytest

from paper_2509_13230_gb300 import workloads


def test_lognormal_workloads():
    for make, n, mu, sigma, weighted in ((workloads.ubcm_n1k, 1000, -3.5, 1.0, False),
                                         (workloads.uecm_n20k, 20_000, -4.0, 1.2, True)):
        net = make()
        assert net.n == n and net.model == (1 if weighted else 0)
        z = np.log(net.x)
        se = sigma / np.sqrt(n)
        assert abs(z.mean() - mu) < 5 * se
        assert abs(z.std() - sigma) < 5 * sigma / np.sqrt(2 * n)
        if weighted:
            assert net.y.min() >= 0.3 and net.y.max() < 0.9
            assert abs(net.y.mean() - 0.6) < 5 * 0.6 / np.sqrt(12 * n)  # 5 standard errors of U(0.3, 0.9)
        again = make()
        assert np.array_equal(again.x, net.x)


def test_capped_pareto_law():
    n, c = 200_000, 6.285e-4
    x = workloads.pareto_ubcm(n, c, seed=3).x
    assert x.min() >= c and x.max() <= 50.0
    for t in (10 * c, 100 * c, 1000 * c):  # P(x > t) = (c / t)^1.1 below the cap
        p = (c / t) ** 1.1
        assert abs((x > t).mean() - p) < 5 * np.sqrt(p * (1 - p) / n)
    assert workloads.ubcm_pareto_n1m(n).x.shape == (n,)
    net = workloads.pareto_uecm(1000, c, seed=9)
    assert np.array_equal(net.x, workloads.pareto_ubcm(1000, c, seed=9).x)
    assert net.y.min() >= 0.3 and net.y.max() < 0.9


def test_ensemble_shapes_and_models():
    nets = workloads.ensemble_128()
    assert len(nets) == 128
    sizes = np.array([net.n for net in nets])
    assert sizes.min() >= 1000 and sizes.max() < 1_000_000
    assert sizes.sum() == 20_048_423  # the node count the ensemble's measurements state
    assert all(net.model == 0 for net in nets[:64]) and all(net.model == 1 for net in nets[64:])
    assert abs(np.log(sizes).mean() - np.log(10**4.5)) < 4 * np.log(1000) / np.sqrt(12 * 128)
    lognormal = workloads.ensemble_128(num_networks=4, n_lo=1000, n_hi=2000, fitness="lognormal")
    assert [net.n for net in lognormal] == [net.n for net in workloads.ensemble_128(4, 1000, 2000)]


def test_degree_strength_targets():
    k, s = workloads.degree_strength_targets()
    assert k.shape == (200_000,) and s.shape == k.shape
    assert k.min() >= 2 and k.max() <= 2000 and np.all(k == np.round(k))
    assert abs(k.mean() - 4.6) < 0.05  # the mean degree of the fit-then-sample workload
    ratio = s / k
    assert ratio.min() >= 1.0 and ratio.max() < 5.0
    # discrete power law P(k) ~ k^-2.5 on [2, 2000]: the exponent's maximum-likelihood
    # estimate, -a sum ln k_i - n ln Z(a) maximised over a by golden-section search
    support = np.arange(2, 2001, dtype=np.float64)
    sum_log = np.log(k).sum()

    def neg_loglik(a):
        return a * sum_log + k.size * np.log(np.sum(support ** -a))

    lo, hi = 1.5, 3.5
    g = (np.sqrt(5.0) - 1.0) / 2.0
    for _ in range(80):
        m1, m2 = hi - g * (hi - lo), lo + g * (hi - lo)
        if neg_loglik(m1) < neg_loglik(m2):
            hi = m2
        else:
            lo = m1
    alpha = 0.5 * (lo + hi)
    assert abs(alpha - 2.5) < 0.02
    k2, s2 = workloads.degree_strength_targets()
    assert np.array_equal(k, k2) and np.array_equal(s, s2)


def test_directed_and_bipartite_workloads():
    x_out, y_out, x_in, y_in = workloads.directed_uecm_n20k()
    for a in (x_out, y_out, x_in, y_in):
        assert a.shape == (20_000,)
    assert not np.array_equal(x_out, x_in)
    for y in (y_out, y_in):
        assert y.min() >= 0.3 and y.max() < 0.9
    xp, xm = workloads.bipartite_ubcm_pareto()
    assert xp.shape == (200_000,) and xm.shape == (20_000,)
    assert xp.min() >= 2e-3 and xm.min() >= 0.0125 and max(xp.max(), xm.max()) <= 50.0
    # about 16 expected edges per + node: sum_j p_ij on a sample of rows
    rows = xp[:200]
    deg = (rows[:, None] * xm[None, :] / (1.0 + rows[:, None] * xm[None, :])).sum(axis=1)
    assert 10.0 < deg.mean() < 25.0


@pytest.mark.parametrize("name", sorted(workloads.WORKLOADS))
def test_registered_workloads_build(name):
    spec = workloads.WORKLOADS[name]
    if "n1m" in name:
        pytest.skip("the N = 10^6 network is covered by the Pareto law test")
    net = spec["make"]()
    assert net.n > 0 and spec["samples"] >= 1
