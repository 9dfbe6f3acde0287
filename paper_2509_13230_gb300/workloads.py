"""Seeded synthetic inputs for the sampler and the fitting path.

This module draws node parameters only; it holds none of the sampling or
expected-degree arithmetic, so the CUDA library and the CPU oracle can both
consume its output.  The paper's 93 unweighted and 10 weighted empirical
networks (Sec. 3) are not available; these heavy-tailed synthetic fitness
sequences stand in for them.

Every generator uses numpy's PCG64 with a fixed seed, so a workload is
identified by its name and sizes alone.  Parameters are x_i = exp(-alpha_i)
and y_i = exp(-beta_i) in the paper's alpha/beta notation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Scale c of the Pareto fitness workload, chosen so the mean expected degree
# (1/N) sum_i sum_{j != i} p_ij is 20 at N = 10^6.  Written by
# oracle/calibrate_scale.py (bisection on the oracle's exact expected degrees).
PARETO_SCALE_N1M = 6.285e-4

# The same calibration over sizes N = 10^(3 + k/4), k = 0..12 (written by
# oracle/calibrate_ensemble_scale.py); sizes in between interpolate log c
# linearly in log N.
PARETO_SCALE_GRID_N = (1000, 1778, 3162, 5623, 10000, 17783, 31623, 56234, 100000, 177828, 316228, 562341, 1000000)
PARETO_SCALE_GRID = (0.03231, 0.021, 0.01528, 0.01048, 0.007334, 0.005434, 0.004009, 0.002909, 0.002062, 0.001531, 0.001151, 0.0008664, 0.0006285)


@dataclass(frozen=True)
class Network:
    model: int                  # 0 = UBCM (Eq. 1), 1 = UECM (Eq. 3)
    x: np.ndarray               # float64[N], x_i = exp(-alpha_i) >= 0
    y: np.ndarray | None        # float64[N] in [0, 1) for UECM, else None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def lognormal_ubcm(n: int, mu: float, sigma: float, seed: int) -> Network:
    """x = exp(z), z ~ Normal(mu, sigma)."""
    rng = np.random.default_rng(seed)
    return Network(0, np.exp(rng.normal(mu, sigma, n)), None)


def lognormal_uecm(n: int, mu: float, sigma: float, y_lo: float, y_hi: float, seed: int) -> Network:
    """x = exp(z), z ~ Normal(mu, sigma); y ~ Uniform(y_lo, y_hi)."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.normal(mu, sigma, n))
    y = rng.uniform(y_lo, y_hi, n)
    return Network(1, x, y)


def pareto_ubcm(n: int, scale: float, x_max: float = 50.0, tail: float = 1.1, seed: int = 3) -> Network:
    """x = min(scale * u^(-1/tail), x_max), u ~ Uniform(0, 1): a Pareto tail
    whose degree exponent is 1 + tail (2.1 for tail = 1.1)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, n)
    u = np.where(u > 0.0, u, np.finfo(np.float64).tiny)
    return Network(0, np.minimum(scale * u ** (-1.0 / tail), x_max), None)


def pareto_scale(n: int) -> float:
    """Scale c giving the capped Pareto fitness a mean expected degree of
    about 20 at size n (clamped to the calibrated range [10^3, 10^6])."""
    if n in PARETO_SCALE_GRID_N:
        return PARETO_SCALE_GRID[PARETO_SCALE_GRID_N.index(n)]
    return float(np.exp(np.interp(np.log(n), np.log(PARETO_SCALE_GRID_N), np.log(PARETO_SCALE_GRID))))


def pareto_uecm(n: int, scale: float, y_lo: float = 0.3, y_hi: float = 0.9, x_max: float = 50.0, tail: float = 1.1,
                seed: int = 3) -> Network:
    """The Pareto fitness of pareto_ubcm with y ~ Uniform(y_lo, y_hi)."""
    x = pareto_ubcm(n, scale, x_max=x_max, tail=tail, seed=seed).x
    y = np.random.default_rng(seed + 7919).uniform(y_lo, y_hi, n)
    return Network(1, x, y)


# --------------------------------------------------------------------------
# The five named workloads.
# --------------------------------------------------------------------------
def ubcm_n1k() -> Network:
    """Unweighted, N = 1,000, z ~ N(-3.5, 1.0); sampled 100 times, COO int32."""
    return lognormal_ubcm(1000, -3.5, 1.0, seed=1)


def uecm_n20k() -> Network:
    """Weighted, N = 20,000, z ~ N(-4.0, 1.2), y ~ U(0.3, 0.9); sampled 10 times,
    COO int32 plus int32 weights."""
    return lognormal_uecm(20_000, -4.0, 1.2, 0.3, 0.9, seed=2)


def ubcm_pareto_n1m(n: int = 1_000_000) -> Network:
    """Unweighted, N = 10^6 Pareto fitness (exponent 2.1) capped at 50, mean
    expected degree about 20; one sample, CSR int64 offsets / int32 indices."""
    return pareto_ubcm(n, PARETO_SCALE_N1M, seed=3)


def ensemble_128(num_networks: int = 128, n_lo: int = 1_000, n_hi: int = 1_000_000, seed: int = 4,
                 fitness: str = "pareto"):
    """Batched ensemble: sizes log-uniform in [n_lo, n_hi], first half UBCM and
    second half UECM (y ~ U(0.3, 0.9)); 64 samples each.  fitness "pareto":
    the capped Pareto law of the N = 10^6 workload with its scale c(N)
    calibrated per size (mean expected degree about 20 for the UBCM half);
    "lognormal": z ~ N(-4.0, 1.2) as in the N = 20,000 workload."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), num_networks))).astype(np.int64)
    nets = []
    for t, n in enumerate(sizes):
        uecm = t >= num_networks // 2
        if fitness == "pareto":
            c = pareto_scale(int(n))
            nets.append(pareto_uecm(int(n), c, seed=10_000 + t) if uecm else pareto_ubcm(int(n), c, seed=10_000 + t))
        elif uecm:
            nets.append(lognormal_uecm(int(n), -4.0, 1.2, 0.3, 0.9, seed=10_000 + t))
        else:
            nets.append(lognormal_ubcm(int(n), -4.0, 1.2, seed=10_000 + t))
    return nets


def degree_strength_targets(n: int = 200_000, exponent: float = 2.5, k_min: int = 2, k_max: int = 2000,
                            seed: int = 5):
    """Targets for fitting: k ~ discrete power law P(k) ~ k^-exponent on
    [k_min, k_max]; s_i = k_i * wbar_i with wbar_i ~ Uniform(1, 5)."""
    rng = np.random.default_rng(seed)
    support = np.arange(k_min, k_max + 1, dtype=np.float64)
    pk = support ** (-exponent)
    pk /= pk.sum()
    k = rng.choice(support, size=n, p=pk)
    wbar = rng.uniform(1.0, 5.0, n)
    return k, k * wbar


def directed_uecm_n20k(n: int = 20_000, seed: int = 6):
    """Directed weighted network (Sec. 2.6): out- and in-parameters of N =
    20,000 nodes, x = exp(z), z ~ N(-4.0, 1.2), y ~ U(0.3, 0.9) on both sides.
    Returns (x_out, y_out, x_in, y_in)."""
    rng = np.random.default_rng(seed)
    return (np.exp(rng.normal(-4.0, 1.2, n)), rng.uniform(0.3, 0.9, n), np.exp(rng.normal(-4.0, 1.2, n)),
            rng.uniform(0.3, 0.9, n))


def bipartite_ubcm_pareto(n_plus: int = 200_000, n_minus: int = 20_000, seed: int = 7):
    """Bipartite unweighted network (Sec. 2.6), e.g. users x items: capped
    Pareto fitness on both sides, scaled so that a + node has about 16
    edges (3.3 M per sample).  Returns (x_plus, x_minus)."""
    rng = np.random.default_rng(seed)
    up = np.where((u := rng.uniform(0.0, 1.0, n_plus)) > 0.0, u, np.finfo(np.float64).tiny)
    um = np.where((u := rng.uniform(0.0, 1.0, n_minus)) > 0.0, u, np.finfo(np.float64).tiny)
    xp = np.minimum(2e-3 * up ** (-1.0 / 1.1), 50.0)
    xm = np.minimum(0.0125 * um ** (-1.0 / 1.1), 50.0)
    return xp, xm


WORKLOADS = {
    "ubcm_n1k_x100": dict(make=ubcm_n1k, samples=100, output="coo"),
    "uecm_n20k_x10": dict(make=uecm_n20k, samples=10, output="coo"),
    "ubcm_pareto_n1m_x1": dict(make=ubcm_pareto_n1m, samples=1, output="csr"),
}
