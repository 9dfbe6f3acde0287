"""Skip decisions near integer boundaries and at large x_i x_j (GPU).

The fast decision levels of the walk estimate t = E / lambda with
lambda = ln(1 + z), while the canonical t divides by log1p(-fl(q)); the two
differ by a relative z 2^-52 / ln(1 + z), which grows with z = x_i x_j (or
A / (1 - c)).  The planted cases of tests/golden/boundary_cases.json put a
draw where the two straddle an integer, for z from 2^11 to about 2^30, and
draws within 2 ulp of an integer (boundary draws, which are counted).  The
CUDA sampler must reproduce the oracle on all of them, through the single,
FP64-only and batched calls, and count the boundary draws as the oracle does.
"""
import numpy as np
import pytest
import torch

import oracle
from parity import check_sample
from test_boundary_cases import CASES, ids, planted_edge
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300.ensemble import Ensemble
from paper_2509_13230_gb300.sampler import Sampler

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def coo(res):
    return (res.src.cpu().numpy(), res.dst.cpu().numpy(), None if res.w is None else res.w.cpu().numpy(),
            np.asarray(res.counts))


@pytest.mark.parametrize("fp64_only", [False, True])
@pytest.mark.parametrize("case", CASES, ids=ids)
def test_planted_case_matches_oracle(case, fp64_only, cuda_lib):
    c, x, y = case
    res = Sampler(c["model"], dev(x), dev(y), num_samples=1, sample_begin=c["sample"], seg_target=32,
                  fp64_only=fp64_only).run()
    same, stats = check_sample(coo(res), c["model"], x, y, num_samples=1, seg_target=32,
                               sample_begin=c["sample"])
    if c["kind"] == "q_rounding":
        # not a boundary draw: the sample must be the oracle's, not the one ln(1 + z) gives
        u, v = planted_edge(c, x)
        src, dst = res.src.cpu().numpy(), res.dst.cpu().numpy()
        assert same and bool(np.any((src == u) & (dst == v))) == c["canonical_edge"]
    assert int(res.stats[nat.MH_STAT_BOUNDARY]) == int(stats[3]) == c["boundary_draws"]
    assert int(res.stats[nat.MH_STAT_PROPOSALS]) == int(stats[0])


def test_planted_cases_batched(cuda_lib):
    # each planted network in a batched wave of its own sample index
    for c, x, y in CASES:
        if c["kind"] != "q_rounding":
            continue
        ens = Ensemble([(c["model"], dev(x), dev(y), 0)], num_samples=1, sample_begin=c["sample"], seg_target=32,
                       layout="coo", capacity=1 << 10)
        got = []
        ens.sample(on_wave=lambda w: got.extend(a.cpu().numpy() if a is not None else None for a in w.coo(0)))
        gs, gd, gw = got
        same, _ = check_sample((gs, gd, gw if c["model"] == UECM else None, np.array([len(gs)])), c["model"], x, y,
                               num_samples=1, seg_target=32, sample_begin=c["sample"])
        assert same


def hub_network(model, seed, n=3000, hubs=40):
    """Hubs of x log-uniform on [10^5, 10^7] against leaves of x = e^N(-3.5, 1.2):
    hub-leaf products z from about 2^10 to 2^26, hub-hub products 2^33 to 2^46."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.normal(-3.5, 1.2, n))
    x[rng.choice(n, hubs, replace=False)] = np.exp(rng.uniform(np.log(1e5), np.log(1e7), hubs))
    y = rng.uniform(0.3, 0.9, n) if model == UECM else None
    return x, y


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_hubs_large_products_bit_exact(model, cuda_lib):
    x, y = hub_network(model, seed=31 + model)
    num_samples = 48
    res = Sampler(model, dev(x), dev(y), num_samples=num_samples, seg_target=16).run()
    same, stats = check_sample(coo(res), model, x, y, num_samples=num_samples, seg_target=16)
    assert same
    assert int(res.stats[nat.MH_STAT_PROPOSALS]) == int(stats[0])
    assert int(res.stats[nat.MH_STAT_BOUNDARY]) == int(stats[3])
    # the hub rows alone make millions of draws at z >= 2^16
    assert int(stats[0]) > 2_000_000
