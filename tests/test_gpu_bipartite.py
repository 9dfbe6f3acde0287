"""Bipartite and directed networks (mh_sample_bipartite) against the CPU
oracle (GPU).  Edge lists, weights, per-sample counts and the proposal, edge
and segment counters bit-exact; the allowance is the one of the one-set
tests (a draw the oracle flags as an integer-boundary draw)."""
import numpy as np
import pytest
import torch

import oracle
from parity import check_bip_sample
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300.sampler import BipartiteSampler

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def sets(n_plus, n_minus, seed, uecm, hubs=2):
    rng = np.random.default_rng(seed)
    xp, xm = np.exp(rng.normal(-3.0, 1.4, n_plus)), np.exp(rng.normal(-3.0, 1.4, n_minus))
    if n_plus > 10:
        xp[rng.choice(n_plus, hubs, replace=False)] = rng.uniform(5, 30, hubs)
        xp[5:12] = xp[3]  # ties
    if n_minus > 10:
        xm[rng.choice(n_minus, hubs, replace=False)] = rng.uniform(5, 30, hubs)
    yp = rng.uniform(0.1, 0.95, n_plus) if uecm else None
    ym = rng.uniform(0.1, 0.95, n_minus) if uecm else None
    return xp, yp, xm, ym


def check(model, xp, yp, xm, ym, *, directed=False, num_samples=3, seg_target=32, seed=0, network_id=0,
          sample_begin=0, layout="both", **kw):
    s = BipartiteSampler(model, dev(xp), dev(yp), dev(xm), dev(ym), directed=directed, num_samples=num_samples,
                         seed=seed, network_id=network_id, sample_begin=sample_begin, seg_target=seg_target,
                         layout=layout, **kw)
    res = s.run()
    kw_o = dict(directed=directed, seed=seed, network_id=network_id, sample_begin=sample_begin,
                num_samples=num_samples, seg_target=seg_target)
    if layout in ("coo", "both"):
        got = (res.src.cpu().numpy(), res.dst.cpu().numpy(), None if res.w is None else res.w.cpu().numpy(),
               res.counts)
        same, (src, dst, w, counts), stats = check_bip_sample(got, model, xp, yp, xm, ym, **kw_o)
        if not same:  # every differing segment holds an oracle boundary draw
            return res, stats
        assert int(res.stats[nat.MH_STAT_PROPOSALS]) == int(stats[0])
        assert int(res.stats[nat.MH_STAT_EDGES]) == int(stats[1])
        assert int(res.stats[nat.MH_STAT_SEGMENTS]) == int(stats[2])
        assert int(res.stats[nat.MH_STAT_BOUNDARY]) == int(stats[3])
    else:
        src, dst, w, counts, stats = oracle.bip_sample(model, xp, yp, xm, ym, **kw_o)
    if layout in ("csr", "both"):
        n_plus = len(xp)
        pos = 0
        for smp in range(num_samples):
            c = int(counts[smp])
            ss, dd = src[pos:pos + c], dst[pos:pos + c]
            order = np.argsort(ss, kind="stable")
            off = np.zeros(n_plus + 1, np.int64)
            off[1:] = np.cumsum(np.bincount(ss, minlength=n_plus))
            got_off = res.csr_offsets[smp * (n_plus + 1):(smp + 1) * (n_plus + 1)].cpu().numpy()
            assert np.array_equal(got_off - got_off[0], off)
            a, b = int(got_off[0]), int(got_off[-1])
            assert np.array_equal(res.csr_indices[a:b].cpu().numpy(), dd[order])
            if w is not None:
                assert np.array_equal(res.csr_weights[a:b].cpu().numpy(), w[pos:pos + c][order])
            pos += c
    if directed:
        assert not bool((res.src == res.dst).any())
    return res, stats


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("T", [2, 7, 32, 1 << 30])
def test_bipartite_matches_oracle(model, T):
    xp, yp, xm, ym = sets(3000, 5200, seed=T, uecm=model == UECM)
    check(model, xp, yp, xm, ym, seg_target=T, seed=0x1234ABCD5678, network_id=3, sample_begin=11)


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("T", [2, 32, 1 << 30])
def test_directed_matches_oracle(model, T):
    xo, yo, xi, yi = sets(4100, 4100, seed=100 + T, uecm=model == UECM)
    res, _ = check(model, xo, yo, xi, yi, directed=True, seg_target=T, seed=77)
    assert res.total > 0


@pytest.mark.parametrize("shape", [(1, 1), (1, 5000), (5000, 1), (2, 3), (9000, 40)])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_bipartite_shapes(model, shape):
    xp, yp, xm, ym = sets(*shape, seed=sum(shape), uecm=model == UECM)
    check(model, xp, yp, xm, ym, seg_target=3, num_samples=4)


@pytest.mark.parametrize("n", [1, 2, 3, 17])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_directed_small(model, n):
    # n = 1 has no pair at all; with T = 2 many segments hold only the excluded candidate
    rng = np.random.default_rng(n)
    xo, xi = np.exp(rng.normal(0.5, 1.0, n)), np.exp(rng.normal(0.5, 1.0, n))
    yo = rng.uniform(0.2, 0.9, n) if model == UECM else None
    yi = rng.uniform(0.2, 0.9, n) if model == UECM else None
    res, _ = check(model, xo, yo, xi, yi, directed=True, seg_target=2, num_samples=20)
    if n == 1:
        assert res.total == 0


@pytest.mark.parametrize("directed", [False, True])
def test_bipartite_fp64_only_and_capacity_retry(directed):
    xp, yp, xm, ym = sets(2500, 2500, seed=9, uecm=True)
    check(UECM, xp, yp, xm, ym, directed=directed, fp64_only=True, num_samples=2)
    s = BipartiteSampler(UECM, dev(xp), dev(yp), dev(xm), dev(ym), directed=directed, num_samples=2, capacity=16)
    assert s.call() == nat.MH_ERR_CAPACITY
    res = s.run()
    src, dst, w, counts, _ = oracle.bip_sample(UECM, xp, yp, xm, ym, directed=directed, num_samples=2)
    assert np.array_equal(res.counts, counts)


@pytest.mark.parametrize("bad", ["directed_unequal", "bound_paper", "init_prev"])
def test_bipartite_argument_errors(bad):
    xp, yp, xm, ym = sets(50, 60 if bad == "directed_unequal" else 50, seed=1, uecm=True)
    kw = dict(directed_unequal=dict(directed=True), bound_paper=dict(bound="paper"), init_prev=dict(init="prev"))[bad]
    with pytest.raises(nat.MhError) as e:
        BipartiteSampler(UECM, dev(xp), dev(yp), dev(xm), dev(ym), **kw).run()
    assert e.value.code == nat.MH_ERR_ARG
