"""Symmetric CSR layout (MH_CSR_SYMMETRIC) against the CPU oracle (GPU).

Offsets, indices and weights bit-exact against oracle.symmetric_csr of the
oracle's own samples; the COO output and counts are those of the plain
layout.  The allowance is the one of the other parity tests: a mismatch is
accepted only when the oracle flags an integer-boundary draw."""
import numpy as np
import pytest
import torch

import oracle
from parity import assert_traced, oracle_sample, same_sample
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300.sampler import Sampler

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def net(n, seed, uecm, ties=True):
    rng = np.random.default_rng(seed)
    mu = -3.0 - max(0.0, np.log(n / 3000))  # mean degree of a few, also at 70,000 nodes
    x = np.exp(rng.normal(mu, 1.4, n))
    if n > 20 and ties:
        x[rng.choice(n, 2, replace=False)] = rng.uniform(5, 30, 2)  # hubs
        x[10:20] = x[3]
    y = rng.uniform(0.1, 0.95, n) if uecm else None
    return x, y


def check(model, x, y, *, num_samples=3, seg_target=32, layout="both", **kw):
    n = len(x)
    s = Sampler(model, dev(x), dev(y), num_samples=num_samples, seg_target=seg_target, layout=layout, symmetric=True,
                **kw)
    res = s.run()
    begin = kw.get("sample_begin", 0)
    ref, stats, log = oracle_sample(model, x, y, num_samples=num_samples, seg_target=seg_target,
                                    sample_begin=begin, seed=kw.get("seed", 0))
    src, dst, w, counts = ref
    off, idx, wts = oracle.symmetric_csr(src, dst, w, counts, n)
    got_off = res.csr_offsets.cpu().numpy()
    if not (np.array_equal(res.counts, counts) and np.array_equal(got_off, off)
            and np.array_equal(res.csr_indices.cpu().numpy(), idx)):
        # a difference must come from segments holding oracle boundary draws,
        # traced on the same call's COO output (a CSR-only call has none)
        assert layout == "both", "symmetric CSR differs from the oracle's"
        got = (res.src.cpu().numpy(), res.dst.cpu().numpy(), None if res.w is None else res.w.cpu().numpy(),
               res.counts)
        assert not same_sample(got, ref), "the COO output equals the oracle's but the symmetric CSR does not"
        assert_traced(model, x, y, got, ref, log, seg_target=seg_target, flags=0, sample_begin=begin)
        return res
    if model == UECM:
        assert np.array_equal(res.csr_weights.cpu().numpy(), wts)
    if layout == "both":
        assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.dst.cpu().numpy(), dst)
    return res


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("T", [2, 32, 1 << 30])
def test_symmetric_matches_oracle(model, T):
    x, y = net(3000, seed=T, uecm=model == UECM)
    check(model, x, y, seg_target=T, num_samples=4)


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_symmetric_several_chunks(model):
    # a large segment-table capacity leaves room for two samples per chunk
    x, y = net(2500, seed=3, uecm=model == UECM)
    check(model, x, y, num_samples=5, max_segments=1 << 21, layout="csr", seed=99, sample_begin=7)


@pytest.mark.parametrize("n", [1, 2, 3, 300, 70_000])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_symmetric_sizes(model, n):
    # 70,000 nodes: more than 2^16 ranks (three key bytes) and the radix node sort
    x, y = net(n, seed=n, uecm=model == UECM)
    if n == 3:
        x[:] = 4.0  # every pair almost surely an edge
    check(model, x, y, num_samples=2, seg_target=3)


def test_symmetric_zero_fitness_and_ties():
    x = np.zeros(500)
    x[::7] = 2.0
    check(UBCM, x, None, num_samples=3, seg_target=2)


def test_symmetric_capacity_retry():
    x, y = net(2000, seed=11, uecm=True)
    s = Sampler(UECM, dev(x), dev(y), num_samples=3, layout="csr", symmetric=True, capacity=64)
    assert s.call() == nat.MH_ERR_CAPACITY
    res = s.run()
    src, dst, w, counts, _ = oracle.mh_sample(UECM, x, y, num_samples=3)
    off, idx, wts = oracle.symmetric_csr(src, dst, w, counts, len(x))
    assert np.array_equal(res.csr_offsets.cpu().numpy(), off)
    assert np.array_equal(res.csr_indices.cpu().numpy(), idx)
    assert np.array_equal(res.csr_weights.cpu().numpy(), wts)


def test_symmetric_bench_workload_full_size():
    from paper_2509_13230_gb300 import workloads
    nw = workloads.uecm_n20k()
    check(UECM, nw.x, nw.y, num_samples=3, seg_target=8)


def test_symmetric_flag_needs_csr():
    x, y = net(100, seed=1, uecm=False)
    with pytest.raises(nat.MhError) as e:
        Sampler(UBCM, dev(x), None, layout="coo", symmetric=True).run()
    assert e.value.code == nat.MH_ERR_ARG
