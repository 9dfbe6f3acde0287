"""The GPU brute-force sampler against the oracle's (GPU).

Every pair u < v is an independent Bernoulli draw with the counter
{u, v, 0xB0F0B0F0, s} (Sec. 2.2); the CUDA sampler's FP32 filter must decide
every pair as the FP64 comparison does, so the edge lists and weights equal
the serial oracle's brute force bit for bit (the oracle's key is the seed
with the network id added to its high word)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import workloads
from paper_2509_13230_gb300.sampler import BruteForceSampler

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def oracle_bf(model, x, y, seed, network_id, samples, sample_begin):
    key_seed = (seed + (network_id << 32)) & 0xFFFFFFFFFFFFFFFF
    out = [oracle.bf_sample(model, x, y, seed=key_seed, sample=sample_begin + s) for s in range(samples)]
    src = np.concatenate([o[0] for o in out])
    dst = np.concatenate([o[1] for o in out])
    w = None if model != UECM else np.concatenate([o[2] for o in out])
    return src, dst, w, np.array([len(o[0]) for o in out]), sum(o[3] for o in out)


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("fp64_only", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 257, 2000])
def test_bf_matches_oracle(model, fp64_only, n, cuda_lib):
    rng = np.random.default_rng(n + 7 * model)
    x = np.exp(rng.normal(-2.0, 1.5, n))
    if n > 10:
        x[:3] = [0.0, 1e9, 1e-40]  # p = 0, p rounding to 1, an operand outside the FP32 range
    y = rng.uniform(0.0, 0.95, n) if model == UECM else None  # y above 7/8 takes FP64
    res = BruteForceSampler(model, dev(x), dev(y), num_samples=3, seed=0x1234, network_id=2, sample_begin=5,
                            fp64_only=fp64_only).run()
    src, dst, w, counts, evals = oracle_bf(model, x, y, 0x1234, 2, 3, 5)
    assert np.array_equal(res.counts, counts)
    assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.dst.cpu().numpy(), dst)
    if w is not None:
        assert np.array_equal(res.w.cpu().numpy(), w)
    assert int(res.stats[nat.MH_STAT_PROPOSALS]) == evals
    assert int(res.stats[nat.MH_STAT_EDGES]) == int(counts.sum())


def test_bf_weighted_workload_and_capacity_retry(cuda_lib):
    net = workloads.uecm_n20k()
    s = BruteForceSampler(UECM, dev(net.x), dev(net.y), num_samples=1, capacity=100)
    assert s.call() == nat.MH_ERR_CAPACITY
    need = int(s.h_counts.sum())
    res = s.run()
    assert res.total == need
    src, dst, w, counts, _ = oracle_bf(UECM, net.x, net.y, 0, 0, 1, 0)
    assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.w.cpu().numpy(), w)


def test_bf_rejects_bad_inputs(cuda_lib):
    x = np.full(50, 0.5)
    x[7] = np.nan
    with pytest.raises(nat.MhError) as e:
        BruteForceSampler(UBCM, dev(x)).run()
    assert e.value.code == nat.MH_ERR_DOMAIN


# --------------------------------------------------------------------------
# Chung-Lu law (MH_CHUNG_LU): p = min(1, x_i x_j), walk and brute force
# --------------------------------------------------------------------------
def chunglu_x(n, seed):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.normal(-2.2, 1.2, n))
    x[: min(4, n)] = [3.0, 1.5, 0.8, 0.9][: min(4, n)]  # pairs with x_i x_j > 1: certain edges
    return x


@pytest.mark.parametrize("T", [2, 16, 1 << 30])
@pytest.mark.parametrize("n", [2, 5, 3000])
def test_chunglu_walk_matches_oracle(T, n, cuda_lib):
    from parity import check_sample
    from paper_2509_13230_gb300.sampler import Sampler
    x = chunglu_x(n, 90 + n)
    res = Sampler(UBCM, dev(x), num_samples=4, seg_target=T, chung_lu=True, sample_begin=3).run()
    got = (res.src.cpu().numpy(), res.dst.cpu().numpy(), None, np.asarray(res.counts))
    same, stats = check_sample(got, oracle.CL, x, num_samples=4, seg_target=T, sample_begin=3)
    assert same
    assert int(res.stats[nat.MH_STAT_PROPOSALS]) == int(stats[0])


@pytest.mark.parametrize("n", [3, 1500])
def test_chunglu_bf_matches_oracle(n, cuda_lib):
    x = chunglu_x(n, 95 + n)
    res = BruteForceSampler(UBCM, dev(x), num_samples=2, chung_lu=True).run()
    src, dst, _, counts, _ = oracle_bf(oracle.CL, x, None, 0, 0, 2, 0)
    assert np.array_equal(res.counts, counts)
    assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.dst.cpu().numpy(), dst)


def test_chunglu_rejected_for_the_uecm(cuda_lib):
    from paper_2509_13230_gb300.sampler import Sampler
    x = chunglu_x(100, 3)
    with pytest.raises(nat.MhError) as e:
        Sampler(UECM, dev(x), dev(np.full(100, 0.5)), extra_flags=nat.MH_CHUNG_LU).run()
    assert e.value.code == nat.MH_ERR_ARG
