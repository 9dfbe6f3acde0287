"""Pieces of the multi-GPU paths, on one GPU (GPU).

mh_sample_range draws the rows [seg_begin, seg_end) of the segment table;
the ranges of a split, concatenated per sample in range order, must be the
whole call's sample bit for bit (and the oracle's).  The Jacobian diagonal's
row-range form must equal the whole call's rows bit for bit.  (The ranks'
exchange, an all-gather of edge counts, and the sharded fit run as gloo ranks
on CPU in tests/test_multirank.py.)
"""
import numpy as np
import pytest
import torch

import oracle
from parity import check_sample
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import workloads
from paper_2509_13230_gb300.distributed import ShardedSums, sample_split, segment_costs, segment_shard
from paper_2509_13230_gb300.sampler import Sampler, expected_jacobian_diag, segment_table

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def pareto_net(n, seed, uecm):
    rng = np.random.default_rng(seed)
    x = np.minimum(workloads.pareto_scale(n) * rng.uniform(0.0, 1.0, n) ** (-1.0 / 1.1), 50.0)
    y = rng.uniform(0.3, 0.9, n) if uecm else None
    return x, y


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("world", [2, 3, 5])
def test_segment_ranges_concatenate_to_the_whole_sample(model, world, cuda_lib):
    x, y = pareto_net(6000, 61 + world, model == UECM)
    T, samples = 16, 2
    table = segment_table(model, dev(x), dev(y), seg_target=T)
    ref = oracle.partition(model, x, y, seg_target=T)
    assert np.array_equal(table["row"], ref["row"]) and np.array_equal(table["a"], ref["a"])
    costs = segment_costs(model, x, y, table)
    parts = []
    for r in range(world):
        s0, s1 = segment_shard(costs, r, world)
        res = Sampler(model, dev(x), dev(y), num_samples=samples, seg_target=T, sample_begin=3,
                      seg_range=(s0, s1)).run()
        segs = int(res.stats[nat.MH_STAT_SEGMENTS])
        assert segs == samples * (s1 - s0)
        parts.append(res)
    src, dst, w, counts = [], [], [], []
    for s in range(samples):
        for res in parts:
            a, b = int(res.counts[:s].sum()), int(res.counts[:s + 1].sum())
            src.append(res.src[a:b].cpu().numpy())
            dst.append(res.dst[a:b].cpu().numpy())
            if model == UECM:
                w.append(res.w[a:b].cpu().numpy())
        counts.append(sum(int(res.counts[s]) for res in parts))
    got = (np.concatenate(src), np.concatenate(dst), np.concatenate(w) if model == UECM else None,
           np.array(counts))
    same, _ = check_sample(got, model, x, y, num_samples=samples, seg_target=T, sample_begin=3)
    assert same
    whole = Sampler(model, dev(x), dev(y), num_samples=samples, seg_target=T, sample_begin=3).run()
    assert np.array_equal(whole.src.cpu().numpy(), got[0]) and np.array_equal(whole.dst.cpu().numpy(), got[1])
    props = sum(int(res.stats[nat.MH_STAT_PROPOSALS]) for res in parts)
    assert props == int(whole.stats[nat.MH_STAT_PROPOSALS])


def test_segment_range_edge_cases(cuda_lib):
    x, y = pareto_net(2000, 71, True)
    S = len(segment_table(UECM, dev(x), dev(y), seg_target=16)["row"])
    empty = Sampler(UECM, dev(x), dev(y), seg_target=16, seg_range=(S // 2, S // 2)).run()
    assert empty.total == 0 and int(empty.stats[nat.MH_STAT_SEGMENTS]) == 0
    past = Sampler(UECM, dev(x), dev(y), seg_target=16, seg_range=(S + 5, S + 100)).run()
    assert past.total == 0
    tail = Sampler(UECM, dev(x), dev(y), seg_target=16, seg_range=(S - 3, S + 100)).run()
    assert int(tail.stats[nat.MH_STAT_SEGMENTS]) == 3
    src, dst, w, counts, _ = oracle.mh_sample_segments(UECM, x, y, seg_begin=S - 3, seg_end=S, seg_target=16)
    assert np.array_equal(tail.src.cpu().numpy(), src) and np.array_equal(tail.w.cpu().numpy(), w)
    s = Sampler(UECM, dev(x), dev(y), seg_target=16, seg_range=(5, 2))
    assert s.call() == nat.MH_ERR_ARG
    with pytest.raises(ValueError):
        Sampler(UECM, dev(x), dev(y), seg_target=16, layout="csr", seg_range=(0, 10))


def test_sample_split_without_process_group_is_the_whole_sample(cuda_lib):
    x, y = pareto_net(3000, 73, False)
    res, offset, total, (s0, s1) = sample_split(UBCM, dev(x), None, seg_target=16, sample_begin=11)
    assert offset == 0 and total == res.total and s0 == 0
    src, dst, _, _, _ = oracle.mh_sample(UBCM, x, seg_target=16, sample_begin=11)
    assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.dst.cpu().numpy(), dst)


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_jacobian_diag_rows_equal_the_whole_call(model, cuda_lib):
    rng = np.random.default_rng(79)
    n = 1537
    x = np.exp(rng.normal(-2.5, 1.2, n))
    y = rng.uniform(0.2, 0.9, n) if model == UECM else None
    whole = expected_jacobian_diag(model, dev(x), dev(y))
    for begin, count in ((0, 64), (63, 130), (700, 837), (1536, 1), (5, 0)):
        part = expected_jacobian_diag(model, dev(x), dev(y), rows=(begin, count))
        for a, b in zip(part, whole):
            assert torch.equal(a, b[begin:begin + count])
    # the sums object of a one-process run returns the whole vectors
    sums = ShardedSums()
    for a, b in zip(sums.diag(model, dev(x), dev(y)), whole):
        assert torch.equal(a, b)
