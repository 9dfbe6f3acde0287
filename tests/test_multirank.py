"""Multi-rank host logic of bench.py on CPU: two gloo ranks shard the samples
and reduce the job's time and edge count (no GPU needed).

Ranks are replicas: rank r draws samples [r S, (r + 1) S), the job's time is
the slowest rank's, its edges all ranks' edges.  Because the Philox counter
is keyed by sample index, the ranks' samples together are exactly the
samples of one call that draws all of them (checked on the oracle)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = bench.rank_samples(rank)
        # stand-in timings: rank r took 10 + 5 r ms and drew 1000 (r + 1) edges
        max_ms, edges = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world,
                                                torch.device("cpu"))
        out[rank] = (first, count, max_ms, edges)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (f0, c0, m0, e0), (f1, c1, m1, e1) = out[0], out[1]
    assert (f0, c0) == (0, 10) and (f1, c1) == (10, 10)  # disjoint, contiguous
    assert m0 == m1 == 15.0                              # the slowest rank's time
    assert e0 == e1 == 3000.0                            # all ranks' edges


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 77, 1, None) == (12.5, 77.0)


def test_rank_samples_union_equals_one_call():
    import bench
    import oracle
    from paper_2509_13230_gb300 import workloads
    net = workloads.ubcm_n1k()
    per_rank = 3
    whole = oracle.mh_sample(oracle.UBCM, net.x, num_samples=2 * per_rank)
    parts = [oracle.mh_sample(oracle.UBCM, net.x, sample_begin=bench.rank_samples(r, per_rank)[0],
                              num_samples=per_rank) for r in range(2)]
    assert np.array_equal(np.concatenate([p[0] for p in parts]), whole[0])
    assert np.array_equal(np.concatenate([p[1] for p in parts]), whole[1])
    assert np.array_equal(np.concatenate([p[3] for p in parts]), whole[3])


def _pairwise_rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2509_13230_gb300.sampler import row_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # every rank holds all of x and y and sums its own block of rows
        rng = np.random.default_rng(31)
        n = 301
        x = np.exp(rng.normal(-2.0, 1.0, n))
        y = rng.uniform(0.2, 0.9, n)
        begin, count = row_shard(n, rank, world)
        k, s = oracle.expected_fwd(oracle.UECM, x, y, rows=np.arange(begin, begin + count))
        width = row_shard(n, 0, world)[1]  # the largest share
        mine = torch.zeros(2, width, dtype=torch.float64)
        mine[0, :count] = torch.from_numpy(k)
        mine[1, :count] = torch.from_numpy(s)
        parts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        counts = [row_shard(n, r, world)[1] for r in range(world)]
        out[rank] = (np.concatenate([p[0, :c].numpy() for p, c in zip(parts, counts)]),
                     np.concatenate([p[1, :c].numpy() for p, c in zip(parts, counts)]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_pairwise_sums_by_rows():
    """Rows of the expected-degree sums split over ranks (each rank sums all
    columns of its rows, so nothing is reduced); the gathered shares are the
    whole call's sums (oracle on CPU)."""
    import oracle
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_pairwise_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rng = np.random.default_rng(31)
    n = 301
    x = np.exp(rng.normal(-2.0, 1.0, n))
    y = rng.uniform(0.2, 0.9, n)
    k, s = oracle.expected_fwd(oracle.UECM, x, y)
    for r in range(world):
        assert np.array_equal(out[r][0], k) and np.array_equal(out[r][1], s)
