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


# --------------------------------------------------------------------------
# A fit sharded by rows and one sample split by segment ranges
# --------------------------------------------------------------------------
def _oracle_row_fns():
    """Row-range sums, gradient and Jacobian diagonal of the oracle, with the
    signatures of sampler.expected_*(..., rows=(begin, count))."""
    import torch

    import oracle

    def idx(rows, n):
        b, c = rows
        return np.arange(b, b + c)

    def t(a):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a))

    def npy(a):
        return None if a is None else a.detach().cpu().numpy()

    def fwd(model, x, y=None, rows=None):
        k, s = oracle.expected_fwd(model, npy(x), npy(y), rows=idx(rows, len(x)))
        return t(k), t(s)

    def bwd(model, x, y, g_k, g_s=None, rows=None):
        gx, gy = oracle.expected_bwd(model, npy(x), npy(y), npy(g_k), npy(g_s), rows=idx(rows, len(x)))
        return t(gx), t(gy)

    def diag(model, x, y=None, rows=None):
        return tuple(t(a) for a in oracle.expected_jacobian_diag(model, npy(x), npy(y), rows=idx(rows, len(x))))

    return fwd, bwd, diag


def _fit_targets():
    import oracle
    rng = np.random.default_rng(47)
    n = 40
    x_true = np.exp(rng.normal(-1.5, 0.8, n))
    y_true = rng.uniform(0.3, 0.85, n)
    return oracle.expected_fwd(oracle.UECM, x_true, y_true)


def _fit_rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_2509_13230_gb300 import expected as E
    from paper_2509_13230_gb300.distributed import ShardedSums
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        fwd, bwd, diag = _oracle_row_fns()
        sums = ShardedSums(fwd=fwd, bwd=bwd, diag=diag)
        k_t, s_t = _fit_targets()
        res = E.fit(torch.from_numpy(k_t), torch.from_numpy(s_t), tol=1e-8, sums=sums)
        out[rank] = (res.x.numpy(), res.y.numpy(), res.newton_steps, res.residual, dict(sums.calls))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_fit_by_row_shards():
    """A Newton-CG fit whose sums, gradients and Jacobian diagonal are split
    by rows over two gloo ranks (oracle row functions on CPU standing in for
    the *_rows kernels) takes exactly the steps of the one-process fit."""
    import torch

    from paper_2509_13230_gb300 import expected as E
    from paper_2509_13230_gb300.distributed import ShardedSums
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_fit_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    fwd, bwd, diag = _oracle_row_fns()
    k_t, s_t = _fit_targets()
    one = E.fit(torch.from_numpy(k_t), torch.from_numpy(s_t), tol=1e-8, sums=ShardedSums(fwd=fwd, bwd=bwd, diag=diag))
    assert one.residual <= 1e-8
    for r in range(world):
        x, y, steps, resid, calls = out[r]
        assert steps == one.newton_steps and resid == one.residual
        assert np.array_equal(x, one.x.numpy()) and np.array_equal(y, one.y.numpy())  # bit for bit
        assert calls["diag"] == steps


def _split_network():
    from paper_2509_13230_gb300 import workloads
    rng = np.random.default_rng(53)
    n = 3000
    u = rng.uniform(0.0, 1.0, n)
    x = np.minimum(workloads.pareto_scale(n) * u ** (-1.0 / 1.1), 50.0)  # heavy tail, mean degree about 20
    y = rng.uniform(0.3, 0.9, n)
    return x, y


def _split_rank_main(rank, world, port, model, out):
    import torch.distributed as dist

    import oracle
    from paper_2509_13230_gb300.distributed import exclusive_offsets, segment_costs, segment_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, y = _split_network()
        y = y if model == oracle.UECM else None
        T = 16
        table = oracle.partition(model, x, y, seg_target=T)  # the table every rank computes
        s0, s1 = segment_shard(segment_costs(model, x, y, table), rank, world)
        src, dst, w, counts, stats = oracle.mh_sample_segments(model, x, y, seg_begin=s0, seg_end=s1,
                                                               seg_target=T, sample_begin=7)
        offset, total = exclusive_offsets(len(src))
        out[rank] = (s0, s1, offset, total, src, dst, w, int(stats[0]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("model", [0, 1])
def test_two_gloo_ranks_split_one_sample_by_segment_ranges(model):
    """One sample split over two gloo ranks by cost-balanced ranges of the
    segment table; the ranks' edges, placed by the exclusive scan of their
    counts, are the one-rank sample bit for bit (oracle on CPU)."""
    import oracle
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_split_rank_main, args=(r, world, port, model, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    x, y = _split_network()
    y = y if model == oracle.UECM else None
    src, dst, w, counts, stats = oracle.mh_sample(model, x, y, seg_target=16, sample_begin=7)
    S = len(oracle.partition(model, x, y, seg_target=16)["row"])
    assert out[0][0] == 0 and out[0][1] == out[1][0] and out[1][1] == S  # the ranges tile the table
    total = len(src)
    got_src, got_dst, got_w = np.zeros(total, np.int32), np.zeros(total, np.int32), np.zeros(total, np.int32)
    for r in range(world):
        s0, s1, offset, tot, rs, rd, rw, props = out[r]
        assert tot == total
        got_src[offset:offset + len(rs)] = rs
        got_dst[offset:offset + len(rs)] = rd
        if rw is not None:
            got_w[offset:offset + len(rs)] = rw
    assert np.array_equal(got_src, src) and np.array_equal(got_dst, dst)
    if w is not None:
        assert np.array_equal(got_w, w)
    # the cost model balances the proposals the ranks draw
    p0, p1 = out[0][7], out[1][7]
    assert p0 + p1 == int(stats[0]) and abs(p0 - p1) < 0.25 * (p0 + p1)


def test_segment_shard_tiles_the_table():
    from paper_2509_13230_gb300.distributed import segment_shard
    costs = np.r_[np.full(10, 5.0), np.full(90, 1.0)]
    for world in (1, 2, 3, 7, 150):
        parts = [segment_shard(costs, r, world) for r in range(world)]
        assert parts[0][0] == 0 and parts[-1][1] == len(costs)
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        assert all(b >= a for a, b in parts)
    assert segment_shard(costs, 0, 2) == (0, 30)  # half of the total cost 140: 10 x 5 + 20 x 1 = 70
