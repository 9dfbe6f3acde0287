"""CUDA sampler and expected-degree kernels against the CPU oracle (GPU).

Edge lists, weights, per-sample counts and the proposal, edge, segment and
boundary-draw counters must equal the serial oracle bit for bit.  The only
allowed difference is a segment holding a boundary draw that the oracle
logged (tests/parity.py states the rule).
"""
import numpy as np
import pytest
import torch

import oracle
from parity import check_sample
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import workloads
from paper_2509_13230_gb300.sampler import Sampler, expected_bwd, expected_fwd, segment_table

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM
FLAG_NAMES = {0: {}, oracle.BOUND_PAPER: dict(bound="paper"), oracle.INIT_PREV: dict(init="prev")}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu_run(model, x, y=None, **kw):
    s = Sampler(model, dev(x), None if y is None else dev(y), **kw)
    return s.run(), s


def assert_matches_oracle(res, model, x, y=None, *, num_samples=1, seg_target=32, flags=0, seed=0, sample_begin=0,
                          network_id=0):
    got = (res.src.cpu().numpy(), res.dst.cpu().numpy(), None if res.w is None else res.w.cpu().numpy(),
           np.asarray(res.counts))
    same, stats = check_sample(got, model, x, y, num_samples=num_samples, seg_target=seg_target, flags=flags,
                               seed=seed, sample_begin=sample_begin, network_id=network_id)
    if same:
        assert int(res.stats[nat.MH_STAT_PROPOSALS]) == int(stats[0])
        assert int(res.stats[nat.MH_STAT_EDGES]) == int(stats[1])
        assert int(res.stats[nat.MH_STAT_SEGMENTS]) == int(stats[2])
        assert int(res.stats[nat.MH_STAT_BOUNDARY]) == int(stats[3])
    return stats


def heavy_tailed(n, seed, hubs=3, uecm=False):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.normal(-2.5, 1.6, n))
    x[rng.choice(n, hubs, replace=False)] = rng.uniform(5, 40, hubs)
    y = rng.uniform(0.2, 0.95, n) if uecm else None
    return x, y


# --------------------------------------------------------------------------
# Segment table (sort, bound prep, partition)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("T", [2, 9, 32, 1 << 30])
@pytest.mark.parametrize("flags", [0, oracle.BOUND_PAPER])
def test_segment_table_matches_oracle(model, T, flags):
    x, y = heavy_tailed(5003, seed=T + flags, uecm=model == UECM)
    x[100:140] = x[7]  # ties across sort tiles
    ref = oracle.partition(model, x, y, seg_target=T, flags=flags)
    got = segment_table(model, dev(x), None if y is None else dev(y), seg_target=T,
                        bound="paper" if flags else "suffix")
    for key in ("perm", "row", "k", "a", "b"):
        assert np.array_equal(got[key], ref[key]), key


@pytest.mark.parametrize("n", [511, 512, 513, 24_576, 24_577, 40_000, 65_536, 65_537])
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_sort_paths_match_oracle(model, n):
    # node sets sorted with 512-key tiles and a shared-memory merge (up to
    # 24,576 nodes), 2048-key tiles and a sampled merge (up to 65,536), or the
    # radix passes; ties across tile boundaries and zero values in each
    x, y = heavy_tailed(n, seed=n, uecm=model == UECM)
    x *= min(1.0, 2000.0 / n)  # a mean degree of a few at every size
    x[n // 3: n // 3 + 700] = x[1]
    x[-50:] = 0.0
    ref = oracle.partition(model, x, y, seg_target=16)
    got = segment_table(model, dev(x), None if y is None else dev(y), seg_target=16)
    for key in ("perm", "row", "k", "a", "b"):
        assert np.array_equal(got[key], ref[key]), key


# --------------------------------------------------------------------------
# Full-size workloads
# --------------------------------------------------------------------------
def test_ubcm_n1k_x100_bit_exact():
    net = workloads.ubcm_n1k()
    res, _ = gpu_run(UBCM, net.x, num_samples=100)
    assert_matches_oracle(res, UBCM, net.x, num_samples=100)


def test_uecm_n20k_x10_bit_exact():
    net = workloads.uecm_n20k()
    res, _ = gpu_run(UECM, net.x, net.y, num_samples=10)
    assert_matches_oracle(res, UECM, net.x, net.y, num_samples=10)


def test_ubcm_pareto_n1m_csr_bit_exact():
    net = workloads.ubcm_pareto_n1m()
    res, _ = gpu_run(UBCM, net.x, num_samples=1, layout="both")
    src, dst, _, counts, _ = oracle.mh_sample(UBCM, net.x, num_samples=1)
    assert np.array_equal(res.counts, counts)
    assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.dst.cpu().numpy(), dst)
    # CSR: row u holds the edges whose higher-ranked endpoint is u, in walk order
    n = net.n
    order = np.argsort(src, kind="stable")
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(np.bincount(src, minlength=n))
    assert np.array_equal(res.csr_offsets.cpu().numpy(), off)
    assert np.array_equal(res.csr_indices.cpu().numpy(), dst[order])


# --------------------------------------------------------------------------
# Variants: segment target, bound and initial-q readings, FP64-only path
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("T", [2, 7, 1 << 30])
@pytest.mark.parametrize("flags", [0, oracle.BOUND_PAPER, oracle.INIT_PREV])
def test_variants_bit_exact(model, T, flags):
    if model == UBCM and flags == oracle.BOUND_PAPER:
        pytest.skip("the bound reading only applies to the UECM")
    x, y = heavy_tailed(2600, seed=11 + T, uecm=model == UECM)
    res, _ = gpu_run(model, x, y, num_samples=3, seg_target=T, seed=0x1234567890ABCDEF, network_id=5,
                     sample_begin=77, **FLAG_NAMES[flags])
    assert_matches_oracle(res, model, x, y, num_samples=3, seg_target=T, flags=flags, seed=0x1234567890ABCDEF,
                          network_id=5, sample_begin=77)


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_fp64_only_path_bit_exact(model):
    x, y = heavy_tailed(3000, seed=21, uecm=model == UECM)
    res, _ = gpu_run(model, x, y, num_samples=4, fp64_only=True)
    assert_matches_oracle(res, model, x, y, num_samples=4)


# --------------------------------------------------------------------------
# Degenerate and edge cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("case", ["n1", "n2", "zeros", "ties", "huge", "y_zero"])
def test_degenerate_inputs(model, case):
    rng = np.random.default_rng(3)
    y = None
    if case == "n1":
        x = np.array([0.7])
    elif case == "n2":
        x = np.array([0.3, 2.0])
    elif case == "zeros":
        x = np.r_[np.zeros(50), np.exp(rng.normal(-1, 1, 30))]
    elif case == "ties":
        x = np.full(300, 0.2)
    elif case == "huge":
        x = np.r_[np.full(3, 1e9), np.exp(rng.normal(-2, 1, 200))]  # x_i x_j > 2^53: p rounds to 1
    else:
        x = np.exp(rng.normal(-1, 1, 200))
    if model == UECM:
        y = rng.uniform(0.0, 0.9, len(x))
        if case == "y_zero":
            y[::3] = 0.0
    res, _ = gpu_run(model, x, y, num_samples=5, seg_target=3)
    assert_matches_oracle(res, model, x, y, num_samples=5, seg_target=3)


def test_many_chunks_and_overflow_rewalk():
    # a hub row with far more edges than a lane's shared-memory slot (64),
    # and a segment-table capacity that splits the samples into several chunks
    rng = np.random.default_rng(4)
    x = np.r_[np.full(2, 30.0), np.exp(rng.normal(-0.5, 0.5, 1500))]
    res, s = gpu_run(UBCM, x, num_samples=7, seg_target=1 << 30, max_segments=1 << 21)
    assert nat.mh_last_call_info().sample_chunks == 4
    assert_matches_oracle(res, UBCM, x, num_samples=7, seg_target=1 << 30)
    assert int(res.counts.max()) > 64


def test_batch_equals_single_samples():
    x, y = heavy_tailed(4000, seed=5, uecm=True)
    batch, _ = gpu_run(UECM, x, y, num_samples=4, sample_begin=10)
    for s in range(4):
        one, _ = gpu_run(UECM, x, y, num_samples=1, sample_begin=10 + s)
        bs, bd, bw = batch.coo(s)
        assert torch.equal(bs, one.src) and torch.equal(bd, one.dst) and torch.equal(bw, one.w)


def test_capacity_retry_reproduces_sample():
    x, _ = heavy_tailed(3000, seed=6)
    s = Sampler(UBCM, dev(x), num_samples=2, capacity=16)
    assert s.call() == nat.MH_ERR_CAPACITY
    need = int(s.h_counts.sum())
    assert need > 16
    res = s.run()
    assert res.total == need
    assert_matches_oracle(res, UBCM, x, num_samples=2)


@pytest.mark.parametrize("bad", ["neg_x", "nan_x", "y_one"])
def test_domain_errors(bad):
    x = np.full(100, 0.5)
    y = np.full(100, 0.5)
    if bad == "neg_x":
        x[3] = -1.0
    elif bad == "nan_x":
        x[3] = np.nan
    else:
        y[3] = 1.0
    with pytest.raises(nat.MhError) as e:
        gpu_run(UECM, x, y)
    assert e.value.code == nat.MH_ERR_DOMAIN


def test_call_info_counts_launches():
    x, _ = heavy_tailed(2000, seed=7)
    s = Sampler(UBCM, dev(x), num_samples=2)
    s.flags |= nat.MH_TIMING
    s.run()
    info = nat.mh_last_call_info()
    assert info.walk_launches == 1 and info.sample_chunks == 1
    assert 5 <= info.kernel_launches <= 30
    assert info.walk_ms > 0 and info.total_ms >= info.walk_ms


# --------------------------------------------------------------------------
# Expected degrees / strengths and gradients
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_expected_fwd_bwd_match_oracle(model):
    x, y = heavy_tailed(1537, seed=8, uecm=model == UECM)
    rng = np.random.default_rng(9)
    gk = rng.normal(size=len(x))
    gs = rng.normal(size=len(x)) if model == UECM else None
    k, s = expected_fwd(model, dev(x), None if y is None else dev(y))
    rk, rs = oracle.expected_fwd(model, x, y)
    np.testing.assert_allclose(k.cpu().numpy(), rk, rtol=1e-10)
    if model == UECM:
        np.testing.assert_allclose(s.cpu().numpy(), rs, rtol=1e-10)
    gx, gy = expected_bwd(model, dev(x), None if y is None else dev(y), dev(gk), None if gs is None else dev(gs))
    rgx, rgy = oracle.expected_bwd(model, x, y, gk, gs)
    np.testing.assert_allclose(gx.cpu().numpy(), rgx, rtol=1e-10, atol=1e-12 * np.abs(rgx).max())
    if model == UECM:
        np.testing.assert_allclose(gy.cpu().numpy(), rgy, rtol=1e-10, atol=1e-12 * np.abs(rgy).max())


def test_expected_fwd_full_size_sampled_rows():
    rng = np.random.default_rng(10)
    n = 200_000
    x = np.exp(rng.normal(-5.5, 1.3, n))
    y = rng.uniform(0.3, 0.9, n)
    k, s = expected_fwd(UECM, dev(x), dev(y))
    rows = rng.choice(n, 12, replace=False)
    rk, rs = oracle.expected_fwd(UECM, x, y, rows=rows)
    np.testing.assert_allclose(k.cpu().numpy()[rows], rk, rtol=1e-10)
    np.testing.assert_allclose(s.cpu().numpy()[rows], rs, rtol=1e-10)


@pytest.mark.parametrize("layout", ["csr", "both"])
def test_csr_call_with_segment_table_overflow_retries(layout):
    # T = 2 on a dense network needs far more table rows than 4 n + 1024: the
    # first call stops at the truncated table (MH_ERR_WORKSPACE, nothing walked
    # or written) and the retry with the needed rows samples exactly.
    rng = np.random.default_rng(17)
    x = np.exp(rng.normal(0.5, 0.3, 400))
    s = Sampler(UBCM, dev(x), num_samples=2, seg_target=2, layout=layout)
    assert s.call() == nat.MH_ERR_WORKSPACE
    res = s.run()
    got = (res.src.cpu().numpy(), res.dst.cpu().numpy(), None, res.counts) if layout == "both" else None
    src, dst, _, counts, stats = oracle.mh_sample(UBCM, x, num_samples=2, seg_target=2)
    if got is not None:
        check_sample(got, UBCM, x, num_samples=2, seg_target=2)
    assert np.array_equal(res.counts, counts)
    n = len(x)
    for k in range(2):
        a, b = int(counts[:k].sum()), int(counts[:k + 1].sum())
        order = np.argsort(src[a:b], kind="stable")
        off = np.zeros(n + 1, np.int64)
        off[1:] = np.cumsum(np.bincount(src[a:b], minlength=n))
        got_off = res.csr_offsets[k * (n + 1):(k + 1) * (n + 1)].cpu().numpy()
        assert np.array_equal(got_off - got_off[0], off)
        assert np.array_equal(res.csr_indices[int(got_off[0]):int(got_off[-1])].cpu().numpy(), dst[a:b][order])


# --------------------------------------------------------------------------
# Bounded device waits
# --------------------------------------------------------------------------
@pytest.mark.parametrize("model", [UBCM, UECM])
def test_bounded_wait_gives_up_and_next_call_is_exact(model):
    # MH_TEST_WAIT_TIMEOUT makes tile 1 of every single-pass scan wait on a
    # flag that nothing sets: the wait must run out after its poll limit, the
    # call must return MH_ERR_DEVICE_TIMEOUT promptly, and the same sampler's
    # next call (same workspace, scan states left cleared) must be exact.
    import time
    x, y = heavy_tailed(20_000, seed=41, uecm=model == UECM)  # tens of thousands of work items: many scan tiles
    s = Sampler(model, dev(x), None if y is None else dev(y), num_samples=2, seg_target=16)
    s.run()  # sizes the buffers
    s.flags |= nat.MH_TEST_WAIT_TIMEOUT
    t0 = time.perf_counter()
    rc = s.call()
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert rc == nat.MH_ERR_DEVICE_TIMEOUT
    assert elapsed < 5.0
    s.flags &= ~nat.MH_TEST_WAIT_TIMEOUT
    res = s.run()
    assert_matches_oracle(res, model, x, y, num_samples=2, seg_target=16)


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_csr_only_calls_equal_the_csr_of_both_layouts(model):
    """A CSR-only call numbers its work items by node id (node-order slot
    maps) while a call that also writes COO keeps the rank order: the CSR
    arrays must agree bit for bit, over several sample chunks."""
    rng = np.random.default_rng(91)
    n = 300_000
    x = np.minimum(workloads.pareto_scale(n) * rng.uniform(0.0, 1.0, n) ** (-1.0 / 1.1), 50.0)
    y = rng.uniform(0.3, 0.9, n) if model == UECM else None
    samples = 30  # more items than one chunk holds: several chunks
    csr, s1 = gpu_run(model, x, y, num_samples=samples, layout="csr", seed=5, sample_begin=2)
    both, s2 = gpu_run(model, x, y, num_samples=samples, layout="both", seed=5, sample_begin=2)
    assert np.array_equal(csr.counts, both.counts)
    assert torch.equal(csr.csr_offsets, both.csr_offsets)
    assert torch.equal(csr.csr_indices, both.csr_indices)
    if model == UECM:
        assert torch.equal(csr.csr_weights, both.csr_weights)
    for k in range(nat.MH_NUM_STATS):
        assert int(csr.stats[k]) == int(both.stats[k])


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_fast_levels_equal_fp64_only_on_long_skips(model):
    """The sparse rows of a large capped-Pareto network make skips of 10^3 to
    10^5 candidates, where the FP32 level's error bound matters most: the
    default levels and the canonical FP64 path must draw the same samples."""
    n = 1_000_000
    rng = np.random.default_rng(97)
    x = np.minimum(workloads.pareto_scale(n) * rng.uniform(0.0, 1.0, n) ** (-1.0 / 1.1), 50.0)
    y = rng.uniform(0.3, 0.9, n) if model == UECM else None
    fast, _ = gpu_run(model, x, y, num_samples=4, seed=41, layout="coo")
    slow, _ = gpu_run(model, x, y, num_samples=4, seed=41, layout="coo", fp64_only=True)
    assert np.array_equal(fast.counts, slow.counts)
    assert torch.equal(fast.src, slow.src) and torch.equal(fast.dst, slow.dst)
    if model == UECM:
        assert torch.equal(fast.w, slow.w)
    assert int(fast.stats[nat.MH_STAT_PROPOSALS]) == int(slow.stats[nat.MH_STAT_PROPOSALS])
