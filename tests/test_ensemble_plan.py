"""Host logic of batched ensembles: the wave planner and the batch ABI's
argument checks and workspace sizing (no GPU needed)."""
import ctypes

import numpy as np
import pytest

from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import build
from paper_2509_13230_gb300.ensemble import plan_waves


def check_plan(waves, begin, end, items, est, S, items_max, capacity, pairs_max):
    # the waves tile [begin, end) in order
    at = begin
    for first, count in waves:
        assert first == at and count >= 1
        at += count
    assert at == end
    for first, count in waves:
        p = np.arange(first, first + count)
        t = p // S
        if count > 1:  # a single pair may exceed the estimate, never the item limit
            assert items[t].sum() <= items_max
            assert est[t].sum() <= capacity + 1e-9
            assert count <= pairs_max
        assert items[t].sum() <= items_max


@pytest.mark.parametrize("seed", range(6))
def test_plan_covers_pairs_within_limits(seed):
    rng = np.random.default_rng(seed)
    nets = int(rng.integers(1, 40))
    S = int(rng.integers(1, 9))
    items = rng.integers(0, 5000, nets)
    est = rng.uniform(0, 3000, nets)
    items_max = int(max(items.max(), 1) * rng.uniform(1, 6))
    capacity = float(rng.uniform(500, 20000))
    pairs_max = int(rng.integers(1, 50))
    begin = int(rng.integers(0, nets * S))
    end = int(rng.integers(begin + 1, nets * S + 1))
    waves = plan_waves(items, est, S, items_max=items_max, capacity=capacity, pair_begin=begin, pair_end=end,
                       pairs_max=pairs_max)
    check_plan(waves, begin, end, items, est, S, items_max, capacity, pairs_max)


def test_plan_is_greedy_and_splits_networks():
    # 3 networks x 4 samples, 10 items per pair, items_max 25: two pairs per wave
    waves = plan_waves([10, 10, 10], [1, 1, 1], 4, items_max=25, capacity=1e9)
    assert waves == [(0, 2), (2, 2), (4, 2), (6, 2), (8, 2), (10, 2)]
    # capacity binds: 3 edges per pair, capacity 7 -> two pairs per wave
    waves = plan_waves([1, 1], [3, 3], 3, items_max=100, capacity=7)
    assert waves == [(0, 2), (2, 2), (4, 2)]
    # one wave holds everything
    assert plan_waves([5, 7], [1, 1], 8, items_max=10_000, capacity=1e6) == [(0, 16)]


def test_plan_rejects_a_pair_above_the_item_limit():
    with pytest.raises(ValueError):
        plan_waves([10, 300], [1, 1], 2, items_max=100, capacity=1e9)


def test_oversized_estimate_still_takes_one_pair():
    assert plan_waves([1, 1], [1e9, 1e9], 2, items_max=100, capacity=10) == [(0, 1), (1, 1), (2, 1), (3, 1)]


# --------------------------------------------------------------------------
# The batch entry points' host-side checks (pointers are never dereferenced
# on these paths, so fake addresses serve).
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def lib():
    build.build()
    return nat.load()


def descs(sizes, models, fake=0x1000):
    return nat.network_descs([(m, 0, n, fake + 0x100 * t, (fake + 0x80 + 0x100 * t) if m == nat.MH_UECM else None)
                              for t, (n, m) in enumerate(zip(sizes, models))])


def test_batch_workspace_grows_with_nodes_items_and_capacity(lib):
    p = nat.make_params(num_samples=4)
    d1 = descs([1000, 5000], [nat.MH_UBCM, nat.MH_UECM])
    d2 = descs([1000, 5000, 20000], [nat.MH_UBCM, nat.MH_UECM, nat.MH_UBCM])
    a = nat.mh_batch_workspace_size(d1, 2, p, 1 << 20, 1 << 20)
    b = nat.mh_batch_workspace_size(d2, 3, p, 1 << 20, 1 << 20)
    c = nat.mh_batch_workspace_size(d1, 2, p, 1 << 22, 1 << 20)
    d = nat.mh_batch_workspace_size(d1, 2, p, 1 << 20, 1 << 24)
    assert b - a >= 20000 * 100           # prepared arrays of the extra network
    assert c - a >= 20 * ((1 << 22) - (1 << 20))   # int32 count, int64 staging base and offset per work item
    assert d - a >= 4 * ((1 << 24) - (1 << 20))    # int32 staging per edge of capacity


@pytest.mark.parametrize("case", ["no_nets", "network_id", "null_x", "null_y", "bad_model", "n0", "wave_items"])
def test_batch_argument_errors(lib, case):
    p = nat.make_params(num_samples=2)
    d = descs([100, 200], [nat.MH_UBCM, nat.MH_UECM])
    n_nets, items = 2, 0
    if case == "no_nets":
        n_nets = 0
    elif case == "network_id":
        p.network_id = 3
    elif case == "null_x":
        d[0].x = None
    elif case == "null_y":
        d[1].y = None
    elif case == "bad_model":
        d[0].model = 5
    elif case == "n0":
        d[1].n = 0
    else:
        items = 1 << 31
    with pytest.raises(nat.MhError) as e:
        nat.mh_batch_workspace_size(d, n_nets, p, items, 1000)
    assert e.value.code == nat.MH_ERR_ARG


def test_sample_batched_rejects_bad_pair_ranges_without_a_gpu(lib):
    p = nat.make_params(num_samples=3)
    d = descs([100, 200], [nat.MH_UBCM, nat.MH_UBCM])
    counts = (ctypes.c_int64 * 8)()
    for begin, count in [(-1, 1), (0, 0), (5, 2), (0, 7)]:
        rc = nat.mh_sample_batched(d, 2, p, 0, ctypes.c_void_p(0x1000), 1 << 30, begin, count, None, None, None,
                                   None, None, None, 0, counts, None, None)
        assert rc == nat.MH_ERR_ARG, (begin, count)


# --------------------------------------------------------------------------
# Autotuner selection rule (timings are inputs here; the GPU probes are
# exercised in tests/test_gpu_batched.py)
# --------------------------------------------------------------------------
def test_autotune_pick_fastest_and_tie_rules():
    from paper_2509_13230_gb300.autotune import pick
    row = lambda T, c, r: {"T": T, "ctas": c, "edges_per_ms": r}
    # clear winner
    assert pick([row(16, 0, 100), row(32, 0, 120), row(64, 2, 300)]) == (64, 2)
    # within 1 %: the default T wins
    assert pick([row(16, 0, 1000), row(32, 0, 995), row(64, 0, 998)]) == (32, 0)
    # within 1 % without the default: the larger T, then full occupancy
    assert pick([row(16, 0, 1000), row(64, 2, 996), row(64, 0, 995)]) == (64, 0)
    # outside the tie band the rate decides
    assert pick([row(32, 0, 900), row(128, 2, 1000)]) == (128, 2)
    with pytest.raises(ValueError):
        pick([])
