"""mh_sample_ubcm_noalloc: the UBCM sampler for callers that cannot allocate
device memory (it runs on a fixed scratch area inside the library).

Its output must equal that of the allocating entry point mh_sample_ubcm,
called through the same C ABI with the same arguments, and the oracle's
sample.  Calls follow one another on the shared scratch: the same call twice,
then calls of other shapes after a larger one (node count, sample count,
output flags and sort path all change the scratch layout).  This file is
collected last so that a run stopping at its first failure has run every
other test already; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import build

pytestmark = pytest.mark.gpu

COO, CSR = nat.MH_OUT_COO, nat.MH_OUT_CSR


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _host(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _setup():
    assert torch.cuda.is_available(), "GPU test collected on a machine without a GPU"
    build.build()
    nat.load()


def _network(n, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(-3.0 - max(0.0, np.log(n / 3000)), 1.2, n))


def _outputs(n, samples, cap, flags, fill):
    coo = bool(flags & COO)
    csr = bool(flags & CSR)
    mk = lambda k, dt: torch.full((k,), fill, dtype=dt, device="cuda")  # noqa: E731
    return (mk(cap, torch.int32) if coo else None, mk(cap, torch.int32) if coo else None,
            mk(samples * (n + 1), torch.int64) if csr else None, mk(cap, torch.int32) if csr else None)


def _allocating(x, n, params, samples, cap, flags):
    ws_bytes = nat.mh_workspace_size(nat.MH_UBCM, n, params, cap)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = _outputs(n, samples, cap, flags, 0)
    counts = np.zeros(samples, np.int64)
    stats = np.zeros(nat.MH_NUM_STATS, np.uint64)
    rc = nat.mh_sample_ubcm(_ptr(x), n, params, _ptr(ws), ws_bytes, *(_ptr(t) for t in out), cap, _host(counts),
                            _host(stats), _stream())
    nat.check(rc, "mh_sample_ubcm")
    return out, counts, stats


def _noalloc(x, n, params, samples, cap, flags):
    out = _outputs(n, samples, cap, flags, -1)
    counts = np.zeros(samples, np.int64)
    stats = np.zeros(nat.MH_NUM_STATS, np.uint64)
    rc = nat.mh_sample_ubcm_noalloc(_ptr(x), n, params, *(_ptr(t) for t in out), cap, _host(counts), _host(stats),
                                    _stream())
    nat.check(rc, "mh_sample_ubcm_noalloc")
    return out, counts, stats


def _check_call(xh, seed, samples, flags, calls, sample_begin=0):
    n = len(xh)
    x = torch.from_numpy(xh).cuda()
    params = nat.make_params(seed=seed, sample_begin=sample_begin, num_samples=samples, flags=flags)
    src_o, dst_o, _, counts_o, stats_o = oracle.mh_sample(oracle.UBCM, xh, seed=seed, sample_begin=sample_begin,
                                                          num_samples=samples)
    total = int(counts_o.sum())
    cap = total + 1024
    ref, ref_counts, ref_stats = _allocating(x, n, params, samples, cap, flags)
    assert np.array_equal(ref_counts, counts_o)
    for call in range(calls):
        got, counts, stats = _noalloc(x, n, params, samples, cap, flags)
        info = nat.mh_last_call_info()
        assert info.kernel_launches > 0 and info.sample_chunks >= 1 and info.walk_launches == info.sample_chunks
        # integer output: the tolerance is exact equality, against both references
        assert np.array_equal(counts, ref_counts) and np.array_equal(counts, counts_o), call
        assert np.array_equal(stats, ref_stats), call
        assert int(stats[nat.MH_STAT_PROPOSALS]) == int(stats_o[0]), call
        for g, r in zip(got, ref):
            if g is not None:
                k = g.numel() if g.dtype == torch.int64 else total
                assert torch.equal(g[:k], r[:k]), call
        if flags & COO:
            assert np.array_equal(got[0][:total].cpu().numpy(), src_o), call
            assert np.array_equal(got[1][:total].cpu().numpy(), dst_o), call
        if flags & CSR:
            # offsets of sample s start where the edges of the samples before it end
            off = got[2].cpu().numpy().reshape(samples, n + 1)
            assert np.array_equal(off[:, -1], np.cumsum(counts_o)), call
    return total


def test_noalloc_matches_allocating_entry_point():
    _setup()
    total = _check_call(_network(3000, 2024), seed=77, samples=3, flags=COO | CSR, calls=2)
    assert total > 1000


def test_noalloc_calls_of_other_shapes_after_a_larger_one():
    # each layout puts the control block, scans and sort state at other
    # offsets of the shared scratch; whatever the previous call left there
    # must not matter
    _setup()
    _check_call(_network(40_000, 5), seed=3, samples=2, flags=COO | CSR, calls=1)  # 2048-key tile sort path
    _check_call(_network(3000, 6), seed=4, samples=3, flags=COO | CSR, calls=1)
    _check_call(_network(700, 7), seed=5, samples=5, flags=COO, calls=1, sample_begin=9)
    _check_call(_network(20_000, 8), seed=6, samples=1, flags=CSR, calls=1)  # 512-key tile sort path
    _check_call(_network(700, 7), seed=5, samples=5, flags=COO, calls=1, sample_begin=9)


def test_noalloc_rejects_calls_beyond_its_scratch():
    _setup()
    n = 2_000_000
    x = torch.full((n,), 1e-3, dtype=torch.float64, device="cuda")
    params = nat.make_params(num_samples=1)
    counts = np.zeros(1, np.int64)
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    rc = nat.mh_sample_ubcm_noalloc(_ptr(x), n, params, _ptr(out), _ptr(out), None, None, 16, _host(counts), None,
                                    _stream())
    assert rc == nat.MH_ERR_WORKSPACE
    assert "fixed scratch" in nat.last_error_detail()


def test_noalloc_rejects_too_many_samples():
    _setup()
    n = 100
    x = torch.full((n,), 0.1, dtype=torch.float64, device="cuda")
    params = nat.make_params(num_samples=1025)
    counts = np.zeros(1025, np.int64)
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    rc = nat.mh_sample_ubcm_noalloc(_ptr(x), n, params, _ptr(out), _ptr(out), None, None, 16, _host(counts), None,
                                    _stream())
    assert rc == nat.MH_ERR_ARG
    assert "1024 samples" in nat.last_error_detail()


def test_noalloc_refuses_a_capturing_stream():
    _setup()
    xh = _network(500, 9)
    x = torch.from_numpy(xh).cuda()
    params = nat.make_params(num_samples=1)
    counts = np.zeros(1, np.int64)
    out = torch.empty(4096, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        rc = nat.mh_sample_ubcm_noalloc(_ptr(x), len(xh), params, _ptr(out), _ptr(out), None, None, 4096,
                                        _host(counts), None, ctypes.c_void_p(side.cuda_stream))
        out.zero_()  # a node, so the captured graph is not empty
    assert rc == nat.MH_ERR_ARG
    assert "capture" in nat.last_error_detail()
    # the refused call enqueued nothing; the next call samples as usual
    _check_call(xh, seed=0, samples=1, flags=COO, calls=1)
