"""mh_sample_ubcm_noalloc: the UBCM sampler for callers that cannot allocate
device memory (it runs on a fixed scratch area inside the library).

Its output must equal that of the allocating entry point mh_sample_ubcm,
called through the same C ABI with the same arguments, on two calls in a
row (the second call reuses the scratch the first one left behind).  This
file is collected last so that a run stopping at its first failure has run
every other test already; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import build

pytestmark = pytest.mark.gpu


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_allocating_entry_point():
    assert torch.cuda.is_available(), "GPU test collected on a machine without a GPU"
    build.build()
    nat.load()
    rng = np.random.default_rng(2024)
    n, samples = 3000, 3
    x = torch.from_numpy(np.exp(rng.normal(-3.0, 1.2, n))).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    params = nat.make_params(seed=77, num_samples=samples, flags=nat.MH_OUT_COO | nat.MH_OUT_CSR)
    cap = 400_000

    # allocating entry point (the caller supplies a workspace)
    ws_bytes = nat.mh_workspace_size(nat.MH_UBCM, n, params, cap)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    ref_src = torch.empty(cap, dtype=torch.int32, device="cuda")
    ref_dst = torch.empty(cap, dtype=torch.int32, device="cuda")
    ref_off = torch.empty(samples * (n + 1), dtype=torch.int64, device="cuda")
    ref_idx = torch.empty(cap, dtype=torch.int32, device="cuda")
    ref_counts = np.zeros(samples, np.int64)
    ref_stats = np.zeros(4, np.uint64)
    rc = nat.mh_sample_ubcm(_ptr(x), n, params, _ptr(ws), ws_bytes, _ptr(ref_src), _ptr(ref_dst), _ptr(ref_off),
                            _ptr(ref_idx), cap, ref_counts.ctypes.data_as(ctypes.c_void_p),
                            ref_stats.ctypes.data_as(ctypes.c_void_p), stream)
    nat.check(rc, "mh_sample_ubcm")
    total = int(ref_counts.sum())
    assert total > 1000

    for call in range(2):
        src = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        dst = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        off = torch.full((samples * (n + 1),), -1, dtype=torch.int64, device="cuda")
        idx = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        counts = np.zeros(samples, np.int64)
        stats = np.zeros(4, np.uint64)
        rc = nat.mh_sample_ubcm_noalloc(_ptr(x), n, params, _ptr(src), _ptr(dst), _ptr(off), _ptr(idx), cap,
                                        counts.ctypes.data_as(ctypes.c_void_p),
                                        stats.ctypes.data_as(ctypes.c_void_p), stream)
        nat.check(rc, "mh_sample_ubcm_noalloc")
        # integer output: the tolerance is exact equality
        assert np.array_equal(counts, ref_counts), call
        assert np.array_equal(stats, ref_stats), call
        assert torch.equal(src[:total], ref_src[:total]), call
        assert torch.equal(dst[:total], ref_dst[:total]), call
        assert torch.equal(off, ref_off), call
        assert torch.equal(idx[:total], ref_idx[:total]), call


def test_noalloc_rejects_calls_beyond_its_scratch():
    assert torch.cuda.is_available(), "GPU test collected on a machine without a GPU"
    nat.load()
    n = 2_000_000
    x = torch.full((n,), 1e-3, dtype=torch.float64, device="cuda")
    params = nat.make_params(num_samples=1)
    counts = np.zeros(1, np.int64)
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    rc = nat.mh_sample_ubcm_noalloc(_ptr(x), n, params, _ptr(out), _ptr(out), None, None, 16,
                                    counts.ctypes.data_as(ctypes.c_void_p), None,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == nat.MH_ERR_WORKSPACE
    assert "fixed scratch" in nat.last_error_detail()
