"""The C-ABI library loads, exports what include/maxent_mh.h declares, and
rejects bad arguments before touching a GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "maxent_mh.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nat.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    assert sorted(nat.EXPORTED) == names
    for name in names:
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in range(0, -8, -1):
        assert nat.error_string(code).startswith("MH_")


def test_workspace_size_and_argument_checks(lib):
    p = nat.make_params(num_samples=10)
    small = nat.mh_workspace_size(nat.MH_UECM, 1000, p, 10_000)
    big = nat.mh_workspace_size(nat.MH_UECM, 1000, p, 1_000_000)
    assert big - small >= 4 * 990_000 - 512  # int32 staging per edge of capacity
    for bad in [dict(num_samples=0), dict(seg_target=1), dict(flags=0x8000)]:
        q = nat.make_params(**bad)
        with pytest.raises(nat.MhError) as e:
            nat.mh_workspace_size(nat.MH_UBCM, 100, q, 10)
        assert e.value.code == nat.MH_ERR_ARG
    with pytest.raises(nat.MhError):
        nat.mh_workspace_size(nat.MH_UBCM, 0, p, 10)
    with pytest.raises(nat.MhError):
        nat.mh_workspace_size(7, 10, p, 10)


def test_sampling_rejects_null_inputs_without_a_gpu(lib):
    p = nat.make_params()
    counts = (ctypes.c_int64 * 1)()
    rc = nat.mh_sample_ubcm(None, 10, p, None, 0, None, None, None, None, 0, counts, None, None)
    assert rc == nat.MH_ERR_ARG
    rc = nat.mh_sample_weighted(None, None, 10, p, None, 0, None, None, None, None, None, None, 0, counts, None, None)
    assert rc == nat.MH_ERR_ARG
    assert nat.maxent_expected_fwd(0, None, None, 5, None, None, None) == nat.MH_ERR_ARG
    assert nat.maxent_expected_bwd(1, None, None, 5, None, None, None, None, None) == nat.MH_ERR_ARG
    info = nat.mh_last_call_info()
    assert info.kernel_launches == 0


def test_bipartite_workspace_and_argument_checks(lib):
    p = nat.make_params(num_samples=3)
    a = nat.mh_bipartite_workspace_size(nat.MH_UECM, 1000, 3000, p, 10_000)
    b = nat.mh_bipartite_workspace_size(nat.MH_UECM, 1000, 30_000, p, 10_000)
    assert b - a >= 27_000 * 48  # the - set's sorted copies grow with n_minus
    for flags, n_plus, n_minus in [(nat.MH_BOUND_PAPER, 10, 10), (nat.MH_INIT_PREV, 10, 10),
                                   (nat.MH_DIRECTED, 10, 11)]:
        q = nat.make_params(flags=nat.MH_OUT_COO | flags)
        with pytest.raises(nat.MhError) as e:
            nat.mh_bipartite_workspace_size(nat.MH_UBCM, n_plus, n_minus, q, 10)
        assert e.value.code == nat.MH_ERR_ARG
    # MH_DIRECTED belongs to the bipartite call only
    with pytest.raises(nat.MhError):
        nat.mh_workspace_size(nat.MH_UBCM, 10, nat.make_params(flags=nat.MH_DIRECTED), 10)
    # a directed network of equal sets is fine
    assert nat.mh_bipartite_workspace_size(nat.MH_UBCM, 10, 10, nat.make_params(flags=nat.MH_DIRECTED), 10) > 0


def test_symmetric_csr_workspace_and_argument_checks(lib):
    sym = nat.MH_OUT_CSR | nat.MH_CSR_SYMMETRIC
    # (CSR with COO: no node-order slot maps, which a CSR-only layout adds)
    plain = nat.mh_workspace_size(nat.MH_UECM, 1000, nat.make_params(flags=nat.MH_OUT_CSR | nat.MH_OUT_COO),
                                  100_000)
    with_sym = nat.mh_workspace_size(nat.MH_UECM, 1000, nat.make_params(flags=sym), 100_000)
    assert with_sym - plain >= 100_000 * 32  # keys, positions, sources and weights of the edges
    csr_only = nat.mh_workspace_size(nat.MH_UECM, 1000, nat.make_params(flags=nat.MH_OUT_CSR), 100_000)
    assert csr_only - plain >= 8 * 1001  # node-order slot maps of a CSR-only call
    for bad in [nat.MH_CSR_SYMMETRIC, nat.MH_OUT_COO | nat.MH_CSR_SYMMETRIC]:  # needs MH_OUT_CSR
        with pytest.raises(nat.MhError) as e:
            nat.mh_workspace_size(nat.MH_UBCM, 10, nat.make_params(flags=bad), 10)
        assert e.value.code == nat.MH_ERR_ARG
    with pytest.raises(nat.MhError) as e:  # one node set only
        nat.mh_bipartite_workspace_size(nat.MH_UBCM, 10, 12, nat.make_params(flags=sym), 10)
    assert e.value.code == nat.MH_ERR_ARG
    desc = nat.network_descs([(nat.MH_UBCM, 0, 10, ctypes.c_void_p(256), None)])  # never dereferenced
    with pytest.raises(nat.MhError) as e:
        nat.mh_batch_workspace_size(desc, 1, nat.make_params(flags=sym), 100, 100)
    assert e.value.code == nat.MH_ERR_ARG


def test_row_range_argument_checks_without_a_gpu(lib):
    # the checks run before anything touches the (never dereferenced) pointers
    fake = ctypes.c_void_p(256)
    for begin, count in ((-1, 2), (0, -1), (4, 2), (6, 0), (2, 4)):
        assert nat.maxent_expected_fwd_rows(1, fake, fake, 5, begin, count, fake, fake, None) == nat.MH_ERR_ARG
        assert nat.maxent_expected_bwd_rows(1, fake, fake, 5, begin, count, fake, fake, fake, fake,
                                            None) == nat.MH_ERR_ARG
    assert "rows" in nat.last_error_detail()
    # an empty range is valid and launches nothing
    assert nat.maxent_expected_fwd_rows(0, fake, None, 5, 5, 0, fake, None, None) == nat.MH_OK
    assert nat.maxent_expected_bwd_rows(0, fake, None, 5, 0, 0, fake, None, fake, None, None) == nat.MH_OK
    assert nat.maxent_expected_fwd_rows(1, None, fake, 5, 0, 1, fake, fake, None) == nat.MH_ERR_ARG


def test_row_shard_covers_every_row_once():
    from paper_2509_13230_gb300.sampler import row_shard
    for n in (0, 1, 7, 64, 1537):
        for world in (1, 2, 3, 8):
            parts = [row_shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0
            for (b0, c0), (b1, _) in zip(parts, parts[1:]):
                assert b0 + c0 == b1
            assert sum(c for _, c in parts) == n
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        row_shard(5, 2, 2)


def test_jacobian_diagonal_argument_checks_without_a_gpu(lib):
    fake = ctypes.c_void_p(256)
    assert nat.maxent_expected_jacobian_diag(1, fake, fake, 5, fake, None, fake, fake, None) == nat.MH_ERR_ARG
    assert nat.maxent_expected_jacobian_diag(0, None, None, 5, fake, None, None, None, None) == nat.MH_ERR_ARG
    assert nat.maxent_expected_jacobian_diag(0, fake, None, 0, fake, None, None, None, None) == nat.MH_ERR_ARG
    assert nat.maxent_expected_jacobian_diag(2, fake, fake, 5, fake, fake, fake, fake, None) == nat.MH_ERR_ARG


def test_sym_workspace_size(lib):
    """The symmetric pair sums' scratch: double-float copies of the operands
    (16 B per node, twice for the UECM), a bit per node, and one FP64 partial
    per (quantity, band of L columns, node), L = max(2048, n / 128 rounded
    up to a multiple of 512), 1 quantity for the UBCM and 3 for the UECM."""
    def align(v):
        return (v + 255) // 256 * 256

    for model, q in ((nat.MH_UBCM, 1), (nat.MH_UECM, 3)):
        for n in (1, 31, 2048, 2049, 200_000, 1_000_000):
            L = max(2048, -(-(-(-n // 128)) // 512) * 512)
            nb = -(-n // L)
            assert nb <= 128
            want = align(16 * n) + (align(16 * n) if model == nat.MH_UECM else 0) + align(4 * (-(-n // 32)))
            want += align(8 * q * nb * n)
            rc, got = nat.maxent_expected_sym_workspace_size(model, n)
            assert rc == nat.MH_OK and got == want, (model, n, got, want)
    assert nat.maxent_expected_sym_workspace_size(nat.MH_UBCM, 0)[0] == nat.MH_ERR_ARG
    assert nat.maxent_expected_sym_workspace_size(5, 10)[0] == nat.MH_ERR_ARG
