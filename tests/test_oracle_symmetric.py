"""Pins of the oracle's symmetric CSR layout (every edge in both rows), no GPU.

The layout is checked against scipy.sparse (the sample's adjacency matrix
plus its transpose), against the degree sequence, and against a property
of the samplers' output order: rows i walk candidates of lower rank only,
in rank order, so a row of the symmetric layout lists its neighbours in
node order (descending key, ties by ascending id, Sec. 2.4 step (i))."""
import numpy as np
import pytest
from scipy import sparse

import oracle

UBCM, UECM = oracle.UBCM, oracle.UECM


def network(model, n, seed):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.normal(-1.5, 1.2, n))
    x[: n // 10] = x[0]  # ties
    y = rng.uniform(0.2, 0.9, n) if model == UECM else None
    return x, y


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_symmetric_csr_matches_adjacency_plus_transpose(model):
    n = 60
    x, y = network(model, n, 3)
    src, dst, w, counts, _ = oracle.mh_sample(model, x, y, num_samples=4, seg_target=3)
    off, idx, wts = oracle.symmetric_csr(src, dst, w, counts, n)
    assert len(idx) == 2 * counts.sum()
    pos = 0
    for s, c in enumerate(counts):
        ss, dd = src[pos:pos + c], dst[pos:pos + c]
        vals = np.ones(c) if w is None else w[pos:pos + c].astype(float)
        a = sparse.coo_matrix((vals, (ss, dd)), shape=(n, n))
        ref = (a + a.T).tocsr()
        o = off[s * (n + 1):(s + 1) * (n + 1)]
        assert np.array_equal(np.diff(o), np.diff(ref.indptr))
        assert np.array_equal(np.diff(o), np.bincount(np.concatenate([ss, dd]), minlength=n))
        for u in range(n):
            got = sorted(zip(idx[o[u]:o[u + 1]].tolist(),
                             (np.ones(o[u + 1] - o[u]) if wts is None else wts[o[u]:o[u + 1]]).tolist()))
            row = ref.getrow(u)
            want = sorted(zip(row.indices.tolist(), row.data.tolist()))
            assert got == want
        pos += c
    assert off[0] == 0 and off[-1] == len(idx)


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_symmetric_rows_list_neighbours_in_node_order(model):
    n = 80
    x, y = network(model, n, 5)
    src, dst, w, counts, _ = oracle.mh_sample(model, x, y, num_samples=3, seg_target=2)
    key = x if model == UBCM else x * y
    rank = np.empty(n, np.int64)
    rank[oracle.sort_desc(key)] = np.arange(n)
    off, idx, _ = oracle.symmetric_csr(src, dst, w, counts, n)
    for s in range(3):
        o = off[s * (n + 1):(s + 1) * (n + 1)]
        for u in range(n):
            r = rank[idx[o[u]:o[u + 1]]]
            assert np.all(np.diff(r) > 0)


def test_symmetric_csr_empty_and_single_edge():
    off, idx, wts = oracle.symmetric_csr(np.zeros(0, np.int32), np.zeros(0, np.int32), None, np.array([0, 0]), 3)
    assert np.array_equal(off, np.zeros(8)) and len(idx) == 0 and wts is None
    off, idx, wts = oracle.symmetric_csr(np.array([2], np.int32), np.array([0], np.int32), np.array([7], np.int32),
                                         np.array([1]), 3)
    assert off.tolist() == [0, 1, 1, 2] and idx.tolist() == [2, 0] and wts.tolist() == [7, 7]
