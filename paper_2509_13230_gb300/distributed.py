"""Work split across the ranks of a torch.distributed group (one GPU each).

Two paths shard without changing a single result:

* The expected-degree/strength sums, their gradient and their Jacobian
  diagonal (Sec. 2.2, Sec. 2.5) by rows: every rank holds all of x and y,
  computes its contiguous block of rows over all columns with the
  ``*_rows`` entry points, and an all-gather assembles the vectors.  A row's
  value does not depend on the rows launched with it, so every rank ends up
  with the single-GPU vectors bit for bit, and a fit driven by them takes the
  same steps on every rank (``ShardedSums``; ``expected.fit(..., sums=...)``).
* One large sample by ranges of the segment table: the walk of a segment
  depends only on the segment, the sample and the key (each segment head
  restarts the proposal bound, Sec. 2.3; the Philox counter names the
  segment), so ranks drawing contiguous table ranges (``mh_sample_range``)
  produce, concatenated in rank order, exactly the one-GPU sample.  The one
  exchange is an all-gather of each rank's edge count, whose exclusive scan
  places the rank's edges (``sample_split``).  The ranges are balanced by the
  partition's cost model (expected proposals per segment).

Ensembles of many samples need neither: ranks take disjoint sample indices
(``sample_begin``), with no exchange at all.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import _native as nat
from .sampler import Sampler, expected_bwd, expected_fwd, expected_jacobian_diag, row_shard, segment_table


def _rank_world(group):
    if not dist.is_available() or not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def gather_rows(part: torch.Tensor, n: int, group=None) -> torch.Tensor:
    """All-gathers the row blocks of row_shard(n, r, world) into one vector."""
    rank, world = _rank_world(group)
    if world == 1:
        return part
    counts = [row_shard(n, r, world)[1] for r in range(world)]
    buf = torch.zeros(max(counts), dtype=part.dtype, device=part.device)
    buf[:part.shape[0]] = part
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


class ShardedSums:
    """The pairwise sums of a fit, each rank computing its row block.

    fwd, bwd and diag are the row-range functions (defaults: the CUDA
    entry points through sampler.expected_*(..., rows=...)); tests on CPU
    pass the oracle's instead."""

    def __init__(self, group=None, fwd=None, bwd=None, diag=None):
        self.group = group
        self._fwd = fwd or expected_fwd
        self._bwd = bwd or expected_bwd
        self._diag = diag or expected_jacobian_diag
        self.calls = {"fwd": 0, "bwd": 0, "diag": 0}

    def _rows(self, n):
        rank, world = _rank_world(self.group)
        return row_shard(n, rank, world)

    def _all(self, parts, n):
        return tuple(None if p is None else gather_rows(p, n, self.group) for p in parts)

    def fwd(self, model, x, y=None):
        self.calls["fwd"] += 1
        n = int(x.shape[0])
        return self._all(self._fwd(model, x, y, rows=self._rows(n)), n)

    def bwd(self, model, x, y, g_k, g_s=None):
        self.calls["bwd"] += 1
        n = int(x.shape[0])
        return self._all(self._bwd(model, x, y, g_k, g_s, rows=self._rows(n)), n)

    def diag(self, model, x, y=None):
        self.calls["diag"] += 1
        n = int(x.shape[0])
        return self._all(self._diag(model, x, y, rows=self._rows(n)), n)


# ---------------------------------------------------------------------------
# One sample split by segment ranges
# ---------------------------------------------------------------------------
def segment_costs(model: int, x: np.ndarray, y: np.ndarray | None, table: dict) -> np.ndarray:
    """Expected work of each segment-table row, for balancing only: one head
    step plus the expected proposals sum_{j in [a, b)} min(1, w_i v_j), with v
    the sort key (x, or a = x y for the UECM) in rank order, w_i = v_i (UBCM)
    or a_i / (1 - y_i max_{j > i} y_j) (UECM), the partition's cost model."""
    perm = np.asarray(table["perm"], np.int64)
    xs = np.asarray(x, np.float64)[perm]
    if model == nat.MH_UECM:
        ys = np.asarray(y, np.float64)[perm]
        v = xs * ys
        ymax_after = np.r_[np.maximum.accumulate(ys[::-1])[::-1][1:], 0.0]
        w = v / np.maximum(1.0 - ys * ymax_after, 1e-300)
    else:
        v = xs
        w = xs
    n = len(v)
    P = np.r_[0.0, np.cumsum(v)]
    row = np.asarray(table["row"], np.int64)
    a = np.asarray(table["a"], np.int64)
    b = np.asarray(table["b"], np.int64)
    wi = w[row]
    # J_i: first rank whose cost w_i v_j falls below one (v is non-increasing)
    with np.errstate(divide="ignore"):
        thresh = np.where(wi > 0, 1.0 / wi, np.inf)
    J = np.searchsorted(-v, -thresh, side="right")  # count of v_j >= 1 / w_i
    J = np.clip(J, row + 1, n)
    whole = np.clip(np.minimum(b, J) - a, 0, None)
    lo = np.maximum(a, J)
    part = np.where(b > lo, wi * (P[np.maximum(b, lo)] - P[lo]), 0.0)
    return 1.0 + whole + part


def segment_shard(costs: np.ndarray, rank: int, world: int) -> tuple[int, int]:
    """Contiguous table rows [begin, end) of `rank`: cut where the cumulative
    cost first reaches rank / world of the total (ranges in rank order tile
    the table; some may be empty)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    c = np.r_[0.0, np.cumsum(np.asarray(costs, np.float64))]
    total = c[-1]
    cuts = [0] + [int(np.searchsorted(c, total * r / world, side="left")) for r in range(1, world)] + [len(costs)]
    cuts = np.maximum.accumulate(np.minimum(cuts, len(costs)))
    return int(cuts[rank]), int(cuts[rank + 1])


def exclusive_offsets(count: int, group=None, device=None) -> tuple[int, int]:
    """(edges of the ranks before this one, edges of all ranks): one
    all-gather of an int64 per rank."""
    rank, world = _rank_world(group)
    if world == 1:
        return 0, int(count)
    t = torch.tensor([int(count)], dtype=torch.int64, device=device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    counts = [int(p.item()) for p in parts]
    return sum(counts[:rank]), sum(counts)


def sample_split(model: int, x: torch.Tensor, y: torch.Tensor | None = None, *, group=None, seed: int = 0,
                 network_id: int = 0, sample_begin: int = 0, seg_target: int = 0, **sampler_kw):
    """This rank's share of one sample of (x, y), every rank holding all of x
    and y: (result, first edge of the share in the whole sample, edges of the
    whole sample, (seg_begin, seg_end)).  Concatenated in rank order the
    shares are the one-GPU sample (COO, and weights for the UECM)."""
    rank, world = _rank_world(group)
    table = segment_table(model, x, y, seg_target=seg_target)
    costs = segment_costs(model, x.cpu().numpy(), None if y is None else y.cpu().numpy(), table)
    s0, s1 = segment_shard(costs, rank, world)
    res = Sampler(model, x, y, num_samples=1, seed=seed, network_id=network_id, sample_begin=sample_begin,
                  seg_target=seg_target, layout="coo", seg_range=(s0, s1), **sampler_kw).run()
    offset, total = exclusive_offsets(res.total, group, device=x.device if dist.is_initialized() and
                                      dist.get_backend(group) == "nccl" else None)
    return res, offset, total, (s0, s1)
