"""Batched ensembles: many networks x many samples through mh_sample_batched.

A batch is a list of networks (UBCM or UECM, any sizes), each sampled
``num_samples`` times.  Its (network, sample) pairs are numbered
network-major and drawn in waves: contiguous pair ranges whose work items
(pairs x segment-table rows) fit the wave buffers and whose edges fit the
output buffers, which every wave reuses.  Every edge comes from the CUDA
library; this module sizes buffers, plans waves on the host and hands each
wave's output to the caller.

Sample s of network t equals the single-network call on that network with
network_id = the network's id and sample_begin = sample_begin + s.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as nat
from .sampler import _check_vec, _ptr, _stream_handle

DEFAULT_WAVE_ITEMS = 1 << 26
MAX_WAVE_PAIRS = 1 << 20


def plan_waves(items_per_pair, est_edges_per_pair, num_samples: int, *, items_max: int, capacity: int,
               pair_begin: int = 0, pair_end: int | None = None, pairs_max: int = MAX_WAVE_PAIRS):
    """Split pairs [pair_begin, pair_end) into waves, in order.

    items_per_pair[t] and est_edges_per_pair[t] are per network t; pair p is
    network p // num_samples.  A wave takes pairs while its items stay
    within items_max, its estimated edges within capacity and its pair count
    within pairs_max; a wave always takes at least one pair.  Returns a list
    of (first pair, pair count).  Raises ValueError for a pair whose items
    alone exceed items_max.
    """
    items = np.asarray(items_per_pair, dtype=np.int64)
    est = np.asarray(est_edges_per_pair, dtype=np.float64)
    total = len(items) * num_samples
    end = total if pair_end is None else pair_end
    waves = []
    p = pair_begin
    while p < end:
        first = p
        w_items = 0
        w_edges = 0.0
        while p < end and p - first < pairs_max:
            t = p // num_samples
            if items[t] > items_max:
                raise ValueError(f"network {t} has {items[t]} work items per sample; max_wave_items is {items_max}")
            if p > first and (w_items + items[t] > items_max or w_edges + est[t] > capacity):
                break
            # whole remaining samples of network t that still fit, at once
            left = min(end - p, (t + 1) * num_samples - p, pairs_max - (p - first))
            by_items = (items_max - w_items) // items[t] if items[t] > 0 else left
            by_edges = int((capacity - w_edges) // est[t]) if est[t] > 0 else left
            take = max(1 if p == first else 0, min(left, by_items, by_edges))
            if take == 0:
                break
            w_items += take * int(items[t])
            w_edges += take * float(est[t])
            p += take
        waves.append((first, p - first))
    return waves


@dataclass
class WaveResult:
    """One wave's output; tensors are views into buffers the next wave reuses."""
    pair_begin: int
    pair_count: int
    counts: np.ndarray                        # int64[pair_count]
    stats: np.ndarray                         # uint64[5] (MH_STAT_*)
    networks: np.ndarray                      # int64[pair_count]: network of each pair
    samples: np.ndarray                       # int64[pair_count]: sample index of each pair (0-based)
    src: torch.Tensor | None = None
    dst: torch.Tensor | None = None
    w: torch.Tensor | None = None
    csr_offsets: torch.Tensor | None = None   # sum over pairs of n_t + 1
    csr_indices: torch.Tensor | None = None
    csr_weights: torch.Tensor | None = None
    _edge_at: np.ndarray = field(default=None, repr=False)  # first edge of each pair
    _off_at: np.ndarray = field(default=None, repr=False)   # first CSR offset of each pair

    @property
    def total(self) -> int:
        return int(self.counts.sum())

    def coo(self, k: int):
        """(src, dst, w) of the wave's k-th pair."""
        a, b = int(self._edge_at[k]), int(self._edge_at[k] + self.counts[k])
        return self.src[a:b], self.dst[a:b], None if self.w is None else self.w[a:b]

    def csr(self, k: int, n: int):
        """(offsets relative to the pair's first edge, indices, weights) of pair k."""
        o = int(self._off_at[k])
        off = self.csr_offsets[o:o + n + 1]
        a = int(off[0])
        b = int(off[-1])
        return off - a, self.csr_indices[a:b], None if self.csr_weights is None else self.csr_weights[a:b]


class Ensemble:
    """Many networks, each sampled num_samples times, drawn in waves.

    networks: list of (model, x, y) or (model, x, y, network_id) with x, y
    1-D float64 CUDA tensors (y None for the UBCM).  Network ids default to
    the network's index.  layout: "coo", "csr" or "both".
    capacity: edges one wave may write (the output buffers' length).
    """

    def __init__(self, networks, *, num_samples: int = 1, seed: int = 0, sample_begin: int = 0,
                 seg_target: int = 0, layout: str = "csr", bound: str = "suffix", init: str = "head",
                 fp64_only: bool = False, max_segments: int = 0, max_wave_items: int = DEFAULT_WAVE_ITEMS,
                 capacity: int = 1 << 24, timing: bool = False, walk_ctas_per_sm: int = 0):
        self.entries = []
        for t, net in enumerate(networks):
            model, x, y = int(net[0]), net[1], net[2]
            nid = int(net[3]) if len(net) > 3 else t
            x = _check_vec("x", x)
            y = _check_vec("y", y, x.shape[0]) if model == nat.MH_UECM else None
            self.entries.append((model, nid, int(x.shape[0]), x, y))
        if not self.entries:
            raise ValueError("an ensemble needs at least one network")
        self.n = np.array([e[2] for e in self.entries], dtype=np.int64)
        self.models = np.array([e[0] for e in self.entries], dtype=np.int64)
        self.num_samples = int(num_samples)
        flags = {"coo": nat.MH_OUT_COO, "csr": nat.MH_OUT_CSR, "both": nat.MH_OUT_COO | nat.MH_OUT_CSR}[layout]
        if bound == "paper":
            flags |= nat.MH_BOUND_PAPER
        if init == "prev":
            flags |= nat.MH_INIT_PREV
        if fp64_only:
            flags |= nat.MH_FP64_ONLY
        if timing:
            flags |= nat.MH_TIMING
        self.layout = layout
        self.params = nat.make_params(seed=seed, sample_begin=sample_begin, num_samples=num_samples,
                                      seg_target=seg_target, flags=flags, max_segments=max_segments,
                                      walk_ctas_per_sm=walk_ctas_per_sm)
        self.descs = nat.network_descs([(m, nid, n, x.data_ptr(), None if y is None else y.data_ptr())
                                        for (m, nid, n, x, y) in self.entries])
        self.max_wave_items = int(max_wave_items)
        self.capacity = int(capacity)
        self.any_uecm = bool((self.models == nat.MH_UECM).any())
        self.num_segments = None
        self.est = None
        self.ws = None
        self._alloc_outputs()

    # ---- buffers ---------------------------------------------------------------
    def _alloc_outputs(self):
        dev = self.entries[0][3].device
        cap = max(self.capacity, 1)
        coo = self.layout in ("coo", "both")
        csr = self.layout in ("csr", "both")
        i32 = dict(dtype=torch.int32, device=dev)
        self.src = torch.empty(cap, **i32) if coo else None
        self.dst = torch.empty(cap, **i32) if coo else None
        self.w = torch.empty(cap, **i32) if coo and self.any_uecm else None
        self.csr_idx = torch.empty(cap, **i32) if csr else None
        self.csr_w = torch.empty(cap, **i32) if csr and self.any_uecm else None
        self.csr_off = None
        self._csr_off_len = 0
        self.h_counts = np.zeros(0, dtype=np.int64)

    def _ensure_workspace(self):
        nbytes = nat.mh_batch_workspace_size(self.descs, len(self.entries), self.params, self.max_wave_items,
                                             self.capacity)
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.entries[0][3].device)

    def _ensure_csr_offsets(self, length: int):
        if self.layout == "coo" or length <= self._csr_off_len:
            return
        self.csr_off = torch.empty(length, dtype=torch.int64, device=self.entries[0][3].device)
        self._csr_off_len = length

    # ---- preparation -------------------------------------------------------------
    def prepare(self, stream=None) -> np.ndarray:
        """Sort and partition every network; returns the segment rows per network."""
        self._ensure_workspace()
        while True:
            segs = np.zeros(len(self.entries), dtype=np.int64)
            rc = nat.mh_batch_prepare(self.descs, len(self.entries), self.params, _ptr(self.ws), self.ws.numel(),
                                      segs.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream))
            over = [t for t in range(len(self.entries)) if segs[t] > self._segment_cap(t)]
            if rc == nat.MH_ERR_WORKSPACE and over:
                # segment tables outgrew their capacity: raise the caps of those networks
                for t in over:
                    self.descs[t].max_segments = int(segs[t]) + int(segs[t]) // 8 + 1024
                self._ensure_workspace()
                continue
            nat.check(rc, "mh_batch_prepare")
            break
        self.num_segments = segs
        if self.est is None:
            T = self.params.seg_target or 32
            self.est = 0.5 * T * segs.astype(np.float64) + 16.0
        return segs

    def _segment_cap(self, t: int) -> int:
        d = self.descs[t]
        if d.max_segments > 0:
            return int(d.max_segments)
        return int(self.params.max_segments) if self.params.max_segments > 0 else 4 * int(d.n) + 1024

    # ---- waves ------------------------------------------------------------------------
    def plan(self, pair_begin: int = 0, pair_end: int | None = None):
        if self.num_segments is None:
            raise RuntimeError("call prepare() first")
        return plan_waves(self.num_segments, self.est, self.num_samples, items_max=self.max_wave_items,
                          capacity=self.capacity, pair_begin=pair_begin, pair_end=pair_end,
                          pairs_max=min(MAX_WAVE_PAIRS, len(self.entries) * self.num_samples))

    def _csr_len(self, first: int, count: int) -> int:
        p = np.arange(first, first + count)
        return int((self.n[p // self.num_samples] + 1).sum())

    def run_wave(self, first: int, count: int, stream=None) -> tuple[int, WaveResult]:
        """Draws pairs [first, first + count); returns (return code, result)."""
        self._ensure_csr_offsets(self._csr_len(first, count))
        counts = np.zeros(count, dtype=np.int64)
        stats = np.zeros(nat.MH_NUM_STATS, dtype=np.uint64)
        rc = nat.mh_sample_batched(self.descs, len(self.entries), self.params, self.max_wave_items, _ptr(self.ws),
                                   self.ws.numel(), first, count, _ptr(self.src), _ptr(self.dst), _ptr(self.w),
                                   _ptr(self.csr_off), _ptr(self.csr_idx), _ptr(self.csr_w), self.capacity,
                                   counts.ctypes.data_as(ctypes.c_void_p), stats.ctypes.data_as(ctypes.c_void_p),
                                   _stream_handle(stream))
        p = np.arange(first, first + count)
        nets = p // self.num_samples
        res = WaveResult(first, count, counts, stats, nets, p % self.num_samples)
        if rc == nat.MH_OK:
            total = int(counts.sum())
            res._edge_at = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
            res._off_at = np.concatenate([[0], np.cumsum(self.n[nets] + 1)[:-1]]).astype(np.int64)
            if self.src is not None:
                res.src, res.dst = self.src[:total], self.dst[:total]
                res.w = None if self.w is None else self.w[:total]
            if self.csr_idx is not None:
                res.csr_offsets = self.csr_off[:int((self.n[nets] + 1).sum())]
                res.csr_indices = self.csr_idx[:total]
                res.csr_weights = None if self.csr_w is None else self.csr_w[:total]
        return rc, res

    def _learn(self, res: WaveResult):
        for t in np.unique(res.networks):
            seen = res.counts[res.networks == t]
            self.est[t] = max(float(seen.max()) * 1.05 + 64.0, 1.0)

    def sample(self, on_wave=None, stream=None, pair_begin: int = 0, pair_end: int | None = None):
        """Draws every pair in [pair_begin, pair_end) (default: all), wave by
        wave; calls on_wave(result) after each wave.  Returns per-pair edge
        counts and the summed stats."""
        if self.num_segments is None:
            self.prepare(stream)
        end = len(self.entries) * self.num_samples if pair_end is None else pair_end
        counts = np.zeros(end - pair_begin, dtype=np.int64)
        stats = np.zeros(nat.MH_NUM_STATS, dtype=np.uint64)
        todo = self.plan(pair_begin, end)
        self.waves_run = 0
        while todo:
            first, count = todo.pop(0)
            rc, res = self.run_wave(first, count, stream)
            if rc == nat.MH_ERR_CAPACITY:
                # exact counts are back: re-plan these pairs with them
                if count == 1:
                    raise nat.MhError(rc, "mh_sample_batched",
                                      f"pair {first} has {int(res.counts[0])} edges; capacity is {self.capacity}")
                self._learn(res)
                sub = []
                # one wave per run of pairs that fits, using the exact counts
                acc, start = 0, first
                for k in range(count):
                    c = int(res.counts[k])
                    if k > 0 and acc + c > self.capacity:
                        sub.append((start, first + k - start))
                        start, acc = first + k, 0
                    acc += c
                sub.append((start, first + count - start))
                todo = sub + todo
                continue
            nat.check(rc, "mh_sample_batched")
            self._learn(res)
            counts[first - pair_begin:first - pair_begin + count] = res.counts
            stats += res.stats
            self.waves_run += 1
            if on_wave is not None:
                on_wave(res)
        return counts, stats
