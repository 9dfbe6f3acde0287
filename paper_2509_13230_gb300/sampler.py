"""Torch-facing helpers around the C ABI: buffers, capacity growth, results.

Every sampled bit and every expected-degree term is computed by the CUDA
library; this module allocates device memory with torch, passes pointers and
the current stream, and grows buffers when the library reports that an
output or the segment table was too small (the retried call reproduces the
same sample, since sampling is a pure function of its arguments).
"""
from __future__ import annotations

import ctypes
import re
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as nat


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream: torch.cuda.Stream | None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_vec(name: str, t: torch.Tensor, n: int | None = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 1:
        raise TypeError(f"{name} must be a 1-D float64 CUDA tensor")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} must have {n} entries")
    return t.contiguous()


@dataclass
class SampleResult:
    """Edges of a sampling call; tensors are views trimmed to the edge total."""
    counts: np.ndarray          # int64[num_samples]
    stats: np.ndarray           # uint64[5]: proposals, edges, segments, fallbacks, boundary draws
    src: torch.Tensor | None = None
    dst: torch.Tensor | None = None
    w: torch.Tensor | None = None
    csr_offsets: torch.Tensor | None = None   # int64[num_samples * (n + 1)]
    csr_indices: torch.Tensor | None = None
    csr_weights: torch.Tensor | None = None

    @property
    def total(self) -> int:
        return int(self.counts.sum())

    def coo(self, s: int):
        """(src, dst, w) of sample s."""
        a = int(self.counts[:s].sum())
        b = a + int(self.counts[s])
        return self.src[a:b], self.dst[a:b], None if self.w is None else self.w[a:b]


class Sampler:
    """Reusable buffers for repeated sampling calls on one network.

    layout: "coo", "csr", "both" or "none" (counts only).  symmetric: with a
    CSR layout, list every edge in both endpoint rows (each row's neighbours
    in node order); the CSR index and weight arrays then hold 2 x capacity.
    bound: "suffix" (c = y_i max_{j >= head} y_j) or "paper" (two largest y
    among unprocessed nodes, Sec. 2.5).  init: "head" (q = p at the segment
    head) or "prev" (q = p at the rank before it; p_ii for a row's first
    segment, Sec. 2.4 step (ii)).
    """

    def __init__(self, model: int, x: torch.Tensor, y: torch.Tensor | None = None, *, num_samples: int = 1,
                 seed: int = 0, network_id: int = 0, sample_begin: int = 0, seg_target: int = 0,
                 layout: str = "coo", bound: str = "suffix", init: str = "head", fp64_only: bool = False,
                 capacity: int | None = None, max_segments: int = 0, walk_ctas_per_sm: int = 0,
                 extra_flags: int = 0, symmetric: bool = False, seg_range: tuple[int, int] | None = None,
                 chung_lu: bool = False):
        self.model = int(model)
        self.x = _check_vec("x", x)
        self.n = int(self.x.shape[0])
        self.y = _check_vec("y", y, self.n) if self.model == nat.MH_UECM else None
        flags = {"coo": nat.MH_OUT_COO, "csr": nat.MH_OUT_CSR, "both": nat.MH_OUT_COO | nat.MH_OUT_CSR,
                 "none": 0}[layout]
        if bound == "paper":
            flags |= nat.MH_BOUND_PAPER
        if init == "prev":
            flags |= nat.MH_INIT_PREV
        if fp64_only:
            flags |= nat.MH_FP64_ONLY
        if symmetric:
            flags |= nat.MH_CSR_SYMMETRIC
        if chung_lu:  # p = min(1, x_i x_j) (MH_UBCM only)
            flags |= nat.MH_CHUNG_LU
        self.flags = flags | int(extra_flags)
        self.num_samples = int(num_samples)
        self.seed, self.network_id, self.sample_begin = int(seed), int(network_id), int(sample_begin)
        self.seg_target = int(seg_target)
        self.max_segments = int(max_segments)
        self.walk_ctas_per_sm = int(walk_ctas_per_sm)
        # seg_range = (seg_begin, seg_end): draw only those rows of the segment
        # table (mh_sample_range; COO layout only)
        self.seg_range = None if seg_range is None else (int(seg_range[0]), int(seg_range[1]))
        if self.seg_range is not None and layout != "coo":
            raise ValueError("a segment range is drawn as COO only")
        self.device = self.x.device
        if capacity is None:
            capacity = max(1024, 16 * self.n * self.num_samples)
        self._alloc(int(capacity))

    def params(self, sample_begin: int | None = None) -> nat.MhParams:
        return nat.make_params(seed=self.seed, network_id=self.network_id,
                               sample_begin=self.sample_begin if sample_begin is None else sample_begin,
                               num_samples=self.num_samples, seg_target=self.seg_target, flags=self.flags,
                               max_segments=self.max_segments, walk_ctas_per_sm=self.walk_ctas_per_sm)

    def _workspace_bytes(self, capacity: int) -> int:
        return nat.mh_workspace_size(self.model, self.n, self.params(), capacity)

    def _alloc(self, capacity: int):
        self.capacity = capacity
        self.ws_bytes = self._workspace_bytes(capacity)
        dev = self.device
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        coo = bool(self.flags & nat.MH_OUT_COO)
        csr = bool(self.flags & nat.MH_OUT_CSR)
        weighted = self.model == nat.MH_UECM
        cap = max(capacity, 1)
        self.src = torch.empty(cap, dtype=torch.int32, device=dev) if coo else None
        self.dst = torch.empty(cap, dtype=torch.int32, device=dev) if coo else None
        self.w = torch.empty(cap, dtype=torch.int32, device=dev) if coo and weighted else None
        self.csr_off = torch.empty(self.num_samples * (self.n + 1), dtype=torch.int64, device=dev) if csr else None
        per_edge = 2 if self.flags & nat.MH_CSR_SYMMETRIC else 1
        self.csr_idx = torch.empty(per_edge * cap, dtype=torch.int32, device=dev) if csr else None
        self.csr_w = torch.empty(per_edge * cap, dtype=torch.int32, device=dev) if csr and weighted else None
        self.h_counts = np.zeros(self.num_samples, dtype=np.int64)
        self.h_stats = np.zeros(nat.MH_NUM_STATS, dtype=np.uint64)
        # host pointers passed on every call, converted once
        self._h_counts_p = self.h_counts.ctypes.data_as(ctypes.c_void_p)
        self._h_stats_p = self.h_stats.ctypes.data_as(ctypes.c_void_p)

    def call(self, sample_begin: int | None = None, stream: torch.cuda.Stream | None = None) -> int:
        """One C-ABI call with the current buffers; returns its code."""
        p = self.params(sample_begin)
        st = _stream_handle(stream)
        counts, stats = self._h_counts_p, self._h_stats_p
        if self.seg_range is not None:
            return nat.mh_sample_range(self.model, _ptr(self.x), _ptr(self.y), self.n, p, self.seg_range[0],
                                       self.seg_range[1], _ptr(self.workspace), self.ws_bytes, _ptr(self.src),
                                       _ptr(self.dst), _ptr(self.w), self.capacity, counts, stats, st)
        if self.model == nat.MH_UBCM:
            return nat.mh_sample_ubcm(_ptr(self.x), self.n, p, _ptr(self.workspace), self.ws_bytes, _ptr(self.src),
                                      _ptr(self.dst), _ptr(self.csr_off), _ptr(self.csr_idx), self.capacity, counts,
                                      stats, st)
        return nat.mh_sample_weighted(_ptr(self.x), _ptr(self.y), self.n, p, _ptr(self.workspace), self.ws_bytes,
                                      _ptr(self.src), _ptr(self.dst), _ptr(self.w), _ptr(self.csr_off),
                                      _ptr(self.csr_idx), _ptr(self.csr_w), self.capacity, counts, stats, st)

    def run(self, sample_begin: int | None = None, stream: torch.cuda.Stream | None = None) -> SampleResult:
        for _ in range(8):
            rc = self.call(sample_begin, stream)
            if rc == nat.MH_ERR_CAPACITY:
                self._alloc(int(self.h_counts.sum() * 1.05) + 1024)
                continue
            if rc == nat.MH_ERR_WORKSPACE:
                m = re.search(r"needs (\d+) rows", nat.last_error_detail())
                if m:
                    self.max_segments = int(int(m.group(1)) * 1.25) + 1024
                    self._alloc(self.capacity)
                    continue
            nat.check(rc, "mh_sample_ubcm" if self.model == nat.MH_UBCM else "mh_sample_weighted")
            return self.result()
        raise RuntimeError("sampling did not converge on buffer sizes")

    def result(self) -> SampleResult:
        tot = int(self.h_counts.sum())
        cut = (lambda t: None if t is None else t[:tot])
        ctot = 2 * tot if self.flags & nat.MH_CSR_SYMMETRIC else tot
        ccut = (lambda t: None if t is None else t[:ctot])
        return SampleResult(self.h_counts.copy(), self.h_stats.copy(), cut(self.src), cut(self.dst), cut(self.w),
                            self.csr_off, ccut(self.csr_idx), ccut(self.csr_w))


class BipartiteSampler(Sampler):
    """Reusable buffers for sampling a bipartite network (Sec. 2.6): rows are
    the + set (x_plus, y_plus), candidates the - set (x_minus, y_minus).  With
    directed=True both sets are the same nodes (out- and in-parameters) and
    the pairs (i, i) are excluded.  CSR rows are + ids.  Other arguments as
    Sampler (bound and init readings do not apply)."""

    def __init__(self, model: int, x_plus: torch.Tensor, y_plus: torch.Tensor | None, x_minus: torch.Tensor,
                 y_minus: torch.Tensor | None, *, directed: bool = False, **kw):
        self.x_minus = _check_vec("x_minus", x_minus)
        self.n_minus = int(self.x_minus.shape[0])
        self.y_minus = _check_vec("y_minus", y_minus, self.n_minus) if int(model) == nat.MH_UECM else None
        self.directed = bool(directed)
        # self.n is the + set's size: CSR offsets take n_plus + 1 per sample
        super().__init__(model, x_plus, y_plus, extra_flags=nat.MH_DIRECTED if self.directed else 0, **kw)

    def _workspace_bytes(self, capacity: int) -> int:
        return nat.mh_bipartite_workspace_size(self.model, self.n, self.n_minus, self.params(), capacity)

    def call(self, sample_begin: int | None = None, stream: torch.cuda.Stream | None = None) -> int:
        p = self.params(sample_begin)
        counts, stats = self._h_counts_p, self._h_stats_p
        return nat.mh_sample_bipartite(self.model, _ptr(self.x), _ptr(self.y), self.n, _ptr(self.x_minus),
                                       _ptr(self.y_minus), self.n_minus, p, _ptr(self.workspace), self.ws_bytes,
                                       _ptr(self.src), _ptr(self.dst), _ptr(self.w), _ptr(self.csr_off),
                                       _ptr(self.csr_idx), _ptr(self.csr_w), self.capacity, counts, stats,
                                       _stream_handle(stream))


def sample_bipartite(model: int, x_plus: torch.Tensor, y_plus, x_minus: torch.Tensor, y_minus, *,
                     directed: bool = False, **kw) -> SampleResult:
    """Samples of a bipartite or directed network (Sec. 2.6)."""
    return BipartiteSampler(model, x_plus, y_plus, x_minus, y_minus, directed=directed, **kw).run()


def sample_ubcm(x: torch.Tensor, **kw) -> SampleResult:
    """UBCM samples (Sec. 2.4); keyword arguments as in Sampler."""
    return Sampler(nat.MH_UBCM, x, None, **kw).run()


def sample_weighted(x: torch.Tensor, y: torch.Tensor, **kw) -> SampleResult:
    """UECM samples with integer weights (Sec. 2.5, Algorithm 1)."""
    return Sampler(nat.MH_UECM, x, y, **kw).run()


class BruteForceSampler:
    """Reusable buffers for the brute-force sampler (mh_sample_bf): every pair
    an independent Bernoulli draw (Sec. 2.2), COO output by (u, v); the
    comparison baseline of the walk (Sec. 3)."""

    def __init__(self, model: int, x: torch.Tensor, y: torch.Tensor | None = None, *, num_samples: int = 1,
                 seed: int = 0, network_id: int = 0, sample_begin: int = 0, fp64_only: bool = False,
                 capacity: int | None = None, chung_lu: bool = False):
        self.model = int(model)
        self.x = _check_vec("x", x)
        self.n = int(self.x.shape[0])
        self.y = _check_vec("y", y, self.n) if self.model == nat.MH_UECM else None
        self.num_samples = int(num_samples)
        self.seed, self.network_id, self.sample_begin = int(seed), int(network_id), int(sample_begin)
        self.flags = (nat.MH_OUT_COO | (nat.MH_FP64_ONLY if fp64_only else 0)
                      | (nat.MH_CHUNG_LU if chung_lu else 0))
        p = self.params()
        self.ws_bytes = nat.mh_bf_workspace_size(self.model, self.n, p)
        self.workspace = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=self.x.device)
        self.h_counts = np.zeros(self.num_samples, dtype=np.int64)
        self.h_stats = np.zeros(nat.MH_NUM_STATS, dtype=np.uint64)
        self._alloc(capacity if capacity is not None else max(1024, 16 * self.n * self.num_samples))

    def params(self, sample_begin: int | None = None) -> nat.MhParams:
        return nat.make_params(seed=self.seed, network_id=self.network_id,
                               sample_begin=self.sample_begin if sample_begin is None else sample_begin,
                               num_samples=self.num_samples, flags=self.flags)

    def _alloc(self, capacity: int):
        self.capacity = int(capacity)
        dev = self.x.device
        self.src = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.dst = torch.empty_like(self.src)
        self.w = torch.empty_like(self.src) if self.model == nat.MH_UECM else None

    def call(self, sample_begin: int | None = None, stream: torch.cuda.Stream | None = None) -> int:
        return nat.mh_sample_bf(self.model, _ptr(self.x), _ptr(self.y), self.n, self.params(sample_begin),
                                _ptr(self.workspace), self.ws_bytes, _ptr(self.src), _ptr(self.dst), _ptr(self.w),
                                self.capacity, self.h_counts.ctypes.data_as(ctypes.c_void_p),
                                self.h_stats.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream))

    def run(self, sample_begin: int | None = None, stream: torch.cuda.Stream | None = None) -> SampleResult:
        for _ in range(4):
            rc = self.call(sample_begin, stream)
            if rc == nat.MH_ERR_CAPACITY:
                self._alloc(int(self.h_counts.sum() * 1.05) + 1024)
                continue
            nat.check(rc, "mh_sample_bf")
            tot = int(self.h_counts.sum())
            return SampleResult(self.h_counts.copy(), self.h_stats.copy(), self.src[:tot], self.dst[:tot],
                                None if self.w is None else self.w[:tot])
        raise RuntimeError("sampling did not converge on buffer sizes")


def segment_table(model: int, x: torch.Tensor, y: torch.Tensor | None = None, *, seg_target: int = 0,
                  bound: str = "suffix", max_segments: int = 0) -> dict:
    """The node order and row-segment table a sampling call walks (numpy arrays)."""
    x = _check_vec("x", x)
    n = int(x.shape[0])
    y = _check_vec("y", y, n) if model == nat.MH_UECM else None
    flags = nat.MH_BOUND_PAPER if bound == "paper" else 0
    for _ in range(4):
        p = nat.make_params(seg_target=seg_target, flags=flags, max_segments=max_segments)
        ws_bytes = nat.mh_workspace_size(model, n, p, 0)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=x.device)
        cap = max_segments if max_segments > 0 else 4 * n + 1024
        row = torch.empty(cap, dtype=torch.int32, device=x.device)
        k = torch.empty(cap, dtype=torch.int32, device=x.device)
        a = torch.empty(cap, dtype=torch.int64, device=x.device)
        b = torch.empty(cap, dtype=torch.int64, device=x.device)
        perm = torch.empty(n, dtype=torch.int32, device=x.device)
        S = ctypes.c_int64(0)
        rc = nat.mh_segment_table(model, _ptr(x), _ptr(y), n, p, _ptr(ws), ws_bytes, _ptr(row), _ptr(k), _ptr(a),
                                  _ptr(b), _ptr(perm), cap, ctypes.byref(S), _stream_handle(None))
        if rc in (nat.MH_ERR_WORKSPACE, nat.MH_ERR_CAPACITY) and S.value > cap:
            max_segments = int(S.value)
            continue
        nat.check(rc, "mh_segment_table")
        s = S.value
        return dict(row=row[:s].cpu().numpy(), k=k[:s].cpu().numpy(), a=a[:s].cpu().numpy(),
                    b=b[:s].cpu().numpy(), perm=perm.cpu().numpy())
    raise RuntimeError("segment table did not fit")


def row_shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """(row_begin, row_count) of rank `rank` out of `world` for the pairwise
    sums: contiguous blocks whose sizes differ by at most one, in rank order."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def _row_range(rows, n: int) -> tuple[int, int]:
    if rows is None:
        return 0, n
    begin, count = (int(v) for v in rows)
    return begin, count


class SymWorkspace:
    """Device scratch of the symmetric pair sums (maxent_expected_*_sym):
    one buffer, grown to the largest (model, n) asked for on its device."""

    def __init__(self):
        self.buf = None

    def get(self, model: int, n: int, device) -> tuple[torch.Tensor, int]:
        rc, need = nat.maxent_expected_sym_workspace_size(model, n)
        nat.check(rc, "maxent_expected_sym_workspace_size")
        if self.buf is None or self.buf.numel() < need or self.buf.device != torch.device(device):
            self.buf = None
            self.buf = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
        return self.buf, need


def _sym_args(sym, model, n, device, rows):
    if rows is not None:
        raise ValueError("the symmetric pair sums cover all rows; rows needs the row form")
    ws, need = sym.get(model, n, device)
    return _ptr(ws), need


def expected_fwd(model: int, x: torch.Tensor, y: torch.Tensor | None = None, stream=None, rows=None,
                 sym: SymWorkspace | None = None):
    """(<k>, <s>) as FP64 CUDA tensors (<s> is None for UBCM).  rows =
    (row_begin, row_count) computes only those rows (outputs of row_count
    entries), bit for bit the values of the whole call.  sym = a
    SymWorkspace evaluates each unordered pair once for both rows (all rows;
    within rounding of the row form, not bit for bit)."""
    x = _check_vec("x", x)
    n = int(x.shape[0])
    y = _check_vec("y", y, n) if model == nat.MH_UECM else None
    begin, count = _row_range(rows, n)
    k = torch.empty(max(count, 0), dtype=torch.float64, device=x.device)
    s = torch.empty_like(k) if model == nat.MH_UECM else None
    if sym is not None:
        ws, need = _sym_args(sym, model, n, x.device, rows)
        rc = nat.maxent_expected_fwd_sym(model, _ptr(x), _ptr(y), n, _ptr(k), _ptr(s), ws, need,
                                         _stream_handle(stream))
    elif rows is None:
        rc = nat.maxent_expected_fwd(model, _ptr(x), _ptr(y), n, _ptr(k), _ptr(s), _stream_handle(stream))
    else:
        rc = nat.maxent_expected_fwd_rows(model, _ptr(x), _ptr(y), n, begin, count, _ptr(k), _ptr(s),
                                          _stream_handle(stream))
    nat.check(rc, "maxent_expected_fwd")
    return k, s


def expected_bwd(model: int, x: torch.Tensor, y: torch.Tensor | None, g_k: torch.Tensor,
                 g_s: torch.Tensor | None = None, stream=None, rows=None, sym: SymWorkspace | None = None,
                 f32: bool = False):
    """(dL/dx, dL/dy) given dL/d<k>, dL/d<s> (FP64 CUDA tensors); rows and
    sym as in expected_fwd.  f32 (with sym): FP32 pair terms, within about
    1e-5 of the sum of the terms' magnitudes (Newton directions)."""
    x = _check_vec("x", x)
    n = int(x.shape[0])
    y = _check_vec("y", y, n) if model == nat.MH_UECM else None
    g_k = _check_vec("g_k", g_k, n)
    g_s = _check_vec("g_s", g_s, n) if model == nat.MH_UECM else None
    begin, count = _row_range(rows, n)
    gx = torch.empty(max(count, 0), dtype=torch.float64, device=x.device)
    gy = torch.empty_like(gx) if model == nat.MH_UECM else None
    if f32 and sym is None:
        raise ValueError("f32 needs the symmetric form (sym=SymWorkspace())")
    if sym is not None:
        ws, need = _sym_args(sym, model, n, x.device, rows)
        fn = nat.maxent_expected_bwd_sym_f32 if f32 else nat.maxent_expected_bwd_sym
        rc = fn(model, _ptr(x), _ptr(y), n, _ptr(g_k), _ptr(g_s), _ptr(gx), _ptr(gy), ws, need,
                _stream_handle(stream))
    elif rows is None:
        rc = nat.maxent_expected_bwd(model, _ptr(x), _ptr(y), n, _ptr(g_k), _ptr(g_s), _ptr(gx), _ptr(gy),
                                     _stream_handle(stream))
    else:
        rc = nat.maxent_expected_bwd_rows(model, _ptr(x), _ptr(y), n, begin, count, _ptr(g_k), _ptr(g_s),
                                          _ptr(gx), _ptr(gy), _stream_handle(stream))
    nat.check(rc, "maxent_expected_bwd")
    return gx, gy


def expected_jacobian_diag(model: int, x: torch.Tensor, y: torch.Tensor | None = None, stream=None, rows=None,
                           sym: SymWorkspace | None = None, f32: bool = False):
    """(d<k>/dx,) for the UBCM or (d<k>/dx, d<k>/dy, d<s>/dx, d<s>/dy) for the
    UECM: each node's derivatives of its own expected degree (and strength)
    with respect to its own parameters, FP64 CUDA tensors; rows, sym and f32
    as in expected_fwd and expected_bwd."""
    x = _check_vec("x", x)
    n = int(x.shape[0])
    y = _check_vec("y", y, n) if model == nat.MH_UECM else None
    begin, count = _row_range(rows, n)
    outs = [torch.empty(max(count, 0), dtype=torch.float64, device=x.device)
            for _ in range(1 if model == nat.MH_UBCM else 4)]
    ptrs = [_ptr(t) for t in outs] + [None] * (4 - len(outs))
    if f32 and sym is None:
        raise ValueError("f32 needs the symmetric form (sym=SymWorkspace())")
    if sym is not None:
        ws, need = _sym_args(sym, model, n, x.device, rows)
        fn = nat.maxent_expected_jacobian_diag_sym_f32 if f32 else nat.maxent_expected_jacobian_diag_sym
        rc = fn(model, _ptr(x), _ptr(y), n, *ptrs, ws, need, _stream_handle(stream))
    elif rows is None:
        rc = nat.maxent_expected_jacobian_diag(model, _ptr(x), _ptr(y), n, *ptrs, _stream_handle(stream))
    else:
        rc = nat.maxent_expected_jacobian_diag_rows(model, _ptr(x), _ptr(y), n, begin, count, *ptrs,
                                                    _stream_handle(stream))
    nat.check(rc, "maxent_expected_jacobian_diag")
    return tuple(outs)
