"""Autotuner for the sampler's schedule: segment length and walk block shape.

Two knobs are tuned by timing probe calls on the GPU:

* seg_target T, the expected proposals per row segment.  A smaller T cuts
  rows into more, shorter segments (more independent work, more segment
  heads and per-item bookkeeping); a larger T gives fewer, longer segments
  (longer per-lane chains and a rougher load balance at the end of a
  launch).  T is part of a sample's identity: every segment head restarts
  the proposal bound and the Philox counter's segment index, so a different
  T draws different (equally exact) samples.  The tuner only chooses T;
  pass the chosen value as seg_target to reproduce samples.
* walk_ctas_per_sm, the persistent walk launch's blocks per SM (0 = as many
  as fit).  It changes the schedule only, never a sampled bit.

Probe calls run with MH_TIMING, so times are device times from CUDA events;
a candidate's score is sampled edges per millisecond of device time.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as nat
from .ensemble import Ensemble
from .sampler import Sampler

DEFAULT_T = 32


@dataclass
class TuneResult:
    seg_target: int
    walk_ctas_per_sm: int
    table: list = field(default_factory=list)  # one dict per candidate: T, ctas, ms, edges, edges_per_ms

    def as_dict(self):
        return {"seg_target": self.seg_target, "walk_ctas_per_sm": self.walk_ctas_per_sm, "table": self.table}


def pick(table, *, default_t: int = DEFAULT_T, tie: float = 0.01):
    """(T, ctas) of the fastest candidate.  Candidates within `tie` (relative)
    of the best rate count as equal; among them the default T wins, then the
    larger T (fewer segments), then ctas = 0 (full occupancy), then fewer
    blocks, so the choice is deterministic for a given table."""
    if not table:
        raise ValueError("empty tuning table")
    best = max(r["edges_per_ms"] for r in table)
    near = [r for r in table if r["edges_per_ms"] >= best * (1.0 - tie)]
    near.sort(key=lambda r: (r["T"] != default_t, -r["T"], r["ctas"] != 0, r["ctas"]))
    return near[0]["T"], near[0]["ctas"]


def tune_sampler(model: int, x: torch.Tensor, y: torch.Tensor | None = None, *, candidates_t=(8, 16, 32, 64, 128),
                 candidates_ctas=(0, 2), num_samples: int = 4, reps: int = 3, seed: int = 0, layout: str = "coo",
                 stream=None) -> TuneResult:
    """Times mh_sample_* calls of num_samples samples for every (T, ctas)."""
    table = []
    for T, ctas in itertools.product(candidates_t, candidates_ctas):
        s = Sampler(model, x, y, num_samples=num_samples, seed=seed, seg_target=T, layout=layout,
                    walk_ctas_per_sm=ctas)
        s.run(stream=stream)                 # sizes buffers and the segment table
        s.flags |= nat.MH_TIMING
        nat.check(s.call(stream=stream), "mh_sample")
        ms, edges = 0.0, 0
        for _ in range(reps):
            nat.check(s.call(stream=stream), "mh_sample")
            ms += nat.mh_last_call_info().total_ms
            edges += int(s.h_counts.sum())
        table.append({"T": T, "ctas": ctas, "ms": ms / reps, "edges": edges // reps,
                      "edges_per_ms": edges / ms if ms > 0 else 0.0})
    T, ctas = pick(table)
    return TuneResult(T, ctas, table)


def tune_ensemble(networks, *, candidates_t=(16, 32, 64), candidates_ctas=(0, 2), num_samples: int = 2,
                  reps: int = 2, seed: int = 0, layout: str = "csr", capacity: int = 1 << 26,
                  max_wave_items: int = 1 << 26) -> TuneResult:
    """Times whole probe ensembles (prepare + every pair of num_samples
    samples per network, in waves) for every (T, ctas)."""
    table = []
    for T, ctas in itertools.product(candidates_t, candidates_ctas):
        ens = Ensemble(networks, num_samples=num_samples, seed=seed, seg_target=T, layout=layout,
                       capacity=capacity, max_wave_items=max_wave_items, walk_ctas_per_sm=ctas)
        ens.sample()                          # warm-up: buffers, workspace, wave estimates
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, edges = 0.0, 0
        for _ in range(reps):
            stream = torch.cuda.current_stream()
            ev0.record(stream)
            ens.prepare()
            counts, _ = ens.sample()
            ev1.record(stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            edges += int(np.sum(counts))
        table.append({"T": T, "ctas": ctas, "ms": ms / reps, "edges": edges // reps,
                      "edges_per_ms": edges / ms if ms > 0 else 0.0})
        del ens
    T, ctas = pick(table)
    return TuneResult(T, ctas, table)
