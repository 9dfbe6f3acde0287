"""Benchmark: sampled edges/s of batched Miller-Hagberg ensembles on one GB300.

One step = the 128-network ensemble (N log-uniform in [10^3, 10^6], 64 UBCM
and 64 UECM networks, capped Pareto fitness with mean expected degree about
20, y ~ U(0.3, 0.9)), 64 samples of every network as CSR (int64 offsets,
int32 indices and weights): mh_batch_prepare (node sorts, bound preparation,
row-segment tables of all networks) and every (network, sample) pair in
mh_sample_batched waves.  Inputs resident in HBM; the L2 is flushed (a
512 MiB write) before every timed step.  Beside it: the same samples drawn by
one call per (network, sample) (the per-sample launch loop), end to end with
the inputs copied from pinned host memory, the walk's roofline, the oracle on
a bounded sample.  Under torchrun rank r draws samples [64 r, 64 r + 64) of
every network (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  At N = 1 the line also carries the other
workloads as sub-objects (the weighted N = 20,000 call, the lognormal
ensemble, the pairwise sums, fit-then-sample, bipartite and directed
networks, the other configurations, output layouts).  `--impl reference`
times the CPU oracle (the serial FP64 walk, one sample of one ensemble
network per step) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "uecm_n20k_x10"
SAMPLES_PER_STEP = 10
BYTES_PER_EDGE = 12          # int32 src + int32 dst + int32 weight
METRIC = "sampled edges/s on 1 GB300 (batched vs per-sample loop), % HBM write roofline"
WALK_SOURCES = ["paper_2509_13230_gb300/csrc/walk.cu", "paper_2509_13230_gb300/csrc/walk_math.cuh",
                "paper_2509_13230_gb300/csrc/mh_internal.cuh"]
WALK_PROFILE = os.path.join(ROOT, "profiles", "walk_kernel_uecm_n20k_x10.json")
FALLBACK_HBM_GBS = 6800.0


def workload():
    from paper_2509_13230_gb300 import workloads
    return workloads.uecm_n20k()


def walk_traffic(T: int):
    """DRAM bytes per walk launch of the 10-sample weighted call at segment
    length T, from the ncu capture in profiles/ while the walk sources are
    unchanged since it (else None)."""
    if os.path.exists(WALK_PROFILE):
        prof = json.load(open(WALK_PROFILE))
        if prof.get("sources_sha") == sources_hash():
            return prof.get("dram_bytes_per_launch_by_seg_target", {}).get(str(T))
    return None


def sources_hash() -> str:
    h = hashlib.sha256()
    for p in WALK_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def rejected(clocks) -> bool:
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clocks.get("reasons", [])):
        return True
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.5 * mx and not clocks.get("reasons"))


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_rate(net, seconds: float, first_sample: int = 0):
    """Edges/s of the serial oracle over whole samples, for about `seconds`."""
    import oracle
    oracle.load()
    edges, t_total, s = 0, 0.0, first_sample
    while t_total < seconds:
        t0 = time.perf_counter()
        _, _, _, counts, _ = oracle.mh_sample(oracle.UECM, net.x, net.y, sample_begin=s, num_samples=1)
        t_total += time.perf_counter() - t0
        edges += int(counts.sum())
        s += 1
    return edges / t_total, s - first_sample, t_total


def _oracle_worker(x, y, first_sample: int, stride: int, seconds: float):
    """One process of the all-cores oracle baseline: samples first, first +
    stride, ... for about `seconds`; returns (edges, samples, busy seconds)."""
    import oracle
    edges, t_total, s, k = 0, 0.0, first_sample, 0
    while t_total < seconds:
        t0 = time.perf_counter()
        _, _, _, counts, _ = oracle.mh_sample(oracle.UECM, x, y, sample_begin=s, num_samples=1)
        t_total += time.perf_counter() - t0
        edges += int(counts.sum())
        s += stride
        k += 1
    return edges, k, t_total


def oracle_rate_all_cores(net, seconds: float):
    """Edges/s of the serial oracle with one process per host core (spawned,
    so no process inherits a CUDA context), each drawing whole samples."""
    import concurrent.futures
    import multiprocessing

    import oracle
    oracle.load()  # built once before the workers load it
    cores = os.cpu_count() or 1
    ctx = multiprocessing.get_context("spawn")
    t0 = time.perf_counter()
    with concurrent.futures.ProcessPoolExecutor(max_workers=cores, mp_context=ctx) as ex:
        futs = [ex.submit(_oracle_worker, net.x, net.y, c, cores, seconds) for c in range(cores)]
        res = [f.result() for f in futs]
    wall = time.perf_counter() - t0
    edges = sum(r[0] for r in res)
    # the workers run concurrently; the rate is over the longest worker's busy time
    busy = max(r[2] for r in res)
    return edges / busy, sum(r[1] for r in res), busy, wall, cores


def oracle_bf_time(net):
    """Seconds of one brute-force sample of the oracle (every pair a Bernoulli)."""
    import oracle
    t0 = time.perf_counter()
    _, _, _, evals = oracle.bf_sample(oracle.UECM, net.x, net.y)
    return time.perf_counter() - t0, evals


def run_reference(args, rank):
    """The oracle (serial FP64 walk, one host core) on a bounded sample of the
    headline's ensemble: step k draws one sample of one network, cycling
    through the ensemble's networks of at most REF_MAX_N nodes in size order."""
    if rank != 0:
        return
    import oracle

    from paper_2509_13230_gb300 import workloads
    oracle.load()
    nets = [(t, nw) for t, nw in enumerate(workloads.ensemble_128()) if nw.n <= REF_MAX_N]
    nets.sort(key=lambda e: e[1].n)
    T = args.ensemble_seg_target or 16

    def step(k):
        t, nw = nets[k % len(nets)]
        t0 = time.perf_counter()
        _, _, _, counts, _ = oracle.mh_sample(nw.model, nw.x, nw.y, network_id=t, sample_begin=k // len(nets),
                                              num_samples=1, seg_target=T)
        return time.perf_counter() - t0, int(counts.sum())

    for w in range(args.warmup):
        step(w)
    edges, t = 0, 0.0
    for k in range(args.steps):
        dt, e = step(k)
        t += dt
        edges += e
    value = edges / t
    sample = (f"one sample of one network per step, cycling through the {len(nets)} networks of the 128-network "
              f"ensemble with at most {REF_MAX_N} nodes in size order; serial FP64 oracle, one host core")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ENSEMBLE_WORKLOAD, "networks": len(nets), "samples_per_step": 1,
                       "seg_target": T, "output": "coo int32 (+ int32 weights for the UECM networks)"},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


REF_MAX_N = 200_000


# ---------------------------------------------------------------------------
# Batched ensemble leg: 128 networks (N log-uniform in [10^3, 10^6], half
# UBCM, half UECM, capped Pareto fitness), 64 samples each, CSR output.
# ---------------------------------------------------------------------------
ENSEMBLE_SAMPLES = 64


def ensemble_leg(args, dev, flush, fitness="pareto", samples=None, capacity=None, seg_target=None,
                 loop_samples=None):
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300 import workloads
    from paper_2509_13230_gb300.ensemble import Ensemble
    from paper_2509_13230_gb300.sampler import Sampler

    nets_np = workloads.ensemble_128(fitness=fitness)
    keep = max(1, min(args.ensemble_networks, len(nets_np)))
    nets_np = [nets_np[t] for t in np.linspace(0, len(nets_np) - 1, keep).round().astype(int)]
    nets = [(nw.model, torch.from_numpy(nw.x).to(dev), None if nw.y is None else torch.from_numpy(nw.y).to(dev), t)
            for t, nw in enumerate(nets_np)]
    n = np.array([nw.n for nw in nets_np], dtype=np.int64)
    uecm = np.array([nw.model == nat.MH_UECM for nw in nets_np])
    samples = samples or args.ensemble_samples
    capacity = capacity or args.ensemble_capacity
    tuned = None
    T, ctas = 0, 0
    if seg_target is not None:
        T = seg_target
    elif args.ensemble_seg_target:
        T = args.ensemble_seg_target
    elif not args.no_tune:
        from paper_2509_13230_gb300.autotune import tune_ensemble
        tuned = tune_ensemble(nets, candidates_t=(8, 16, 32), candidates_ctas=(0, 2), num_samples=2, reps=2)
        T, ctas = tuned.seg_target, tuned.walk_ctas_per_sm
    ens = Ensemble(nets, num_samples=samples, layout="csr", capacity=capacity, timing=True, seg_target=T,
                   walk_ctas_per_sm=ctas, max_wave_items=args.ensemble_wave_items)
    stream = torch.cuda.current_stream()
    walk = {"ms": 0.0, "emit_ms": 0.0, "prepare_ms": 0.0}

    def on_wave(res):
        info = nat.mh_last_call_info()
        walk["ms"] += info.walk_ms
        walk["emit_ms"] += info.emit_ms

    def one_pass():
        ens.prepare()                # sort + segment tables are part of a step
        walk["prepare_ms"] += nat.mh_last_call_info().prepare_ms
        return ens.sample(on_wave=on_wave)

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 3))
    total_ms, edges, out_bytes, waves, proposals = 0.0, 0, 0, 0, 0
    for k in walk:
        walk[k] = 0.0
    for _ in range(steps):
        flush.zero_()
        ev0.record(stream)
        counts, st = one_pass()
        proposals += int(st[nat.MH_STAT_PROPOSALS])
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        edges += int(counts.sum())
        per_net = counts.reshape(len(nets), samples).sum(axis=1)
        out_bytes += int((4 * per_net + 4 * per_net * uecm + 8 * (n + 1) * samples).sum())
        waves += ens.waves_run
    value = edges / (total_ms / 1e3)

    # per-sample loop: one mh_sample_* call per (network, sample), same networks
    loop_ms, loop_edges = 0.0, 0
    loop_samples = args.ensemble_loop_samples if loop_samples is None else loop_samples
    for (m, x, y, nid) in (nets if loop_samples > 0 else []):
        s1 = Sampler(m, x, y, num_samples=1, network_id=nid, layout="csr", seg_target=T, walk_ctas_per_sm=ctas)
        s1.run()
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(loop_samples):
            nat.check(s1.call(sample_begin=k), "mh_sample")
            loop_edges += int(s1.h_counts.sum())
        ev1.record(stream)
        ev1.synchronize()
        loop_ms += ev0.elapsed_time(ev1)
        del s1
    loop_value = loop_edges / (loop_ms / 1e3) if loop_ms > 0 else None
    del ens
    torch.cuda.empty_cache()
    hbm_gbs, peak_kind = peaks()
    # the oracle on a bounded sample of the same ensemble: whole samples of
    # the networks in size order, up to about 8 s of one host core
    import oracle
    oracle.load()
    cpu_edges, cpu_s, cpu_pairs = 0, 0.0, 0
    for t in np.argsort(n):
        if cpu_s > 8.0:
            break
        nw = nets_np[t]
        t0 = time.perf_counter()
        _, _, _, c, _ = oracle.mh_sample(nw.model, nw.x, nw.y, network_id=nets[t][3], num_samples=1,
                                         seg_target=T or 32)
        cpu_s += time.perf_counter() - t0
        cpu_edges += int(c.sum())
        cpu_pairs += 1
    walk_ms = walk["ms"] / steps
    return {
        "workload": f"ensemble_{len(nets)}_x{samples}" + ("" if fitness == "pareto" else f"_{fitness}"),
        "fitness": fitness, "networks": len(nets), "nodes": int(n.sum()),
        "samples_per_network": samples, "value": value, "unit": "edges/s", "ms_per_step": total_ms / steps,
        "edges_per_step": edges // steps, "proposals_per_step": proposals // steps, "waves_per_step": waves / steps,
        "output": "CSR int64 offsets + int32 indices (+ int32 weights for the UECM half)",
        "write_gbs_of_step": out_bytes / steps / (total_ms / steps / 1e3) / 1e9,
        "walk_ms_per_step": walk_ms,
        "prepare_ms_per_step": walk["prepare_ms"] / steps,
        "scan_emit_ms_per_step": walk["emit_ms"] / steps,
        "write_gbs_of_walk": out_bytes / steps / (walk_ms / 1e3) / 1e9 if walk_ms > 0 else None,
        "hbm_peak": hbm_gbs, "peak_kind": peak_kind,
        "roofline": {"bound": "hbm", "kernel": "walk_kernel (batched, both models)",
                     "achieved": out_bytes / steps / (walk_ms / 1e3) / 1e9 if walk_ms > 0 else None,
                     "peak": hbm_gbs, "unit": "GB/s",
                     "frac": (out_bytes / steps / (walk_ms / 1e3) / 1e9) / hbm_gbs if walk_ms > 0 else None,
                     "traffic": None, "basis": "CSR output bytes (4 B index, 4 B UECM weight, 8 B per offset) / "
                                               "walk time of the step (both walks' fork-join interval per wave)"},
        "cpu_baseline": {"value": cpu_edges / cpu_s, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": f"one sample of each of the {cpu_pairs} smallest networks of the ensemble, "
                                   f"serial FP64 walk, {cpu_s:.1f} s on one host core"},
        "per_sample_loop": None if loop_value is None else {
            "value": loop_value, "unit": "edges/s", "calls": len(nets) * loop_samples,
            "samples_per_network": loop_samples, "batched_over_loop": value / loop_value},
        "step": "mh_batch_prepare of all networks + every (network, sample) pair in waves",
        "seg_target": T or 32, "walk_ctas_per_sm": ctas,
        "autotune": None if tuned is None else {
            "probe": "all networks x 2 samples, prepare + waves, CUDA events", "table": tuned.table},
    }


# ---------------------------------------------------------------------------
# Pairwise leg: expected degrees / strengths and their gradient (UECM, N =
# 200,000, the size of the fitting workload), the O(N^2) sums of inference.
# ---------------------------------------------------------------------------
PAIR_N = 200_000
# FP32 operations per ordered pair of the UECM double-float evaluation,
# counted from its operation sequence (two_sum 6, fast_two_sum 3, products 4
# and quotients 8 plus a reciprocal, both left unnormalised, sloppy addition
# 11, 1 - r 7, accumulation 8 per term plus a 6-operation renormalisation
# every 8 terms).  Forward: a_i a_j, y_i y_j, 1 - r, D, two divisions, two
# sums.  Backward: r, 1 - r, A, D, D^2, Q, g_k and g_s sums, the x term and
# the y term, two sums.  Jacobian diagonal: A, r, 1 - r, D, D^2, Q, (1 - r) Q,
# r D, 1 - r + r D, (1 - r)^2, a division and a product, three sums.
PAIR_OPS = {"fwd": 59, "bwd": 142, "jacobian_diag": 99}
# the symmetric forms, per unordered pair (products and quotients without the
# renormalising fast_two_sum: 4 and 8 operations plus the reciprocal): the
# shared terms once (forward 42, backward 141, Jacobian diagonal 97), both
# rows' and both columns' accumulations (8 per term and 6 per 8-term
# renormalisation: 35 for two quantities, 53 for three)
PAIR_SYM_OPS = {"fwd": 77, "bwd": 176, "jacobian_diag": 150}
# the FP32 forms (Newton directions): r, 1 - r, D, D^2, the factor
# (1 - r + r D) / (1 - r)^2 (3, with two reciprocals), then bwd: g sums (2),
# U and V (4), four products; diag: two products, six; both: the row sums and
# the column sums (two rows' column terms added before the shuffle)
PAIR_SYM_F32_OPS = {"bwd": 21, "jacobian_diag": 21}
FP32_LANES_PER_SM = 128


def pairwise_inputs(dev):
    """Heavy-tailed x (log-normal), y ~ U(0.3, 0.9) and standard normal
    gradients for the pairwise leg (seeded)."""
    import torch
    rng = np.random.default_rng(11)
    x_np = np.exp(rng.normal(-5.5, 1.3, PAIR_N))
    y_np = rng.uniform(0.3, 0.9, PAIR_N)
    x = torch.from_numpy(x_np).to(dev)
    y = torch.from_numpy(y_np).to(dev)
    gk = torch.from_numpy(rng.normal(size=PAIR_N)).to(dev)
    gs = torch.from_numpy(rng.normal(size=PAIR_N)).to(dev)
    return rng, x_np, y_np, x, y, gk, gs


def kernels_once(dev):
    """Each profiled kernel once, untimed, for ncu captures: the headline call
    (10 samples of the weighted N = 20,000 workload) at segment lengths 8, 16
    and 32 (three walk launches, in that order), then the UECM pairwise
    forward, backward and Jacobian diagonal at N = 200,000 (one launch each)."""
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300.sampler import Sampler, expected_bwd, expected_fwd, expected_jacobian_diag

    net = workload()
    x = torch.from_numpy(net.x).to(dev)
    y = torch.from_numpy(net.y).to(dev)
    edges = {}
    for T in (8, 16, 32):
        res = Sampler(nat.MH_UECM, x, y, num_samples=SAMPLES_PER_STEP, seg_target=T).run()
        edges[T] = res.total
    _, _, _, px, py, gk, gs = pairwise_inputs(dev)
    expected_fwd(nat.MH_UECM, px, py)
    expected_bwd(nat.MH_UECM, px, py, gk, gs)
    expected_jacobian_diag(nat.MH_UECM, px, py)
    torch.cuda.synchronize()
    return {"workload": WORKLOAD, "edges_by_seg_target": edges, "pairwise_n": PAIR_N}


def pairwise_leg(args, dev, sm_mhz):
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300.sampler import SymWorkspace, expected_bwd, expected_fwd, expected_jacobian_diag

    rng, x_np, y_np, x, y, gk, gs = pairwise_inputs(dev)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    ws = SymWorkspace()
    for kind in ("fwd", "bwd", "jacobian_diag", "fwd_sym", "bwd_sym", "jacobian_diag_sym", "bwd_sym_f32",
                 "jacobian_diag_sym_f32"):
        f32 = kind.endswith("_f32")
        sym = ws if "_sym" in kind else None
        base = kind.split("_sym")[0]

        def call():
            if base == "fwd":
                return expected_fwd(nat.MH_UECM, x, y, sym=sym)
            if base == "jacobian_diag":
                return expected_jacobian_diag(nat.MH_UECM, x, y, sym=sym, f32=f32)
            return expected_bwd(nat.MH_UECM, x, y, gk, gs, sym=sym, f32=f32)
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize()
        reps = 5
        with ClockSampler(dev.index or 0) as clk:
            ev0.record(stream)
            for _ in range(reps):
                call()
            ev1.record(stream)
            ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        pairs = PAIR_N * (PAIR_N - 1)
        if sym is None:
            out[kind] = {"ms": ms, "pairs_per_s": pairs / (ms / 1e3), "fp32_ops_per_pair": PAIR_OPS[kind],
                         "achieved_gops": PAIR_OPS[kind] * pairs / (ms / 1e3) / 1e9, "clocks": clk.summary()}
        else:
            # one evaluation per unordered pair serves both rows
            ops = (PAIR_SYM_F32_OPS if f32 else PAIR_SYM_OPS)[base]
            out[kind] = {"ms": ms, "unordered_pairs_per_s": pairs / 2 / (ms / 1e3),
                         "fp32_ops_per_unordered_pair": ops,
                         "achieved_gops": ops * pairs / 2 / (ms / 1e3) / 1e9,
                         "speedup_over_row_form": out[base]["ms"] / ms, "clocks": clk.summary()}
    import torch.cuda as tc
    sms = tc.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz or 2070.0
    peak = sms * FP32_LANES_PER_SM * mhz * 1e6 / 1e9
    for kind in out:
        out[kind]["frac"] = out[kind]["achieved_gops"] / peak
    # the oracle (compensated FP64 sums, one host core) on a few sampled rows
    import oracle
    rows = rng.choice(PAIR_N, 4, replace=False)
    t0 = time.perf_counter()
    oracle.expected_fwd(oracle.UECM, x_np, y_np, rows=rows)
    t_cpu = time.perf_counter() - t0
    return {"workload": f"uecm_pairwise_n{PAIR_N // 1000}k", "n": PAIR_N, "bound": "alu",
            "peak_gops": peak, "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz "
                                              "(median SM clock of the sampler's timed region)",
            **out,
            "cpu_baseline": {"value": len(rows) * (PAIR_N - 1) / t_cpu, "unit": "pairs/s (forward)", "cores": 1,
                             "kind": "oracle", "sample": f"{len(rows)} rows of the forward sums, FP64 compensated"}}


# ---------------------------------------------------------------------------
# Fit-then-sample leg: degree and strength targets for N = 200,000 (discrete
# power law 2.5 on [2, 2000], s = k U(1, 5)), x and y fitted to a 1e-8
# relative residual, then 1,000 weighted networks drawn in batched waves.
# ---------------------------------------------------------------------------
FIT_N = 200_000
FIT_SAMPLES = 1000


def fit_leg(args, dev):
    import torch

    import oracle
    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300 import workloads
    from paper_2509_13230_gb300.ensemble import Ensemble
    from paper_2509_13230_gb300.expected import fit

    # warm-up (untimed): a fit of 20,000 nodes, so that the torch kernels of the
    # fit's vector algebra are loaded (their first use costs 0.25-1.6 s each)
    k_w, s_w = workloads.degree_strength_targets(n=20_000)
    fit(torch.from_numpy(k_w).to(dev), torch.from_numpy(s_w).to(dev), tol=1e-8)
    k_np, s_np = workloads.degree_strength_targets(n=FIT_N)
    k_t = torch.from_numpy(k_np).to(dev)
    s_t = torch.from_numpy(s_np).to(dev)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # count the pairwise calls the fit makes (wrappers installed here only)
    from paper_2509_13230_gb300 import expected as expected_mod
    calls = {"fwd": 0, "bwd": 0, "jacobian_diag": 0}
    orig = expected_mod.expected_fwd, expected_mod.expected_bwd, expected_mod.expected_jacobian_diag

    def counted(kind, fn):
        def wrapper(*a, **kw):
            calls[kind] += 1
            return fn(*a, **kw)
        return wrapper

    expected_mod.expected_fwd = counted("fwd", orig[0])
    expected_mod.expected_bwd = counted("bwd", orig[1])
    expected_mod.expected_jacobian_diag = counted("jacobian_diag", orig[2])
    try:
        torch.cuda.synchronize()
        with ClockSampler(dev.index or 0) as clk:
            ev0.record(stream)
            res = fit(k_t, s_t, tol=1e-8)
            ev1.record(stream)
            ev1.synchronize()
    finally:
        expected_mod.expected_fwd, expected_mod.expected_bwd, expected_mod.expected_jacobian_diag = orig
    fit_ms = ev0.elapsed_time(ev1)
    # the oracle's compensated FP64 sums at the fitted parameters, on sampled rows
    rng = np.random.default_rng(12)
    rows = rng.choice(FIT_N, 6, replace=False)
    x_np, y_np = res.x.cpu().numpy(), res.y.cpu().numpy()
    kk, ss = oracle.expected_fwd(oracle.UECM, x_np, y_np, rows=rows)
    oracle_resid = float(max(np.max(np.abs(kk - k_np[rows]) / k_np[rows]),
                             np.max(np.abs(ss - s_np[rows]) / s_np[rows])))
    ens = Ensemble([(nat.MH_UECM, res.x, res.y, 0)], num_samples=FIT_SAMPLES, layout="coo", capacity=1 << 27)
    ens.sample()                                 # warm-up: buffers, estimates
    torch.cuda.synchronize()
    ev0.record(stream)
    ens.prepare()
    counts, _ = ens.sample()
    ev1.record(stream)
    ev1.synchronize()
    sample_ms = ev0.elapsed_time(ev1)
    edges = int(counts.sum())
    return {"workload": f"fit_uecm_n{FIT_N // 1000}k_then_x{FIT_SAMPLES}", "n": FIT_N,
            "fit_ms": fit_ms, "residual": res.residual, "residual_oracle_sampled_rows": oracle_resid,
            "adam_steps": res.adam_steps, "newton_steps": res.newton_steps,
            "warmup": "an untimed fit of 20,000 nodes first (loads the torch kernels of the vector algebra)",
            "pairwise_calls": calls, "fit_clocks": clk.summary(),
            "sample_ms": sample_ms, "samples": FIT_SAMPLES, "edges": edges,
            "edges_per_s": edges / (sample_ms / 1e3), "mean_degree": 2.0 * edges / FIT_SAMPLES / FIT_N,
            "target_mean_degree": float(k_np.mean()),
            "output": "COO int32 + w int32, 1,000 samples in batched waves"}


# ---------------------------------------------------------------------------
# Bipartite / directed leg (Sec. 2.6): a directed weighted network of 20,000
# nodes (10 samples per call, COO + weights) and a 200,000 x 20,000 bipartite
# unweighted network (2 samples per call, COO).
# ---------------------------------------------------------------------------
def bipartite_leg(args, dev, flush):
    import torch

    import oracle
    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300 import workloads
    from paper_2509_13230_gb300.autotune import pick
    from paper_2509_13230_gb300.sampler import BipartiteSampler

    hbm_gbs, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    out = {}
    xo, yo, xi, yi = workloads.directed_uecm_n20k()
    xp, xm = workloads.bipartite_ubcm_pareto()
    cases = [("directed_uecm_n20k_x10", nat.MH_UECM, (xo, yo, xi, yi), True, 10, 12),
             ("bipartite_ubcm_200k_20k_x2", nat.MH_UBCM, (xp, None, xm, None), False, 2, 8)]
    for name, model, arrays, directed, samples, bytes_per_edge in cases:
        t_arrays = [None if a is None else torch.from_numpy(a).to(dev) for a in arrays]
        # segment length from the autotuner's rule on a short probe
        table = []
        for T in (8, 16, 32):
            s = BipartiteSampler(model, *t_arrays, directed=directed, num_samples=samples, seg_target=T)
            s.run()
            s.flags |= nat.MH_TIMING
            ms, edges = 0.0, 0
            for _ in range(4):
                nat.check(s.call(), "mh_sample_bipartite")
                ms += nat.mh_last_call_info().total_ms
                edges += int(s.h_counts.sum())
            table.append({"T": T, "ctas": 0, "ms": ms / 4, "edges": edges // 4, "edges_per_ms": edges / ms})
        T, _ = pick(table)
        s = BipartiteSampler(model, *t_arrays, directed=directed, num_samples=samples, seg_target=T)
        s.run()
        s.flags |= nat.MH_TIMING
        for _ in range(args.warmup):
            nat.check(s.call(), "mh_sample_bipartite")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total_ms, edges = 0.0, 0
        phase = np.zeros(3)
        steps = max(args.steps, 5)
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            nat.check(s.call(), "mh_sample_bipartite")
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            info = nat.mh_last_call_info()
            phase += (info.prepare_ms, info.walk_ms, info.emit_ms)
            edges += int(s.h_counts.sum())
        walk_ms = phase[1]
        achieved = bytes_per_edge * edges / (walk_ms / 1e3) / 1e9
        t0 = time.perf_counter()
        _, _, _, c, _ = oracle.bip_sample(model, *arrays, directed=directed, num_samples=1, seg_target=T)
        cpu_s = time.perf_counter() - t0
        out[name] = {"value": edges / (total_ms / 1e3), "unit": "edges/s", "ms_per_step": total_ms / steps,
                     "samples_per_step": samples, "edges_per_step": edges // steps, "seg_target": T,
                     "phases_ms_per_step": dict(zip(("prepare", "walk", "scan_emit"), (phase / steps).tolist())),
                     "autotune": table,
                     "roofline": {"bound": "hbm", "kernel": "walk_kernel", "achieved": achieved, "peak": hbm_gbs,
                                  "unit": "GB/s", "frac": achieved / hbm_gbs, "traffic": None,
                                  "peak_kind": peak_kind, "walk_ms_per_step": walk_ms / steps,
                                  "bytes_per_edge": bytes_per_edge},
                     "cpu_baseline": {"value": int(c.sum()) / cpu_s, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                      "sample": f"one sample of the same network, serial FP64 walk, {cpu_s:.2f} s"}}
        del s
    return out


# ---------------------------------------------------------------------------
# The other single-network configurations: unweighted N = 1,000 x 100
# samples (COO) and unweighted Pareto N = 10^6, one sample (CSR); the
# oracle's serial walk and its brute-force sampler timed beside them.
# ---------------------------------------------------------------------------
def configs_leg(args, dev, flush):
    import torch

    import oracle
    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300 import workloads
    from paper_2509_13230_gb300.autotune import pick
    from paper_2509_13230_gb300.sampler import Sampler

    hbm_gbs, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    ubcm_bf_rate = None
    out = {}
    n1m = workloads.ubcm_pareto_n1m()
    cases = [("ubcm_n1k_x100", workloads.ubcm_n1k(), 100, "coo", 8, 0),
             ("ubcm_pareto_n1m_x1", n1m, 1, "csr", 4, 8),
             ("ubcm_pareto_n1m_x100_sustained", n1m, 100, "csr", 4, 8)]
    for name, net, samples, layout, bytes_per_edge, bytes_per_node in cases:
        x = torch.from_numpy(net.x).to(dev)
        table = []
        for T in (8, 16, 32):
            s = Sampler(nat.MH_UBCM, x, None, num_samples=samples, seg_target=T, layout=layout)
            s.run()
            s.flags |= nat.MH_TIMING
            ms, edges = 0.0, 0
            for _ in range(4):
                nat.check(s.call(), "mh_sample_ubcm")
                ms += nat.mh_last_call_info().total_ms
                edges += int(s.h_counts.sum())
            table.append({"T": T, "ctas": 0, "ms": ms / 4, "edges": edges // 4, "edges_per_ms": edges / ms})
            del s
        T, _ = pick(table)
        s = Sampler(nat.MH_UBCM, x, None, num_samples=samples, seg_target=T, layout=layout)
        s.run()
        s.flags |= nat.MH_TIMING
        for _ in range(args.warmup):
            nat.check(s.call(), "mh_sample_ubcm")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total_ms, edges, phase = 0.0, 0, np.zeros(3)
        steps = max(args.steps, 5)
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            nat.check(s.call(), "mh_sample_ubcm")
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            info = nat.mh_last_call_info()
            phase += (info.prepare_ms, info.walk_ms, info.emit_ms)
            edges += int(s.h_counts.sum())
        walk_ms = phase[1]
        out_bytes = bytes_per_edge * edges + bytes_per_node * (net.n + 1) * samples * steps
        achieved = out_bytes / (walk_ms / 1e3) / 1e9
        # oracle: a bounded share of the samples, and one brute-force sample
        k = min(samples, 10) if net.n < 1_000_000 else 1
        t0 = time.perf_counter()
        _, _, _, c, _ = oracle.mh_sample(oracle.UBCM, net.x, num_samples=k, seg_target=T)
        mh_s = time.perf_counter() - t0
        bf = None
        if net.n <= 20_000:
            t0 = time.perf_counter()
            _, _, _, evals = oracle.bf_sample(oracle.UBCM, net.x)
            bf_s = time.perf_counter() - t0
            bf = {"pairs_per_s": evals / bf_s, "seconds_per_sample": bf_s,
                  "mh_over_bf_speedup_cpu": bf_s / (mh_s / k)}
            ubcm_bf_rate = evals / bf_s
        else:
            # one brute-force sample evaluates every pair: extrapolated from the
            # UBCM brute-force rate measured on the smaller network above
            pairs = net.n * (net.n - 1) / 2
            bf = {"pairs": pairs, "note": "not run: extrapolated at the brute-force pair rate of the UBCM "
                                          "N = 1,000 network in this run"}
            if ubcm_bf_rate:
                bf["extrapolated_seconds_per_sample"] = pairs / ubcm_bf_rate
                bf["mh_over_bf_speedup_cpu_extrapolated"] = (pairs / ubcm_bf_rate) / (mh_s / k)
        out[name] = {"value": edges / (total_ms / 1e3), "unit": "edges/s", "ms_per_step": total_ms / steps,
                     "samples_per_step": samples, "edges_per_step": edges // steps, "seg_target": T,
                     "output": f"{layout} ({bytes_per_edge} B/edge" + (f" + {bytes_per_node} B/node)" if
                                                                      bytes_per_node else ")"),
                     "phases_ms_per_step": dict(zip(("prepare", "walk", "scan_emit"), (phase / steps).tolist())),
                     "autotune": table,
                     "roofline": {"bound": "hbm", "kernel": "walk_kernel", "achieved": achieved, "peak": hbm_gbs,
                                  "unit": "GB/s", "frac": achieved / hbm_gbs, "traffic": None,
                                  "peak_kind": peak_kind, "walk_ms_per_step": walk_ms / steps},
                     "cpu_baseline": {"value": int(c.sum()) / mh_s, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                      "sample": f"{k} samples of the same network, serial FP64 walk, {mh_s:.2f} s"},
                     "cpu_brute_force": bf}
        del s
    return out


# ---------------------------------------------------------------------------
# Brute force against the walk on the GPU (the comparison of the paper's
# Fig. 3A, Sec. 3.1, on synthetic Pareto fitness with mean degree about 20):
# one sample per call, device time of each, N from 10^3 to 10^6.
# ---------------------------------------------------------------------------
BF_SIZES = (1_000, 10_000, 100_000, 1_000_000)


def bf_leg(args, dev):
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300 import workloads
    from paper_2509_13230_gb300.sampler import BruteForceSampler, Sampler

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for n in BF_SIZES:
        rng = np.random.default_rng(1000 + n)
        x_np = np.minimum(workloads.pareto_scale(n) * rng.uniform(0.0, 1.0, n) ** (-1.0 / 1.1), 50.0)
        x = torch.from_numpy(x_np).to(dev)

        def timed(call, reps):
            call()
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                call()
            ev1.record(stream)
            ev1.synchronize()
            return ev0.elapsed_time(ev1) / reps

        mh = Sampler(nat.MH_UBCM, x, None, num_samples=1, seg_target=16)
        mh.run()
        mh_ms = timed(lambda: nat.check(mh.call(), "mh_sample_ubcm"), 10)
        bf = BruteForceSampler(nat.MH_UBCM, x, None, num_samples=1)
        bf.run()
        bf_ms = timed(lambda: nat.check(bf.call(), "mh_sample_bf"), 3 if n <= 100_000 else 1)
        pairs = n * (n - 1) / 2
        rows.append({"n": n, "edges_mh": int(mh.h_counts.sum()), "edges_bf": int(bf.h_counts.sum()),
                     "mh_ms": mh_ms, "bf_ms": bf_ms, "bf_pairs_per_s": pairs / (bf_ms / 1e3),
                     "bf_over_mh_time": bf_ms / mh_ms})
        del mh, bf
    return {"workload": "ubcm_pareto_bf_vs_mh", "model": "UBCM", "fitness": "x = min(c(N) u^(-1/1.1), 50)",
            "note": "one sample per call, whole call (prepare + walk + emit for the walk; both passes of the "
                    "brute force), CUDA events; the paper reports 10-100x on CPU (Sec. 3.1, Fig. 3A)",
            "sizes": rows}


# ---------------------------------------------------------------------------
# Output layouts of the headline workload: one-row CSR and the symmetric CSR
# (every edge in both endpoint rows), same samples and segment length.
# ---------------------------------------------------------------------------
def layouts_leg(args, dev, flush, T):
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300.sampler import Sampler

    net = workload()
    x = torch.from_numpy(net.x).to(dev)
    y = torch.from_numpy(net.y).to(dev)
    stream = torch.cuda.current_stream()
    out = {}
    for name, sym in (("csr", False), ("csr_symmetric", True)):
        s = Sampler(nat.MH_UECM, x, y, num_samples=SAMPLES_PER_STEP, seg_target=T, layout="csr", symmetric=sym)
        s.run()
        s.flags |= nat.MH_TIMING
        for _ in range(args.warmup):
            nat.check(s.call(), "mh_sample_weighted")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total_ms, edges, phase = 0.0, 0, np.zeros(3)
        steps = max(args.steps, 5)
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            nat.check(s.call(), "mh_sample_weighted")
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            info = nat.mh_last_call_info()
            phase += (info.prepare_ms, info.walk_ms, info.emit_ms)
            edges += int(s.h_counts.sum())
        per_edge = 16 if sym else 8  # index + weight per entry, one or two entries per edge
        out[name] = {"value": edges / (total_ms / 1e3), "unit": "edges/s", "ms_per_step": total_ms / steps,
                     "output": f"int64 offsets + int32 indices and weights, {per_edge} B/edge",
                     "phases_ms_per_step": dict(zip(("prepare", "walk", "scan_emit"), (phase / steps).tolist()))}
        del s
    return out


# ---------------------------------------------------------------------------
# Replicas: rank r draws samples [r S, (r + 1) S) of the same network (the
# counters are keyed by sample, so the union is the single-GPU ensemble);
# the job's time is the slowest rank's and its edges are all ranks' edges.
# ---------------------------------------------------------------------------
def rank_samples(rank: int, per_rank: int = SAMPLES_PER_STEP):
    """(first sample index, sample count) of a rank."""
    return rank * per_rank, per_rank


def reduce_over_ranks(total_ms: float, edges: float, world: int, device):
    """(max over ranks of the timed milliseconds, sum over ranks of the edges)."""
    if world <= 1:
        return total_ms, float(edges)
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, float(edges)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def single_call_leg(args, dev, flush, local_rank=0):
    """The weighted N = 20,000 workload, 10 samples per mh_sample_weighted call:
    device-timed rate, walk roofline, end to end with host buffers, the
    per-sample launch loop and the oracle baselines (one process, N = 1)."""
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300.sampler import Sampler

    rank, world = 0, 1

    def barrier():
        torch.cuda.synchronize()

    net = workload()
    x = torch.from_numpy(net.x).to(dev)
    y = torch.from_numpy(net.y).to(dev)
    first, _ = rank_samples(rank)
    # segment length and walk block shape from the autotuner (probe: the same
    # 10-sample call, device time); every rank tunes the same workload alike
    T, ctas, tuned = 0, 0, None
    if args.seg_target:
        T = args.seg_target
    elif not args.no_tune:
        from paper_2509_13230_gb300.autotune import tune_sampler
        tuned = tune_sampler(nat.MH_UECM, x, y, candidates_t=(8, 16, 32), candidates_ctas=(0,),
                             num_samples=SAMPLES_PER_STEP, reps=5)
        T, ctas = tuned.seg_target, tuned.walk_ctas_per_sm
    s = Sampler(nat.MH_UECM, x, y, num_samples=SAMPLES_PER_STEP, sample_begin=first, seg_target=T,
                walk_ctas_per_sm=ctas)
    s.run()                                     # sizes the output buffers
    s.flags |= nat.MH_TIMING
    stream = torch.cuda.current_stream()

    def timed_region():
        for _ in range(args.warmup):
            nat.check(s.call(), "mh_sample_weighted")
        barrier()
        total_ms, walk_ms, edges, launches = 0.0, [], 0, 0
        phases.clear()
        counters[:] = [0, 0]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            for _ in range(args.steps):
                flush.zero_()
                ev0.record(stream)
                nat.check(s.call(), "mh_sample_weighted")
                ev1.record(stream)
                ev1.synchronize()
                total_ms += ev0.elapsed_time(ev1)
                info = nat.mh_last_call_info()
                walk_ms.append(info.walk_ms)
                phases.append((info.prepare_ms, info.walk_ms, info.emit_ms, info.total_ms))
                launches += info.kernel_launches
                edges += int(s.h_counts.sum())
                counters[0] += int(s.h_stats[nat.MH_STAT_PROPOSALS])
                counters[1] += int(s.h_stats[nat.MH_STAT_BOUNDARY])
        barrier()
        return total_ms, walk_ms, edges, launches, clk.summary()

    phases = []
    counters = [0, 0]
    total_ms, walk_ms, edges, launches, clocks = timed_region()
    if rejected(clocks):
        total_ms, walk_ms, edges, launches, clocks = timed_region()
        clocks["remeasured"] = True
    max_ms, value = total_ms, edges / (total_ms / 1e3)
    proposals, boundary = counters

    # per-sample launch loop: the same samples drawn by one call each
    s1 = Sampler(nat.MH_UECM, x, y, num_samples=1, sample_begin=first, seg_target=T, walk_ctas_per_sm=ctas)
    s1.run()
    for _ in range(args.warmup):
        s1.call()
    torch.cuda.synchronize()
    loop_ms, loop_edges = 0.0, 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(1, args.steps // 2)):
        flush.zero_()
        ev0.record(stream)
        for k in range(SAMPLES_PER_STEP):
            nat.check(s1.call(sample_begin=first + k), "mh_sample_weighted")
            loop_edges += int(s1.h_counts.sum())
        ev1.record(stream)
        ev1.synchronize()
        loop_ms += ev0.elapsed_time(ev1)
    loop_value = loop_edges / (loop_ms / 1e3)

    # end to end through the public API with host buffers: x, y copied in from
    # pinned host memory before every call, the edges copied back after it
    hx = torch.from_numpy(net.x).pin_memory()
    hy = torch.from_numpy(net.y).pin_memory()
    e2e_flags = s.flags & ~nat.MH_TIMING
    cap = s.capacity
    d2h_step = None

    def host_out():
        return [torch.empty(cap, dtype=torch.int32).pin_memory() for _ in range(3)]

    def copy_back(smp, hb, m):
        for h, d in zip(hb, (smp.src, smp.dst, smp.w)):
            h[:m].copy_(d[:m], non_blocking=True)

    # serial: copy in, call, copy back, one step after another
    s.flags = e2e_flags
    hb = host_out()
    ser_ms, ser_edges = 0.0, 0
    for it in range(args.warmup + args.steps):
        flush.zero_()
        ev0.record(stream)
        x.copy_(hx, non_blocking=True)
        y.copy_(hy, non_blocking=True)
        nat.check(s.call(), "mh_sample_weighted")
        m = int(s.h_counts.sum())
        copy_back(s, hb, m)
        ev1.record(stream)
        ev1.synchronize()
        if it >= args.warmup:
            ser_ms += ev0.elapsed_time(ev1)
            ser_edges += m
            d2h_step = 12 * m + 8 * SAMPLES_PER_STEP
    ser_value = ser_edges / (ser_ms / 1e3)

    # pipelined: two samplers with their own inputs and outputs alternate; while
    # step t runs, the results of step t - 1 go back on one copy stream and
    # the inputs of step t + 1 come in on another.  Step t's window opens after
    # the L2 flush (no copy in flight: the flush waits for both copy streams)
    # and closes when its call and both copies are done, so each timed window
    # holds one copy-in, one call and one equal-sized copy-back.
    xb, yb = torch.empty_like(x), torch.empty_like(y)
    sb = Sampler(nat.MH_UECM, xb, yb, num_samples=SAMPLES_PER_STEP, sample_begin=first, seg_target=T,
                 walk_ctas_per_sm=ctas, capacity=cap)
    sb.flags = e2e_flags
    pairs = [(s, x, y, hb), (sb, xb, yb, host_out())]
    back = torch.cuda.Stream(device=dev)
    ahead = torch.cuda.Stream(device=dev)
    n_it = args.warmup + args.steps
    back_done = [None] * n_it
    in_ready = [None] * (n_it + 1)
    pipe_ms, pipe_edges, m_prev = 0.0, 0, 0
    parts = {"call": 0.0, "copy_back": 0.0, "copy_in": 0.0}
    x.copy_(hx, non_blocking=True)  # inputs of step 0
    y.copy_(hy, non_blocking=True)
    for it in range(n_it):
        smp = pairs[it & 1][0]
        if it >= 2:
            stream.wait_event(back_done[it - 2])
        if in_ready[it] is not None:
            stream.wait_event(in_ready[it])
        flush.zero_()
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        if it >= 1:
            prev = pairs[(it - 1) & 1]
            back.wait_event(start)
            with torch.cuda.stream(back):
                copy_back(prev[0], prev[3], m_prev)
            back_done[it - 1] = torch.cuda.Event(enable_timing=True)
            back_done[it - 1].record(back)
        # the next step's sampler finished its last call (step t - 1) before this one began
        nxt = pairs[(it + 1) & 1]
        ahead.wait_event(start)
        with torch.cuda.stream(ahead):
            nxt[1].copy_(hx, non_blocking=True)
            nxt[2].copy_(hy, non_blocking=True)
        in_ready[it + 1] = torch.cuda.Event(enable_timing=True)
        in_ready[it + 1].record(ahead)
        nat.check(smp.call(), "mh_sample_weighted")
        m_prev = int(smp.h_counts.sum())
        called = torch.cuda.Event(enable_timing=True)
        called.record(stream)
        called.synchronize()
        in_ready[it + 1].synchronize()
        if it >= 1:
            back_done[it - 1].synchronize()
        if it >= args.warmup:
            t_call = start.elapsed_time(called)
            t_in = start.elapsed_time(in_ready[it + 1])
            t_back = start.elapsed_time(back_done[it - 1]) if it >= 1 else 0.0
            pipe_ms += max(t_call, t_in, t_back)
            pipe_edges += m_prev
            parts["call"] += t_call
            parts["copy_back"] += t_back
            parts["copy_in"] += t_in
    copy_back(*[pairs[(n_it - 1) & 1][q] for q in (0, 3)], m_prev)  # last results, untimed
    torch.cuda.synchronize()
    s.flags = e2e_flags | nat.MH_TIMING
    e2e_value = pipe_edges / (pipe_ms / 1e3)
    e2e_parts = parts
    hbm_gbs, peak_kind = peaks()
    walk_avg_ms = float(np.mean(walk_ms))
    edges_per_step = edges / args.steps
    achieved = BYTES_PER_EDGE * edges_per_step / (walk_avg_ms / 1e3) / 1e9
    traffic = walk_traffic(T or 32)
    # CPU oracle on a bounded sample of the same workload
    rate, nsamp, secs = oracle_rate(net, 10.0)
    cpu = {"value": rate, "unit": "edges/s", "cores": 1, "kind": "oracle",
           "sample": f"{nsamp} whole samples of {WORKLOAD} (N = {net.n}), serial FP64 walk, "
                     f"{secs:.1f} s on one host core"}
    cpu_all = cpu_bf = None
    if not args.no_ensemble:
        rate_a, nsamp_a, busy_a, wall_a, cores_a = oracle_rate_all_cores(net, 8.0)
        cpu_all = {"value": rate_a, "unit": "edges/s", "cores": cores_a, "kind": "oracle",
                   "sample": f"{nsamp_a} whole samples of {WORKLOAD}, one spawned process per host core, "
                             f"{busy_a:.1f} s busy per process ({wall_a:.1f} s wall with start-up)"}
        bf_s, evals = oracle_bf_time(net)
        cpu_bf = {"seconds_per_sample": bf_s, "pairs": evals, "pairs_per_s": evals / bf_s,
                  "edges_per_s": (edges / args.steps / SAMPLES_PER_STEP) / bf_s,
                  "mh_over_bf_speedup_cpu": bf_s / (secs / nsamp), "kind": "oracle brute force", "cores": 1}
    return {
        "workload": WORKLOAD, "value": value, "unit": "edges/s", "ms_per_step": max_ms / args.steps,
        "n": net.n, "samples_per_step": SAMPLES_PER_STEP, "seg_target": T or 32, "walk_ctas_per_sm": ctas,
        "autotune": None if tuned is None else tuned.table,
        "output": "coo int32 + w int32 (12 B/edge)", "l2": "flushed (512 MiB write) before every step",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                     "frac": achieved / hbm_gbs, "traffic": traffic, "kernel": "walk_kernel",
                     "peak_kind": peak_kind, "walk_ms_per_launch": walk_avg_ms},
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "cpu_brute_force": cpu_bf,
        "e2e": {"value": e2e_value, "unit": "edges/s", "h2d_bytes_per_step": 16 * net.n,
                "d2h_bytes_per_step": d2h_step,
                "copies": "two samplers alternate (double-buffered inputs and outputs): during step t the "
                          "edges of step t - 1 go device-to-host and x, y of step t + 1 host-to-device on two "
                          "copy streams; L2 flushed between steps with no copy in flight",
                "window_ms": {k: v / args.steps for k, v in e2e_parts.items()},
                "serial": {"value": ser_value, "unit": "edges/s",
                           "copies": "copy in, call, copy back, one step after another"}},
        "gpu_launches": launches,
        "phases_ms_per_step": dict(zip(("prepare", "walk", "scan_emit", "call"),
                                       (float(v) for v in np.mean(np.array(phases), axis=0)))),
        "per_sample_loop": {"value": loop_value, "unit": "edges/s", "batched_over_loop": value / loop_value},
        "boundary_draws": boundary, "proposals": proposals,
        "clocks": clocks,
    }


# ---------------------------------------------------------------------------
# Headline: the batched ensemble of 128 networks (N log-uniform in
# [10^3, 10^6], half UBCM and half UECM, capped Pareto fitness with mean
# expected degree about 20), 64 samples each, CSR output, drawn by
# mh_batch_prepare + mh_sample_batched waves; beside it the same samples
# drawn by one mh_sample_* call per (network, sample).  Rank r draws samples
# [64 r, 64 (r + 1)) of every network (weak scaling, no data-path collective).
# ---------------------------------------------------------------------------
ENSEMBLE_WORKLOAD = "ensemble_128_x64"
ENSEMBLE_PROFILE = os.path.join(ROOT, "profiles", "walk_kernel_batched_ensemble.json")
LOOP_REPEATS = 3


def ensemble_profile():
    """Per-proposal figures of the batched walks from the ncu capture in
    profiles/ (thread instructions, DRAM bytes), while the walk sources are
    unchanged since it; else None."""
    if os.path.exists(ENSEMBLE_PROFILE):
        prof = json.load(open(ENSEMBLE_PROFILE))
        if prof.get("sources_sha") == sources_hash():
            return prof
    return None


def ensemble_networks(args, dev):
    """The 128 networks (or an evenly spaced subset) with x and y of all
    networks in two concatenated device arrays (one copy each end to end)."""
    import torch

    from paper_2509_13230_gb300 import workloads

    nets_np = workloads.ensemble_128()
    keep = max(1, min(args.ensemble_networks, len(nets_np)))
    sel = np.linspace(0, len(nets_np) - 1, keep).round().astype(int)
    nets_np = [(int(t), nets_np[t]) for t in sel]
    x_host = np.concatenate([nw.x for _, nw in nets_np])
    y_host = np.concatenate([nw.y for _, nw in nets_np if nw.y is not None] or [np.zeros(0)])
    x_all = torch.from_numpy(x_host).to(dev)
    y_all = torch.from_numpy(y_host).to(dev)
    nets, ox, oy = [], 0, 0
    for t, nw in nets_np:
        xv = x_all[ox:ox + nw.n]
        ox += nw.n
        yv = None
        if nw.y is not None:
            yv = y_all[oy:oy + nw.n]
            oy += nw.n
        nets.append((nw.model, xv, yv, t))
    return nets_np, nets, x_host, y_host, x_all, y_all


def oracle_ensemble_rate(nets_np, T, seconds):
    """The oracle on whole samples of the smallest networks, about `seconds` of one core."""
    import oracle
    oracle.load()
    n = np.array([nw.n for _, nw in nets_np])
    edges, secs, pairs = 0, 0.0, 0
    for k in np.argsort(n, kind="stable"):
        if secs > seconds:
            break
        t, nw = nets_np[k]
        t0 = time.perf_counter()
        _, _, _, c, _ = oracle.mh_sample(nw.model, nw.x, nw.y, network_id=t, num_samples=1, seg_target=T)
        secs += time.perf_counter() - t0
        edges += int(c.sum())
        pairs += 1
    return edges / secs, pairs, secs


def ensemble_headline(args, dev, flush, rank, world, barrier):
    import torch

    from paper_2509_13230_gb300 import _native as nat
    from paper_2509_13230_gb300.ensemble import Ensemble
    from paper_2509_13230_gb300.sampler import Sampler

    nets_np, nets, x_host, y_host, x_all, y_all = ensemble_networks(args, dev)
    n = np.array([nw.n for _, nw in nets_np], dtype=np.int64)
    uecm = np.array([nw.model == nat.MH_UECM for _, nw in nets_np])
    samples = args.ensemble_samples
    first = rank * samples
    T, ctas, tuned = 0, 0, None
    if args.ensemble_seg_target:
        T = args.ensemble_seg_target
    elif not args.no_tune:
        from paper_2509_13230_gb300.autotune import tune_ensemble
        tuned = tune_ensemble(nets, candidates_t=(8, 16, 32), candidates_ctas=(0, 2), num_samples=2, reps=2)
        T, ctas = tuned.seg_target, tuned.walk_ctas_per_sm
    ens = Ensemble(nets, num_samples=samples, sample_begin=first, layout="csr", capacity=args.ensemble_capacity,
                   timing=True, seg_target=T, walk_ctas_per_sm=ctas, max_wave_items=args.ensemble_wave_items)
    stream = torch.cuda.current_stream()
    acc = {}

    def on_wave(res):
        info = nat.mh_last_call_info()
        acc["walk"] += info.walk_ms
        acc["emit"] += info.emit_ms
        acc["launches"] += info.kernel_launches
        acc["waves"] += 1

    def one_step():
        ens.prepare()  # sort + bound prep + segment tables of every network are part of a step
        info = nat.mh_last_call_info()
        acc["prepare"] += info.prepare_ms
        acc["launches"] += info.kernel_launches
        counts, stats = ens.sample(on_wave=on_wave)
        return counts, stats

    def reset():
        acc.update(walk=0.0, emit=0.0, prepare=0.0, launches=0, waves=0)

    def out_bytes(counts):
        per_net = counts.reshape(len(nets), samples).sum(axis=1)
        return int((4 * per_net + 4 * per_net * uecm + 8 * (n + 1) * samples).sum())

    def timed(steps, e2e=False):
        reset()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot_ms, edges, nbytes, props, bnd, fb = 0.0, 0, 0, 0, 0, 0
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            if e2e:  # this step's inputs from pinned host memory
                x_all.copy_(hx, non_blocking=True)
                y_all.copy_(hy, non_blocking=True)
            counts, stats = one_step()  # per-pair counts come back to the host in every wave
            ev1.record(stream)
            ev1.synchronize()
            tot_ms += ev0.elapsed_time(ev1)
            edges += int(counts.sum())
            nbytes += out_bytes(counts)
            props += int(stats[nat.MH_STAT_PROPOSALS])
            bnd += int(stats[nat.MH_STAT_BOUNDARY])
            fb += int(stats[nat.MH_STAT_FALLBACKS])
        return dict(ms=tot_ms, edges=edges, bytes=nbytes, proposals=props, boundary=bnd, fallbacks=fb,
                    **{k: v for k, v in acc.items()})

    reset()
    for _ in range(args.warmup):
        one_step()
    barrier()
    with ClockSampler(dev.index or 0) as clk:
        r = timed(args.steps)
    barrier()
    clocks = clk.summary()
    if rejected(clocks):
        with ClockSampler(dev.index or 0) as clk:
            r = timed(args.steps)
        barrier()
        clocks = clk.summary()
        clocks["remeasured"] = True
    max_ms, all_edges = reduce_over_ranks(r["ms"], r["edges"], world, dev)
    value = all_edges / (max_ms / 1e3)

    # end to end: the same steps with x and y of all networks copied in from
    # pinned host memory first (one copy each), counts read back per wave
    hx = torch.from_numpy(x_host).pin_memory()
    hy = torch.from_numpy(y_host).pin_memory()
    e2e_steps = max(3, min(args.steps, 8))
    re = timed(e2e_steps, e2e=True)
    barrier()
    e_max_ms, e_edges = reduce_over_ranks(re["ms"], re["edges"], world, dev)
    e2e_value = e_edges / (e_max_ms / 1e3)

    # per-sample launch loop: one mh_sample_* call per (network, sample),
    # the first loop_samples samples of each network, repeated
    loop = None
    loop_samples = args.ensemble_loop_samples
    if loop_samples > 0:
        samplers = []
        for (m, x, y, nid) in nets:
            s1 = Sampler(m, x, y, num_samples=1, network_id=nid, sample_begin=first, layout="csr", seg_target=T,
                         walk_ctas_per_sm=ctas)
            s1.run()
            samplers.append(s1)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = []
        for _ in range(LOOP_REPEATS):
            flush.zero_()
            l_edges = 0
            ev0.record(stream)
            for s1 in samplers:
                for k in range(loop_samples):
                    nat.check(s1.call(sample_begin=first + k), "mh_sample")
                    l_edges += int(s1.h_counts.sum())
            ev1.record(stream)
            ev1.synchronize()
            reps.append(l_edges / (ev0.elapsed_time(ev1) / 1e3))
        del samplers
        ratios = sorted(value / world / v for v in reps)
        loop = {"value": statistics.median(reps), "unit": "edges/s", "repeats": reps,
                "calls_per_repeat": len(nets) * loop_samples, "samples_per_network": loop_samples,
                "batched_over_loop": statistics.median(ratios), "batched_over_loop_min": ratios[0],
                "batched_over_loop_median": statistics.median(ratios),
                "note": "batched: the headline's per-GPU rate; loop: one call per (network, sample), "
                        "each call preparing its network and reading its counts back"}
    del ens
    torch.cuda.empty_cache()

    hbm_gbs, peak_kind = peaks()
    steps = args.steps
    walk_s = r["walk"] / steps / 1e3
    prof = ensemble_profile()
    achieved = r["bytes"] / steps / walk_s / 1e9 if walk_s > 0 else None
    issue = None
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sms * 128 * sm_mhz * 1e6
    if prof is not None and walk_s > 0:
        ipp = prof["thread_inst_per_proposal"]
        issue_ach = ipp * r["proposals"] / steps / walk_s
        issue = {"bound": "issue", "achieved": issue_ach / 1e12, "peak": issue_peak / 1e12,
                 "unit": "T thread-instructions/s", "frac": issue_ach / issue_peak,
                 "thread_inst_per_proposal": ipp,
                 "basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock of the timed region); "
                          "instructions per proposal from the ncu capture in profiles/"}
    else:
        issue = {"bound": "issue", "achieved": None, "peak": issue_peak / 1e12, "unit": "T thread-instructions/s",
                 "frac": None, "note": "no ncu capture of the current walk sources"}
    traffic = None if prof is None else prof["dram_bytes_per_proposal"] * r["proposals"] / steps
    cpu = None
    if rank == 0 and world == 1:
        rate, pairs, secs = oracle_ensemble_rate(nets_np, T or 32, 10.0)
        cpu = {"value": rate, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"one sample of each of the {pairs} smallest networks of the ensemble, serial FP64 "
                         f"walk, {secs:.1f} s on one host core"}
    return {
        "value": value, "max_ms": max_ms, "edges_per_step": r["edges"] / steps,
        "config": {"workload": ENSEMBLE_WORKLOAD, "networks": len(nets), "nodes": int(n.sum()),
                   "samples_per_network": samples, "samples_per_step": samples * len(nets) * world,
                   "fitness": "x = min(c(N) u^(-1/1.1), 50), u ~ U(0, 1), mean expected degree about 20; "
                              "y ~ U(0.3, 0.9) for the 64 UECM networks",
                   "seg_target": T or 32, "walk_ctas_per_sm": ctas, "autotune": None if tuned is None else tuned.table,
                   "output": "CSR: int64 offsets, int32 indices (+ int32 weights for the UECM half)",
                   "waves_per_step": r["waves"] / steps, "wave_edges": args.ensemble_capacity,
                   "wave_items": args.ensemble_wave_items,
                   "l2": "inputs and outputs far larger than L2; a 512 MiB write flushes it before every step",
                   "parallelism": f"replicas x{world} (rank r draws samples [64 r, 64 r + 64) of every network)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                     "frac": achieved / hbm_gbs if achieved else None, "traffic": traffic,
                     "kernel": "walk_kernel (batched; the UBCM and UECM launches of a wave run concurrently)",
                     "peak_kind": peak_kind, "walk_ms_per_step": r["walk"] / steps,
                     "basis": "CSR output bytes of the step (4 B index, 4 B UECM weight, 8 B per offset) / walk "
                              "time of the step (CUDA events around each wave's two concurrent walk launches); "
                              "traffic: DRAM bytes per step scaled from the capture's bytes per proposal",
                     "issue": issue},
        "phases_ms_per_step": {"prepare": r["prepare"] / steps, "walk": r["walk"] / steps,
                               "scan_emit": r["emit"] / steps},
        "gpu_launches": r["launches"],
        "proposals_per_step": r["proposals"] / steps,
        "boundary_draws": {"count": r["boundary"], "draws": r["proposals"],
                           "rate": r["boundary"] / max(1, r["proposals"]),
                           "bound": 1e-8, "ok": r["boundary"] / max(1, r["proposals"]) < 1e-8},
        "fp64_fallbacks": r["fallbacks"],
        "e2e": {"value": e2e_value, "unit": "edges/s", "h2d_bytes_per_step": int(x_host.nbytes + y_host.nbytes),
                "d2h_bytes_per_step": 8 * len(nets) * samples,
                "copies": "every step copies x and y of all networks from pinned host memory (one copy each) "
                          "before the batched prepare and waves; the per-pair edge counts come back to the host "
                          "with every wave; the sampled graphs stay in the device's reused wave buffers",
                "steps": e2e_steps, "ms_per_step": re["ms"] / e2e_steps},
        "per_sample_loop": loop,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    head = ensemble_headline(args, dev, flush, rank, world, barrier)
    subs = {}
    if world == 1 and not args.headline_only:
        subs["uecm_n20k_x10"] = single_call_leg(args, dev, flush)
        if not args.no_ensemble:
            subs["ensemble_lognormal"] = ensemble_leg(args, dev, flush, fitness="lognormal", samples=8,
                                                      capacity=1 << 31, seg_target=head["config"]["seg_target"],
                                                      loop_samples=1)
            subs["pairwise"] = pairwise_leg(args, dev, head["clocks"].get("sm_mhz"))
            subs["fit_then_sample"] = fit_leg(args, dev)
            subs["bipartite"] = bipartite_leg(args, dev, flush)
            subs["configs"] = configs_leg(args, dev, flush)
            subs["brute_force"] = bf_leg(args, dev)
        subs["layouts"] = layouts_leg(args, dev, flush, subs["uecm_n20k_x10"]["seg_target"])
        fitted, cpu_bf = subs.get("fit_then_sample"), subs["uecm_n20k_x10"].get("cpu_brute_force")
        if fitted is not None and cpu_bf is not None:
            # config 5 brute force: N (N - 1) / 2 pairs per sample at the UECM pair
            # rate measured on the weighted N = 20,000 network in this run
            pairs5 = FIT_N * (FIT_N - 1) / 2
            fitted["cpu_brute_force"] = {
                "pairs": pairs5, "extrapolated_seconds_per_sample": pairs5 / cpu_bf["pairs_per_s"],
                "note": "not run: extrapolated at the UECM brute-force pair rate of the N = 20,000 network"}
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    loop = head["per_sample_loop"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["max_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": head["config"],
        "roofline": head["roofline"],
        "cpu_baseline": head["cpu_baseline"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "per_sample_loop": loop,
        "batched_over_loop": None if loop is None else loop["batched_over_loop_median"],
        "batched_over_loop_min": None if loop is None else loop["batched_over_loop_min"],
        "edges_per_step": head["edges_per_step"],
        "phases_ms_per_step": head["phases_ms_per_step"],
        "proposals_per_step": head["proposals_per_step"],
        "boundary_draws": head["boundary_draws"],
        "fp64_fallbacks": head["fp64_fallbacks"],
        **subs,
        "clocks": head["clocks"],
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the long sub-legs (lognormal ensemble, pairwise, fit, bipartite, configs)")
    ap.add_argument("--headline-only", action="store_true", help="only the batched-ensemble headline")
    ap.add_argument("--leg", choices=["all", "ensemble", "pairwise", "fit", "bipartite", "layouts", "configs", "kernels",
                                      "bf"],
                    default="all",
                    help="run only that leg and print its object; kernels: each profiled kernel once, "
                         "untimed (walk at T = 8, 16, 32, then pairwise forward, backward, Jacobian "
                         "diagonal), for ncu")
    ap.add_argument("--no-tune", action="store_true", help="ensemble leg: default T and block shape, no autotuner")
    ap.add_argument("--seg-target", type=int, default=0,
                    help="headline call: use this seg_target instead of tuning (profiling runs)")
    ap.add_argument("--ensemble-seg-target", type=int, default=0,
                    help="ensemble leg: use this seg_target instead of tuning (profiling runs)")
    ap.add_argument("--ensemble-networks", type=int, default=128,
                    help="networks of the ensemble leg (evenly spaced subset of the 128)")
    ap.add_argument("--ensemble-samples", type=int, default=ENSEMBLE_SAMPLES, help="samples per network")
    ap.add_argument("--ensemble-capacity", type=int, default=1 << 31,
                    help="edges per wave (output buffers reused by every wave)")
    ap.add_argument("--ensemble-wave-items", type=int, default=1 << 29,
                    help="work items (sample, segment) per wave")
    ap.add_argument("--ensemble-loop-samples", type=int, default=4,
                    help="samples per network of the ensemble's per-sample loop (0 skips the loop)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.leg == "ensemble" and args.impl != "reference":
        import torch
        torch.cuda.set_device(local_rank)
        dev = torch.device("cuda", local_rank)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps({"ensemble": ensemble_leg(args, dev, flush)}), flush=True)
    elif args.leg == "fit":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"fit_then_sample": fit_leg(args, torch.device("cuda", local_rank))}), flush=True)
    elif args.leg == "configs":
        import torch
        torch.cuda.set_device(local_rank)
        dev = torch.device("cuda", local_rank)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps({"configs": configs_leg(args, dev, flush)}), flush=True)
    elif args.leg == "layouts":
        import torch
        torch.cuda.set_device(local_rank)
        dev = torch.device("cuda", local_rank)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps({"layouts": layouts_leg(args, dev, flush, args.ensemble_seg_target or 8)}), flush=True)
    elif args.leg == "bipartite":
        import torch
        torch.cuda.set_device(local_rank)
        dev = torch.device("cuda", local_rank)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps({"bipartite": bipartite_leg(args, dev, flush)}), flush=True)
    elif args.leg == "kernels":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"kernels_once": kernels_once(torch.device("cuda", local_rank))}), flush=True)
    elif args.leg == "bf":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"brute_force": bf_leg(args, torch.device("cuda", local_rank))}), flush=True)
    elif args.leg == "pairwise":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"pairwise": pairwise_leg(args, torch.device("cuda", local_rank), None)}), flush=True)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
