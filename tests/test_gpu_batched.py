"""Batched ensembles (mh_batch_prepare / mh_sample_batched) against the CPU
oracle (GPU).

Every (network, sample) pair of a wave must equal the serial oracle's
sample of that network with the pair's network id and sample index, bit for
bit, in COO and CSR; the allowance is the one of the single-network tests (a
draw the oracle flags as lying on an integer boundary of ln U / ln v)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity import assert_traced, check_sample, oracle_sample, same_sample
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import workloads
from paper_2509_13230_gb300.ensemble import Ensemble
from paper_2509_13230_gb300.sampler import Sampler

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM
SEED = 0x0123456789ABCDEF


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def mixed_networks(seed, sizes=(1, 2, 57, 1500, 4000, 9000, 300), models=None):
    rng = np.random.default_rng(seed)
    models = models or [UBCM, UECM, UECM, UBCM, UECM, UBCM, UECM]
    nets = []
    for t, (n, m) in enumerate(zip(sizes, models)):
        x = np.exp(rng.normal(-4.0, 1.2, n))
        if n > 100:
            x[rng.choice(n, 3, replace=False)] = rng.uniform(5, 30, 3)
        y = rng.uniform(0.2, 0.95, n) if m == UECM else None
        nets.append((m, x, y, 100 + 7 * t))
    return nets


def to_device(nets):
    return [(m, dev(x), None if y is None else dev(y), nid) for (m, x, y, nid) in nets]


def expected_csr(src, dst, n):
    order = np.argsort(src, kind="stable")
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(np.bincount(src, minlength=n))
    return off, dst[order], order


class Checker:
    """on_wave callback: compares every pair with the oracle."""

    def __init__(self, nets, *, seed, sample_begin, seg_target=32, flags=0, layout="both", only=None):
        self.nets, self.seed, self.sample_begin = nets, seed, sample_begin
        self.seg_target, self.flags, self.layout = seg_target, flags, layout
        self.only = only
        self.pairs = 0
        self.boundary = 0
        self.waves = []
        self.any_uecm = any(m == UECM for (m, _, _, _) in nets)

    def __call__(self, res):
        self.waves.append(set(int(t) for t in res.networks))
        for k in range(res.pair_count):
            t, s = int(res.networks[k]), int(res.samples[k])
            if self.only is not None and (t, s) not in self.only:
                continue
            m, x, y, nid = self.nets[t]
            ref, stats, log = oracle_sample(m, x, y, seed=self.seed, network_id=nid,
                                            sample_begin=self.sample_begin + s, num_samples=1,
                                            seg_target=self.seg_target, flags=self.flags)
            src, dst, w, counts = ref
            self.pairs += 1
            if self.layout in ("coo", "both"):
                gs, gd, gw = (None if a is None else a.cpu().numpy() for a in res.coo(k))
                got = (gs, gd, gw if m == UECM else None, np.array([len(gs)], np.int64))
                if not same_sample(got, ref):
                    # only segments holding an oracle boundary draw may differ
                    assert_traced(m, x, y, got, ref, log, seg_target=self.seg_target, flags=self.flags,
                                  sample_begin=self.sample_begin + s)
                    self.boundary += 1
                    continue
                if m == UBCM and gw is not None:
                    assert (gw == 1).all()
                assert int(res.counts[k]) == int(counts[0])
            if self.layout in ("csr", "both"):
                off, idx, wts = res.csr(k, len(x))
                e_off, e_idx, order = expected_csr(src, dst, len(x))
                assert np.array_equal(off.cpu().numpy(), e_off), (t, s)
                assert np.array_equal(idx.cpu().numpy(), e_idx), (t, s)
                if m == UECM:
                    assert np.array_equal(wts.cpu().numpy(), w[order]), (t, s)


@pytest.mark.parametrize("layout", ["both", "csr"])
def test_mixed_batch_matches_oracle(layout):
    nets = mixed_networks(1)
    ens = Ensemble(to_device(nets), num_samples=3, seed=SEED, sample_begin=5, layout=layout,
                   max_wave_items=25_000, capacity=1 << 20)
    segs = ens.prepare()
    assert segs[0] == 0 and segs[1] == 1  # n = 1 has no candidates; n = 2 one segment
    chk = Checker(nets, seed=SEED, sample_begin=5, layout=layout)
    counts, stats = ens.sample(on_wave=chk)
    assert chk.pairs == len(nets) * 3
    # the item limit split the pairs into waves, and some network's samples across two of them
    assert ens.waves_run == len(chk.waves) >= 2
    assert any(len(a & b) for a, b in zip(chk.waves, chk.waves[1:]))
    assert int(stats[nat.MH_STAT_EDGES]) == int(counts.sum())


def test_waves_split_a_network_and_retry_on_capacity():
    nets = mixed_networks(2, sizes=(3000, 2500, 4000), models=[UECM, UBCM, UECM])
    ens = Ensemble(to_device(nets), num_samples=5, seed=7, layout="both", capacity=30_000)
    ens.prepare()
    ens.est[:] = 1.0  # optimistic estimates: the first waves overflow and are re-planned from exact counts
    chk = Checker(nets, seed=7, sample_begin=0)
    counts, _ = ens.sample(on_wave=chk)
    assert chk.pairs == 15
    assert counts.max() < 30_000 and counts.sum() > 30_000


@pytest.mark.parametrize("variant", ["paper_bound", "init_prev", "fp64_only", "T2"])
def test_batch_equals_single_network_calls(variant):
    nets = mixed_networks(3, sizes=(2600, 1800), models=[UECM, UBCM])
    kw = dict(paper_bound=dict(bound="paper"), init_prev=dict(init="prev"), fp64_only=dict(fp64_only=True),
              T2=dict(seg_target=2))[variant]
    ens = Ensemble(to_device(nets), num_samples=2, seed=99, sample_begin=3, layout="coo", **kw)
    got = {}

    def keep(res):
        for k in range(res.pair_count):
            got[(int(res.networks[k]), int(res.samples[k]))] = [None if a is None else a.clone() for a in res.coo(k)]

    ens.sample(on_wave=keep)
    for t, (m, x, y, nid) in enumerate(nets):
        for s in range(2):
            one = Sampler(m, dev(x), None if y is None else dev(y), num_samples=1, seed=99, network_id=nid,
                          sample_begin=3 + s, **kw).run()
            gs, gd, gw = got[(t, s)]
            assert torch.equal(gs, one.src) and torch.equal(gd, one.dst)
            if m == UECM:
                assert torch.equal(gw, one.w)


def test_workspace_prepared_for_other_networks_is_rejected():
    nets = to_device(mixed_networks(4, sizes=(500, 700), models=[UBCM, UECM]))
    ens = Ensemble(nets, num_samples=2, layout="coo")
    ens.prepare()
    other = [(m, x.clone(), None if y is None else y.clone(), nid) for (m, x, y, nid) in nets]
    d = nat.network_descs([(m, nid, x.shape[0], x.data_ptr(), None if y is None else y.data_ptr())
                           for (m, x, y, nid) in other])
    counts = np.zeros(4, np.int64)
    rc = nat.mh_sample_batched(d, 2, ens.params, ens.max_wave_items, ctypes.c_void_p(ens.ws.data_ptr()),
                               ens.ws.numel(), 0, 4, ctypes.c_void_p(ens.src.data_ptr()),
                               ctypes.c_void_p(ens.dst.data_ptr()), ctypes.c_void_p(ens.w.data_ptr()), None, None,
                               None, ens.capacity, counts.ctypes.data_as(ctypes.c_void_p), None, None)
    assert rc == nat.MH_ERR_ARG
    assert "prepare" in nat.last_error_detail()


def test_wave_over_its_item_limit_is_rejected():
    nets = to_device(mixed_networks(5, sizes=(3000,), models=[UBCM]))
    ens = Ensemble(nets, num_samples=8, layout="coo", max_wave_items=5000)
    segs = ens.prepare()
    assert segs[0] <= 5000
    k = 5000 // int(segs[0]) + 1  # one pair more than the wave buffers hold
    rc, _ = ens.run_wave(0, k)
    assert rc == nat.MH_ERR_WORKSPACE
    rc, res = ens.run_wave(0, k - 1)
    assert rc == nat.MH_OK and res.total > 0


def test_domain_error_names_the_network():
    nets = mixed_networks(6, sizes=(400, 500), models=[UBCM, UECM])
    nets[1][2][17] = 1.0  # y = 1 is outside [0, 1)
    ens = Ensemble(to_device(nets), num_samples=1, layout="coo")
    with pytest.raises(nat.MhError) as e:
        ens.prepare()
    assert e.value.code == nat.MH_ERR_DOMAIN and "network 1" in str(e.value)


def test_batched_call_info_reports_both_walks():
    nets = to_device(mixed_networks(7, sizes=(3000, 3000), models=[UBCM, UECM]))
    ens = Ensemble(nets, num_samples=2, layout="csr", timing=True)
    ens.sample()
    info = nat.mh_last_call_info()
    assert info.walk_launches == 2
    assert info.walk_ms > 0 and info.total_ms >= info.walk_ms
    assert 6 <= info.kernel_launches <= 16


def test_ensemble_128_full_size_sampled_pairs():
    """The 128-network ensemble at full size (N log-uniform in [10^3, 10^6],
    64 samples) in the bench's launch configuration; sampled pairs of small,
    middle and the largest sizes against the oracle, every pair's count
    against the walk's edge counter."""
    nets_np = workloads.ensemble_128()
    nets = [(nw.model, nw.x, nw.y, t) for t, nw in enumerate(nets_np)]
    sizes = np.array([nw.n for nw in nets_np])
    pick = {(int(np.argmin(sizes)), 0), (int(np.argmin(sizes)), 63)}
    for model in (UBCM, UECM):
        idx = [t for t in range(len(nets_np)) if nets_np[t].model == model]
        order = sorted(idx, key=lambda t: sizes[t])
        pick |= {(order[len(order) // 2], 31), (order[-1] if model == UBCM else order[len(order) * 3 // 4], 7)}
    ens = Ensemble(to_device(nets), num_samples=64, layout="csr", capacity=1 << 30, max_wave_items=1 << 28)
    chk = Checker(nets, seed=0, sample_begin=0, layout="csr", only=pick)
    counts, stats = ens.sample(on_wave=chk)
    assert chk.pairs == len(pick)
    assert int(stats[nat.MH_STAT_EDGES]) == int(counts.sum())
    mean_deg = np.array([2 * counts[t * 64:(t + 1) * 64].mean() / sizes[t] for t in range(len(nets_np))])
    assert np.all(mean_deg[:64] > 10) and np.all(mean_deg[:64] < 40)  # UBCM: about 20 by construction


def test_autotuner_choice_is_a_candidate_and_samples_exactly():
    from paper_2509_13230_gb300.autotune import tune_ensemble, tune_sampler
    nets = mixed_networks(8, sizes=(6000, 3000), models=[UBCM, UECM])
    m, x, y, nid = nets[0]
    res = tune_sampler(m, dev(x), None, candidates_t=(8, 32, 128), candidates_ctas=(0, 1), num_samples=2, reps=2)
    assert res.seg_target in (8, 32, 128) and res.walk_ctas_per_sm in (0, 1)
    assert len(res.table) == 6 and all(r["edges_per_ms"] > 0 for r in res.table)
    # block shape changes no bit; T changes the sample, which stays exact
    for T in (8, 128):
        a = Sampler(m, dev(x), num_samples=2, seg_target=T, walk_ctas_per_sm=1).run()
        b = Sampler(m, dev(x), num_samples=2, seg_target=T).run()
        assert torch.equal(a.src, b.src) and torch.equal(a.dst, b.dst)
    chosen = Sampler(m, dev(x), num_samples=1, seg_target=res.seg_target,
                     walk_ctas_per_sm=res.walk_ctas_per_sm).run()
    check_sample((chosen.src.cpu().numpy(), chosen.dst.cpu().numpy(), None, chosen.counts), m, x, None,
                 num_samples=1, seg_target=res.seg_target)
    ens_res = tune_ensemble(to_device(nets), candidates_t=(16, 32), candidates_ctas=(0, 2), num_samples=2, reps=1)
    assert ens_res.seg_target in (16, 32) and len(ens_res.table) == 4


def test_segment_table_caps_grow_per_network():
    # T = 2 on a dense network needs far more rows than the default 4 n + 1024
    rng = np.random.default_rng(9)
    dense = (UBCM, np.exp(rng.normal(0.5, 0.3, 300)), None, 1)
    sparse = (UECM, np.exp(rng.normal(-4.0, 1.2, 5000)), rng.uniform(0.3, 0.9, 5000), 2)
    nets = [dense, sparse]
    ens = Ensemble(to_device(nets), num_samples=2, seed=3, seg_target=2, layout="both")
    segs = ens.prepare()
    assert segs[0] > 4 * 300 + 1024 and ens.descs[0].max_segments >= segs[0]
    assert ens.descs[1].max_segments == 0  # the sparse network kept the default cap
    chk = Checker(nets, seed=3, sample_begin=0, seg_target=2)
    ens.sample(on_wave=chk)
    assert chk.pairs == 4
