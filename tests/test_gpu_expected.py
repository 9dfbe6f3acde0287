"""Expected degrees / strengths, their autograd Function and fitting (GPU).

Targets are produced by the CPU oracle from known parameters; fitted
parameters are checked by the oracle again, so no expected value comes from
the CUDA path."""
import numpy as np
import pytest
import torch

import oracle
from parity import check_sample
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300.expected import ExpectedDegrees, fit
from paper_2509_13230_gb300.sampler import expected_bwd, expected_fwd, expected_jacobian_diag

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("model", [nat.MH_UBCM, nat.MH_UECM])
def test_out_of_range_operands_take_the_fp64_terms(model):
    rng = np.random.default_rng(12)
    n = 700
    x = np.exp(rng.normal(-1.0, 1.5, n))
    x[:3] = [1e30, 1e-30, 0.0]  # outside the double-float range, and an isolated node
    y = rng.uniform(0.1, 0.95, n) if model == nat.MH_UECM else None
    k, s = expected_fwd(model, dev(x), None if y is None else dev(y))
    rk, rs = oracle.expected_fwd(model, x, y)
    np.testing.assert_allclose(k.cpu().numpy(), rk, rtol=1e-10, atol=1e-300)
    if y is not None:
        np.testing.assert_allclose(s.cpu().numpy(), rs, rtol=1e-10, atol=1e-300)
    gk = rng.normal(size=n)
    gs = rng.normal(size=n) if y is not None else None
    keep = np.arange(3, n)  # the oracle's closed forms divide by x_i
    gx, gy = expected_bwd(model, dev(x), None if y is None else dev(y), dev(gk), None if gs is None else dev(gs))
    rgx, rgy = oracle.expected_bwd(model, x, y, gk, gs, rows=keep)
    np.testing.assert_allclose(gx.cpu().numpy()[keep], rgx, rtol=1e-10, atol=1e-12 * np.abs(rgx).max())
    if y is not None:
        np.testing.assert_allclose(gy.cpu().numpy()[keep], rgy, rtol=1e-10, atol=1e-12 * np.abs(rgy).max())


@pytest.mark.parametrize("model", [nat.MH_UBCM, nat.MH_UECM])
def test_double_float_range_boundaries(model):
    """Operands on both sides of the double-float range: a (x for the UBCM,
    x y for the UECM) at 2^-30 and 2^30, y at 1 - 2^-12, gradients at 2^40.
    Pairs outside it take the FP64 terms; every sum stays within 1e-10 of
    the oracle's."""
    rng = np.random.default_rng(21)
    n = 600
    x = np.exp(rng.normal(-1.0, 1.0, n))
    y = rng.uniform(0.2, 0.9, n) if model == nat.MH_UECM else None
    a_edges = np.array([2.0**-31, 2.0**-30, 2.0**-29, 2.0**29, 2.0**30, 2.0**31])
    if y is not None:
        y[:6] = 0.5
        x[:6] = a_edges / 0.5  # a = x y exactly at and around the bounds
        y[6:10] = [1 - 2.0**-11, 1 - 2.0**-12, 1 - 2.0**-13, 1 - 2.0**-20]
    else:
        x[:6] = a_edges
    k, s = expected_fwd(model, dev(x), None if y is None else dev(y))
    rk, rs = oracle.expected_fwd(model, x, y)
    np.testing.assert_allclose(k.cpu().numpy(), rk, rtol=1e-10)
    if y is not None:
        np.testing.assert_allclose(s.cpu().numpy(), rs, rtol=1e-10)
    gk = rng.normal(size=n)
    gk[10:14] = [2.0**40, -(2.0**40), 2.0**41, -(2.0**41)]
    gs = None
    if y is not None:
        gs = rng.normal(size=n)
        gs[14:18] = [2.0**40, -(2.0**40), 2.0**41, -(2.0**41)]
    # rows with a >= 2^20 are left out: there p is within 2^-20 of 1 for most
    # pairs and the oracle's closed forms p (1 - p) / x_i lose digits in 1 - p
    a = x * y if y is not None else x
    keep = np.flatnonzero(a < 2.0**20)
    gx, gy = expected_bwd(model, dev(x), None if y is None else dev(y), dev(gk), None if gs is None else dev(gs))
    rgx, rgy = oracle.expected_bwd(model, x, y, gk, gs, rows=keep)
    np.testing.assert_allclose(gx.cpu().numpy()[keep], rgx, rtol=1e-10, atol=1e-12 * np.abs(rgx).max())
    if y is not None:
        np.testing.assert_allclose(gy.cpu().numpy()[keep], rgy, rtol=1e-10, atol=1e-12 * np.abs(rgy).max())


@pytest.mark.parametrize("model", [nat.MH_UBCM, nat.MH_UECM])
def test_row_ranges_equal_the_whole_call_bit_for_bit(model):
    """Ragged row ranges (a rank's share of a call sharded by rows, cut
    across 64-row groups and 32-column batches) give exactly the whole call's
    values for their rows, also where operands take the FP64 terms."""
    from paper_2509_13230_gb300.sampler import row_shard
    rng = np.random.default_rng(22)
    n = 1537
    x = np.exp(rng.normal(-1.0, 1.5, n))
    x[[5, 700]] = [1e30, 1e-30]
    y = rng.uniform(0.1, 0.95, n) if model == nat.MH_UECM else None
    gk = rng.normal(size=n)
    gs = rng.normal(size=n) if y is not None else None
    X, Y = dev(x), None if y is None else dev(y)
    GK, GS = dev(gk), None if gs is None else dev(gs)
    k, s = expected_fwd(model, X, Y)
    gx, gy = expected_bwd(model, X, Y, GK, GS)
    cuts = [0, 1, 64, 129, 700, 829, 1536, 1537]
    ranges = list(zip(cuts, cuts[1:])) + [(b, b + c) for b, c in (row_shard(n, r, 3) for r in range(3))]
    for a, b in ranges:
        kr, sr = expected_fwd(model, X, Y, rows=(a, b - a))
        gxr, gyr = expected_bwd(model, X, Y, GK, GS, rows=(a, b - a))
        assert torch.equal(kr, k[a:b]) and torch.equal(gxr, gx[a:b]), (a, b)
        if y is not None:
            assert torch.equal(sr, s[a:b]) and torch.equal(gyr, gy[a:b]), (a, b)
    kr, _ = expected_fwd(model, X, Y, rows=(n, 0))
    assert kr.numel() == 0


@pytest.mark.parametrize("model", [nat.MH_UBCM, nat.MH_UECM])
def test_jacobian_diagonal_matches_oracle(model):
    """Each node's derivatives of its own <k_i> (and <s_i>) with respect to
    its own x_i (and y_i), against the oracle's closed forms (pinned by
    central differences), with operands on both sides of the double-float
    range; and equal to half the backward kernel with unit upstream
    gradients."""
    rng = np.random.default_rng(23)
    n = 1537
    x = np.exp(rng.normal(-1.0, 1.5, n))
    x[[4, 900]] = [1e30, 2.0**-31]
    y = rng.uniform(0.1, 0.95, n) if model == nat.MH_UECM else None
    if y is not None:
        y[[11, 12]] = [1 - 2.0**-13, 1 - 2.0**-11]
    X, Y = dev(x), None if y is None else dev(y)
    got = [t.cpu().numpy() for t in expected_jacobian_diag(model, X, Y)]
    keep = np.flatnonzero(x < 2.0**20)  # the oracle's closed forms lose digits in 1 - p for p near 1
    ref = oracle.expected_jacobian_diag(model, x, y, rows=keep)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g[keep], r, rtol=1e-10)
    ones, zeros = torch.ones_like(X), torch.zeros_like(X)
    if model == nat.MH_UBCM:
        gx, _ = expected_bwd(model, X, None, ones)
        np.testing.assert_allclose(got[0], 0.5 * gx.cpu().numpy(), rtol=1e-12)
    else:
        gxk, gyk = expected_bwd(model, X, Y, ones, zeros)
        gxs, gys = expected_bwd(model, X, Y, zeros, ones)
        for g, b in zip(got, (gxk, gyk, gxs, gys)):
            np.testing.assert_allclose(g, 0.5 * b.cpu().numpy(), rtol=1e-12)


@pytest.mark.parametrize("model", [nat.MH_UBCM, nat.MH_UECM])
def test_autograd_function_gradcheck(model):
    # The forward is accurate to about 2^-45 relative (double-float terms), so
    # the finite-difference step is 1e-5: truncation and rounding noise both
    # stay near 1e-7, below the tolerance.
    rng = np.random.default_rng(13)
    n = 24
    x = dev(np.exp(rng.normal(-0.5, 1.0, n))).requires_grad_(True)
    if model == nat.MH_UBCM:
        assert torch.autograd.gradcheck(lambda a: ExpectedDegrees.apply(a, None), (x,), eps=1e-5, atol=1e-5,
                                        rtol=1e-4)
    else:
        y = dev(rng.uniform(0.2, 0.9, n)).requires_grad_(True)
        assert torch.autograd.gradcheck(lambda a, b: ExpectedDegrees.apply(a, b), (x, y), eps=1e-5, atol=1e-5,
                                        rtol=1e-4)


def test_fit_ubcm_to_1e8():
    rng = np.random.default_rng(14)
    n = 600
    x_true = np.exp(rng.normal(-2.5, 1.2, n))
    k_t, _ = oracle.expected_fwd(oracle.UBCM, x_true)
    res = fit(dev(k_t), tol=1e-8, adam_steps=100, newton_steps=300)
    assert res.residual <= 1e-8
    k_fit, _ = oracle.expected_fwd(oracle.UBCM, res.x.cpu().numpy())
    assert np.max(np.abs(k_fit - k_t) / k_t) <= 2e-8


def test_fit_uecm_to_1e8():
    rng = np.random.default_rng(15)
    n = 500
    x_true = np.exp(rng.normal(-1.5, 1.0, n))
    y_true = rng.uniform(0.3, 0.9, n)
    k_t, s_t = oracle.expected_fwd(oracle.UECM, x_true, y_true)
    res = fit(dev(k_t), dev(s_t), tol=1e-8, adam_steps=100, newton_steps=400)
    assert res.residual <= 1e-8, res.history[-5:]
    k_fit, s_fit = oracle.expected_fwd(oracle.UECM, res.x.cpu().numpy(), res.y.cpu().numpy())
    assert np.max(np.abs(k_fit - k_t) / k_t) <= 2e-8
    assert np.max(np.abs(s_fit - s_t) / s_t) <= 2e-8


@pytest.mark.parametrize("model", [nat.MH_UBCM, nat.MH_UECM])
def test_jacobian_vector_product_is_the_symmetric_vjp(model):
    # fit() uses J v = (backward kernel with upstream v) * (x, y) in
    # log-parameters; check it against central differences of the oracle's
    # sums along a random direction.
    from paper_2509_13230_gb300.expected import _LocalSums, _jvp
    rng = np.random.default_rng(16)
    n = 300
    theta = rng.normal(-1.5, 1.0, n)
    phi = np.log(rng.uniform(0.2, 0.9, n)) if model == nat.MH_UECM else None
    v = [rng.normal(size=n)] + ([rng.normal(size=n)] if model == nat.MH_UECM else [])
    x, y = np.exp(theta), None if phi is None else np.exp(phi)
    got = _jvp(model, dev(x), None if y is None else dev(y), tuple(dev(a) for a in v),
               _LocalSums(f32_direction=False))
    got32 = _jvp(model, dev(x), None if y is None else dev(y), tuple(dev(a) for a in v), _LocalSums())
    eps = 1e-6

    def sums(sign):
        xs = np.exp(theta + sign * eps * v[0])
        ys = None if phi is None else np.exp(phi + sign * eps * v[1])
        return oracle.expected_fwd(model, xs, ys)

    (kp, sp), (km, sm) = sums(1), sums(-1)
    fd = [(kp - km) / (2 * eps)] + ([(sp - sm) / (2 * eps)] if model == nat.MH_UECM else [])
    for g, g32, f in zip(got, got32, fd):
        np.testing.assert_allclose(g.cpu().numpy(), f, rtol=1e-6, atol=1e-8 * np.abs(f).max())
        # the fit's default: FP32 terms for the Newton direction
        np.testing.assert_allclose(g32.cpu().numpy(), f, rtol=1e-4, atol=1e-5 * np.abs(f).max())


def test_fit_then_sample_full_size():
    """The fit-then-sample workload at full size: N = 200,000 power-law degree
    targets with strengths s = k U(1, 5), fitted to 1e-8 (checked by the
    oracle's sums on sampled rows), then samples drawn in batched waves and
    checked against the oracle's samples of the fitted network."""
    from paper_2509_13230_gb300 import workloads
    from paper_2509_13230_gb300.ensemble import Ensemble
    k_np, s_np = workloads.degree_strength_targets(n=200_000)
    res = fit(dev(k_np), dev(s_np), tol=1e-8)
    assert res.residual <= 1e-8, res.history[-4:]
    x, y = res.x.cpu().numpy(), res.y.cpu().numpy()
    rows = np.random.default_rng(18).choice(len(x), 8, replace=False)
    kk, ss = oracle.expected_fwd(oracle.UECM, x, y, rows=rows)
    assert np.max(np.abs(kk - k_np[rows]) / k_np[rows]) <= 2e-8
    assert np.max(np.abs(ss - s_np[rows]) / s_np[rows]) <= 2e-8
    ens = Ensemble([(nat.MH_UECM, res.x, res.y, 0)], num_samples=40, layout="coo", capacity=1 << 25)
    got = {}

    def keep(w):
        for k in range(w.pair_count):
            if int(w.samples[k]) in (0, 39):
                got[int(w.samples[k])] = [a.cpu().numpy() for a in w.coo(k)]

    counts, _ = ens.sample(on_wave=keep)
    assert abs(2 * counts.mean() / len(x) - k_np.mean()) < 0.05 * k_np.mean()
    for smp, (gs, gd, gw) in got.items():
        check_sample((gs, gd, gw, np.array([len(gs)], np.int64)), oracle.UECM, x, y, sample_begin=smp,
                     num_samples=1)
