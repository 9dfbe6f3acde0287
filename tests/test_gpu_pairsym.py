"""Symmetric pair sums (maxent_expected_*_sym): each unordered pair once (GPU).

Checked against the CPU oracle's compensated FP64 sums (which share nothing
with either CUDA form) and against the row forms within the bound the two
forms share: about 1e-11 of the sum of the terms' magnitudes.  Sizes cross
the band length (2048), the sub-band (512) and the tile (32) with ragged
tails, so off-diagonal units, diagonal units and diagonal tiles are all
exercised; operands outside the double-float range send their tiles to the
FP64 terms.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300.sampler import (SymWorkspace, expected_bwd, expected_fwd, expected_jacobian_diag,
                                            _ptr)

pytestmark = pytest.mark.gpu

UBCM, UECM = nat.MH_UBCM, nat.MH_UECM


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def params(model, n, seed, extremes=False):
    rng = np.random.default_rng(seed)
    x = np.exp(rng.normal(-2.0, 1.5, n))
    y = rng.uniform(0.1, 0.95, n) if model == UECM else None
    if extremes and n > 40:
        x[[3, n // 2]] = [1e30, 2.0**-33]  # outside the double-float range: FP64 tiles
        x[n - 7] = 0.0                     # an isolated node
        if y is not None:
            y[17] = 1 - 2.0**-13
    return x, y


def close(got, ref, scale, tol=2e-11):
    got, ref = np.asarray(got), np.asarray(ref)
    assert np.all(np.abs(got - ref) <= tol * np.maximum(scale, 1e-300)), np.max(np.abs(got - ref) / scale)


SIZES = [1, 2, 31, 33, 517, 2048, 2049, 4700, 6145]


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("n", SIZES)
def test_sym_sums_equal_the_row_form(model, n):
    x, y = params(model, n, 100 + n, extremes=True)
    X, Y = dev(x), dev(y)
    ws = SymWorkspace()
    k, s = expected_fwd(model, X, Y, sym=ws)
    kr, sr = expected_fwd(model, X, Y)
    close(k.cpu().numpy(), kr.cpu().numpy(), kr.cpu().numpy())  # positive terms: the sum is its own scale
    if model == UECM:
        close(s.cpu().numpy(), sr.cpu().numpy(), sr.cpu().numpy())
    got = expected_jacobian_diag(model, X, Y, sym=ws)
    ref = expected_jacobian_diag(model, X, Y)
    for g, r in zip(got, ref):
        r = r.cpu().numpy()
        close(g.cpu().numpy(), r, np.abs(r))
    rng = np.random.default_rng(n)
    gk = rng.normal(size=n)
    gs = rng.normal(size=n) if model == UECM else None
    GK, GS = dev(gk), dev(gs)
    gx, gy = expected_bwd(model, X, Y, GK, GS, sym=ws)
    rx, ry = expected_bwd(model, X, Y, GK, GS)
    # the terms are linear in the upstream gradients with positive factors:
    # the sums with |g| bound the sums of the terms' magnitudes
    ax, ay = expected_bwd(model, X, Y, GK.abs(), None if GS is None else GS.abs())
    close(gx.cpu().numpy(), rx.cpu().numpy(), ax.cpu().numpy())
    if model == UECM:
        close(gy.cpu().numpy(), ry.cpu().numpy(), ay.cpu().numpy())


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_sym_sums_match_the_oracle(model):
    n = 5000
    x, y = params(model, n, 7)
    X, Y = dev(x), dev(y)
    ws = SymWorkspace()
    k, s = expected_fwd(model, X, Y, sym=ws)
    rk, rs = oracle.expected_fwd(model, x, y)
    np.testing.assert_allclose(k.cpu().numpy(), rk, rtol=1e-10)
    if model == UECM:
        np.testing.assert_allclose(s.cpu().numpy(), rs, rtol=1e-10)
    rows = np.array([0, 1, 31, 32, 511, 512, 2047, 2048, 2049, 4095, 4999])
    got = [t.cpu().numpy()[rows] for t in expected_jacobian_diag(model, X, Y, sym=ws)]
    ref = oracle.expected_jacobian_diag(model, x, y, rows=rows)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=1e-10)
    rng = np.random.default_rng(8)
    gk = rng.normal(size=n)
    gs = rng.normal(size=n) if model == UECM else None
    gx, gy = expected_bwd(model, X, Y, dev(gk), dev(gs), sym=ws)
    rgx, rgy = oracle.expected_bwd(model, x, y, gk, gs, rows=rows)
    np.testing.assert_allclose(gx.cpu().numpy()[rows], rgx, rtol=1e-9, atol=1e-12 * np.abs(rgx).max())
    if model == UECM:
        np.testing.assert_allclose(gy.cpu().numpy()[rows], rgy, rtol=1e-9, atol=1e-12 * np.abs(rgy).max())


@pytest.mark.parametrize("model", [UBCM, UECM])
def test_sym_sums_are_deterministic(model):
    n = 4700
    x, y = params(model, n, 9, extremes=True)
    X, Y = dev(x), dev(y)
    ws = SymWorkspace()
    a = expected_fwd(model, X, Y, sym=ws)
    b = expected_fwd(model, X, Y, sym=SymWorkspace())
    for u, v in zip(a, b):
        if u is not None:
            assert torch.equal(u, v)
    d1 = expected_jacobian_diag(model, X, Y, sym=ws)
    d2 = expected_jacobian_diag(model, X, Y, sym=ws)
    for u, v in zip(d1, d2):
        assert torch.equal(u, v)


def test_sym_argument_errors():
    n = 100
    x, y = params(UECM, n, 3)
    X, Y = dev(x), dev(y)
    rc, need = nat.maxent_expected_sym_workspace_size(UECM, n)
    assert rc == nat.MH_OK and need > 0
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    k = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.empty_like(k)
    stream = None
    assert nat.maxent_expected_fwd_sym(UECM, _ptr(X), _ptr(Y), n, _ptr(k), _ptr(s), _ptr(ws), need - 1,
                                       stream) == nat.MH_ERR_WORKSPACE
    assert nat.maxent_expected_fwd_sym(UECM, _ptr(X), _ptr(Y), n, _ptr(k), _ptr(s), None, need,
                                       stream) == nat.MH_ERR_WORKSPACE
    assert nat.maxent_expected_fwd_sym(UECM, _ptr(X), None, n, _ptr(k), _ptr(s), _ptr(ws), need,
                                       stream) == nat.MH_ERR_ARG
    misaligned = ctypes.c_void_p(ws.data_ptr() + 8)
    assert nat.maxent_expected_fwd_sym(UECM, _ptr(X), _ptr(Y), n, _ptr(k), _ptr(s), misaligned, need,
                                       stream) == nat.MH_ERR_ARG
    assert nat.maxent_expected_fwd_sym(7, _ptr(X), _ptr(Y), n, _ptr(k), _ptr(s), _ptr(ws), need,
                                       stream) == nat.MH_ERR_ARG
    assert nat.maxent_expected_fwd_sym(UECM, _ptr(X), _ptr(Y), 0, _ptr(k), _ptr(s), _ptr(ws), need,
                                       stream) == nat.MH_ERR_ARG
    with pytest.raises(ValueError):
        expected_fwd(UECM, X, Y, rows=(0, 10), sym=SymWorkspace())
    assert nat.maxent_expected_fwd_sym(UECM, _ptr(X), _ptr(Y), n, _ptr(k), _ptr(s), _ptr(ws), need,
                                       stream) == nat.MH_OK
    torch.cuda.synchronize()


@pytest.mark.parametrize("model", [UBCM, UECM])
@pytest.mark.parametrize("n", [1, 33, 2049, 6145])
def test_f32_forms_within_their_bound(model, n):
    """The FP32 forms (Newton directions) against the double-float forms:
    within 2e-5 of the sum of the terms' magnitudes (FP32 terms of a few ulp,
    FP32 sums over tiles of 32 and 64 terms), extremes taking FP64 tiles."""
    x, y = params(model, n, 500 + n, extremes=True)
    X, Y = dev(x), dev(y)
    ws = SymWorkspace()
    got = expected_jacobian_diag(model, X, Y, sym=ws, f32=True)
    ref = expected_jacobian_diag(model, X, Y, sym=ws)
    for g, r in zip(got, ref):
        r = r.cpu().numpy()
        close(g.cpu().numpy(), r, np.abs(r), tol=2e-5)  # positive terms
    rng = np.random.default_rng(n + 1)
    GK = dev(rng.normal(size=n))
    GS = dev(rng.normal(size=n)) if model == UECM else None
    gx, gy = expected_bwd(model, X, Y, GK, GS, sym=ws, f32=True)
    rx, ry = expected_bwd(model, X, Y, GK, GS, sym=ws)
    ax, ay = expected_bwd(model, X, Y, GK.abs(), None if GS is None else GS.abs(), sym=ws)
    close(gx.cpu().numpy(), rx.cpu().numpy(), ax.cpu().numpy(), tol=2e-5)
    if model == UECM:
        close(gy.cpu().numpy(), ry.cpu().numpy(), ay.cpu().numpy(), tol=2e-5)
    # deterministic, like the other symmetric forms
    gx2, _ = expected_bwd(model, X, Y, GK, GS, sym=SymWorkspace(), f32=True)
    assert torch.equal(gx, gx2)


def test_f32_forms_need_the_symmetric_form():
    x, y = params(UECM, 10, 1)
    X, Y = dev(x), dev(y)
    with pytest.raises(ValueError):
        expected_jacobian_diag(UECM, X, Y, f32=True)
    with pytest.raises(ValueError):
        expected_bwd(UECM, X, Y, X, X, f32=True)
