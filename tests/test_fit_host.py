"""Host logic of fit() on CPU: the Newton-CG driver (block-diagonal
preconditioner, conjugate gradients, step cap, backtracking) with the oracle's
sums, gradient and Jacobian diagonal standing in for the CUDA kernels, so the
algorithm is checked without a GPU.  Targets come from known parameters; the
fitted parameters are checked by the oracle again."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300 import expected as E


def _np(t):
    return None if t is None else t.detach().cpu().numpy()


@pytest.fixture
def oracle_kernels(monkeypatch):
    calls = {"fwd": 0, "bwd": 0, "diag": 0}

    def fwd(model, x, y=None, stream=None, rows=None, sym=None):
        calls["fwd"] += 1
        k, s = oracle.expected_fwd(model, _np(x), _np(y))
        return torch.from_numpy(k), None if s is None else torch.from_numpy(s)

    def bwd(model, x, y, g_k, g_s=None, stream=None, rows=None, sym=None, f32=False):
        calls["bwd"] += 1
        gx, gy = oracle.expected_bwd(model, _np(x), _np(y), _np(g_k), _np(g_s))
        return torch.from_numpy(gx), None if gy is None else torch.from_numpy(gy)

    def diag(model, x, y=None, stream=None, rows=None, sym=None, f32=False):
        calls["diag"] += 1
        return tuple(torch.from_numpy(a) for a in oracle.expected_jacobian_diag(model, _np(x), _np(y)))

    monkeypatch.setattr(E, "expected_fwd", fwd)
    monkeypatch.setattr(E, "expected_bwd", bwd)
    monkeypatch.setattr(E, "expected_jacobian_diag", diag)
    return calls


def test_newton_cg_fits_the_ubcm_from_the_sparse_limit(oracle_kernels):
    rng = np.random.default_rng(40)
    x_true = np.exp(rng.normal(-2.0, 1.0, 60))
    k_t, _ = oracle.expected_fwd(oracle.UBCM, x_true)
    res = E.fit(torch.from_numpy(k_t), tol=1e-8)
    assert res.adam_steps == 0 and res.residual <= 1e-8
    k_fit, _ = oracle.expected_fwd(oracle.UBCM, res.x.numpy())
    assert np.max(np.abs(k_fit - k_t) / k_t) <= 1e-8
    assert oracle_kernels["diag"] == res.newton_steps  # one preconditioner per Newton step
    np.testing.assert_allclose(res.x.numpy(), x_true, rtol=1e-6)  # the UBCM solution is unique


def test_newton_cg_fits_the_uecm_from_the_sparse_limit(oracle_kernels):
    rng = np.random.default_rng(41)
    n = 50
    x_true = np.exp(rng.normal(-1.5, 0.8, n))
    y_true = rng.uniform(0.3, 0.85, n)
    k_t, s_t = oracle.expected_fwd(oracle.UECM, x_true, y_true)
    res = E.fit(torch.from_numpy(k_t), torch.from_numpy(s_t), tol=1e-8)
    assert res.residual <= 1e-8
    k_fit, s_fit = oracle.expected_fwd(oracle.UECM, res.x.numpy(), res.y.numpy())
    assert np.max(np.abs(k_fit - k_t) / k_t) <= 1e-8
    assert np.max(np.abs(s_fit - s_t) / s_t) <= 1e-8
    assert oracle_kernels["diag"] == res.newton_steps


def test_newton_direction_solves_the_linear_system(oracle_kernels):
    # with enough iterations and a tight tolerance, CG returns J d = b
    rng = np.random.default_rng(42)
    n = 30
    x = torch.from_numpy(np.exp(rng.normal(-1.0, 0.7, n)))
    y = torch.from_numpy(rng.uniform(0.3, 0.8, n))
    b = (torch.from_numpy(rng.normal(size=n)), torch.from_numpy(rng.normal(size=n)))
    ops = E._LocalSums()
    blocks = E._diagonal_blocks(nat.MH_UECM, x, y, n, ops)
    d = E._newton_direction(nat.MH_UECM, x, y, blocks, b, rtol=1e-12, maxiter=200, ops=ops)
    jd = E._jvp(nat.MH_UECM, x, y, d, ops)
    for lhs, rhs in zip(jd, b):
        np.testing.assert_allclose(lhs.numpy(), rhs.numpy(), rtol=1e-8, atol=1e-9)
