"""Differentiable expected degrees / strengths and fitting of x, y to targets.

``ExpectedDegrees`` exposes the CUDA kernels behind ``maxent_expected_fwd`` /
``maxent_expected_bwd`` as a ``torch.autograd.Function``: the forward
evaluates <k_i> = sum_j p_ij (and <s_i> = sum_j p_ij / (1 - r_ij)), the
backward recomputes every pair term tile by tile, so nothing of size N^2 is
stored (the maximum-likelihood conditions of Sec. 2.2 and Sec. 2.5).

``fit`` finds x (and y) whose expected degrees (and strengths) match target
sequences, the inference step that precedes sampling (Sec. 3 uses a
quasi-Newton solver for it): Adam on log-parameters through the autograd
Function, then Newton steps on the per-node 1x1 (UBCM) or 2x2 (UECM)
diagonal blocks of the Jacobian until the largest relative residual is at
most ``tol``.  The diagonal blocks come from the backward kernel itself: with
dL/d<k> = 1 and dL/d<s> = 0 it returns 2 d<k_i>/dx_i and 2 d<k_i>/dy_i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import _native as nat
from .sampler import expected_bwd, expected_fwd


class ExpectedDegrees(torch.autograd.Function):
    """(x) -> <k> for the UBCM; (x, y) -> (<k>, <s>) for the UECM."""

    @staticmethod
    def forward(ctx, x, y=None):
        model = nat.MH_UECM if y is not None else nat.MH_UBCM
        ctx.model = model
        ctx.save_for_backward(x, y)
        k, s = expected_fwd(model, x, y)
        if model == nat.MH_UBCM:
            return k
        return k, s

    @staticmethod
    def backward(ctx, g_k, g_s=None):
        x, y = ctx.saved_tensors
        g_k = torch.zeros_like(x) if g_k is None else g_k.contiguous()
        if ctx.model == nat.MH_UBCM:
            gx, _ = expected_bwd(nat.MH_UBCM, x, None, g_k)
            return gx, None
        g_s = torch.zeros_like(x) if g_s is None else g_s.contiguous()
        gx, gy = expected_bwd(nat.MH_UECM, x, y, g_k, g_s)
        return gx, gy


def expected_degrees(x: torch.Tensor, y: torch.Tensor | None = None):
    """Differentiable <k> (UBCM) or (<k>, <s>) (UECM)."""
    return ExpectedDegrees.apply(x, y)


@dataclass
class FitResult:
    x: torch.Tensor
    y: torch.Tensor | None
    residual: float          # max_i |<k_i> - k_i| / k_i (and strengths)
    adam_steps: int
    newton_steps: int
    history: list


def _residual(model, x, y, k_t, s_t):
    k, s = expected_fwd(model, x, y)
    rk = (k - k_t) / k_t
    rs = None if s is None else (s - s_t) / s_t
    worst = float(rk.abs().max()) if rs is None else max(float(rk.abs().max()), float(rs.abs().max()))
    return k, s, rk, rs, worst


def fit(k_target: torch.Tensor, s_target: torch.Tensor | None = None, *, x0=None, y0=None, tol: float = 1e-8,
        adam_steps: int = 200, lr: float = 0.05, newton_steps: int = 200, verbose: bool = False) -> FitResult:
    """Fit x (UBCM) or x, y (UECM) so that the expected degrees (and strengths)
    equal the targets.  Targets are float64 CUDA tensors with k_i > 0 (and
    s_i > k_i, since every weight is at least 1)."""
    model = nat.MH_UECM if s_target is not None else nat.MH_UBCM
    k_t = k_target.to(torch.float64).contiguous()
    s_t = None if s_target is None else s_target.to(torch.float64).contiguous()
    n = k_t.shape[0]
    two_m = float(k_t.sum())
    if x0 is None:
        x0 = k_t / math.sqrt(two_m)  # the sparse limit p_ij ~ x_i x_j
    theta = torch.log(x0.to(torch.float64)).clone()
    phi = None
    if model == nat.MH_UECM:
        if y0 is None:
            # mean weight s/k = 1 / (1 - r): start from r = 1 - k/s spread evenly over both ends
            y0 = torch.sqrt(torch.clamp(1.0 - k_t / s_t, 1e-6, 0.98))
        phi = torch.log(y0.to(torch.float64)).clone()
    history = []

    # --- Adam on (log x, log y) through the autograd Function ---
    params = [theta.requires_grad_(True)] + ([phi.requires_grad_(True)] if phi is not None else [])
    opt = torch.optim.Adam(params, lr=lr)
    steps = 0
    for steps in range(1, adam_steps + 1):
        opt.zero_grad()
        x = torch.exp(theta)
        if model == nat.MH_UBCM:
            k = ExpectedDegrees.apply(x, None)
            loss = torch.mean(((k - k_t) / k_t) ** 2)
        else:
            y = torch.exp(torch.clamp(phi, max=-1e-6))
            k, s = ExpectedDegrees.apply(x, y)
            loss = torch.mean(((k - k_t) / k_t) ** 2) + torch.mean(((s - s_t) / s_t) ** 2)
        loss.backward()
        opt.step()
        if steps % 50 == 0:
            history.append(("adam", steps, float(loss.detach())))
            if verbose:
                print("adam", steps, float(loss.detach()))

    # --- Newton on the diagonal blocks ---
    theta = theta.detach()
    phi = None if phi is None else phi.detach()
    ones = torch.ones(n, dtype=torch.float64, device=k_t.device)
    zeros = torch.zeros_like(ones)
    x = torch.exp(theta)
    y = None if phi is None else torch.exp(phi)
    _, _, rk, rs, worst = _residual(model, x, y, k_t, s_t)
    it = 0
    for it in range(1, newton_steps + 1):
        if worst <= tol:
            it -= 1
            break
        if model == nat.MH_UBCM:
            gx, _ = expected_bwd(model, x, None, ones)
            dk_dtheta = 0.5 * gx * x
            step = -(rk * k_t) / dk_dtheta
            step = torch.clamp(step, -1.0, 1.0)
            t = 1.0
            while True:
                x_new = torch.exp(theta + t * step)
                _, _, rk_new, _, worst_new = _residual(model, x_new, None, k_t, None)
                if worst_new < worst or t < 1e-3:
                    break
                t *= 0.5
            theta = theta + t * step
            x, rk, worst = x_new, rk_new, worst_new
        else:
            gx_k, gy_k = expected_bwd(model, x, y, ones, zeros)
            gx_s, gy_s = expected_bwd(model, x, y, zeros, ones)
            a11, a12 = 0.5 * gx_k * x, 0.5 * gy_k * y   # d<k>/dtheta, d<k>/dphi
            a21, a22 = 0.5 * gx_s * x, 0.5 * gy_s * y   # d<s>/dtheta, d<s>/dphi
            b1, b2 = -rk * k_t, -rs * s_t
            det = a11 * a22 - a12 * a21
            d_theta = (b1 * a22 - a12 * b2) / det
            d_phi = (a11 * b2 - a21 * b1) / det
            d_theta = torch.clamp(d_theta, -1.0, 1.0)
            d_phi = torch.clamp(d_phi, -1.0, 1.0)
            t = 1.0
            while True:
                th_new = theta + t * d_theta
                ph_new = torch.clamp(phi + t * d_phi, max=-1e-9)
                x_new, y_new = torch.exp(th_new), torch.exp(ph_new)
                _, _, rk_new, rs_new, worst_new = _residual(model, x_new, y_new, k_t, s_t)
                if worst_new < worst or t < 1e-3:
                    break
                t *= 0.5
            theta, phi = th_new, ph_new
            x, y, rk, rs, worst = x_new, y_new, rk_new, rs_new, worst_new
        history.append(("newton", it, worst))
        if verbose:
            print("newton", it, worst)
    return FitResult(x=x, y=y, residual=worst, adam_steps=steps, newton_steps=it, history=history)
