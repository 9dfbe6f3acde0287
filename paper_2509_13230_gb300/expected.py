"""Differentiable expected degrees / strengths and fitting of x, y to targets.

``ExpectedDegrees`` exposes the CUDA kernels behind ``maxent_expected_fwd`` /
``maxent_expected_bwd`` as a ``torch.autograd.Function``: the forward
evaluates <k_i> = sum_j p_ij (and <s_i> = sum_j p_ij / (1 - r_ij)), the
backward recomputes every pair term tile by tile, so nothing of size N^2 is
stored (the maximum-likelihood conditions of Sec. 2.2 and Sec. 2.5).

``fit`` finds x (and y) whose expected degrees (and strengths) match target
sequences, the inference step that precedes sampling (Sec. 3 uses a
quasi-Newton solver for it): Adam on log-parameters through the autograd
Function, then inexact Newton steps until the largest relative residual is
at most ``tol``.  In log-parameters (theta = log x, phi = log y) the
Jacobian of (<k>, <s>) is symmetric: <k_i> and <s_i> are the derivatives of
the model's log-partition function, and pair by pair
d<k_i>/dtheta_j = p_ij (1 - p_ij), d<k_i>/dphi_j = d<s_j>/dtheta_i = A / D^2.
So J v equals the backward kernel's vector-Jacobian product times x (and y),
and each Newton step solves J d = -(residual) by conjugate gradients
preconditioned with the per-node 1x1 / 2x2 diagonal blocks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import _native as nat
from .sampler import SymWorkspace, expected_bwd, expected_fwd, expected_jacobian_diag


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


class _LocalSums:
    """The sums of a fit on this process's GPU (the module's functions, looked
    up at call time): each unordered pair evaluated once for both of its rows
    (the symmetric forms), with one scratch buffer for the fit.  The residual
    (fwd) takes the double-float terms; the Newton direction's products (bwd)
    and preconditioner (diag) take the FP32 terms unless f32_direction is
    False: conjugate gradients stopped at a relative residual of 5e-2 need
    nothing closer than their 1e-5."""

    def __init__(self, f32_direction: bool = True):
        self.ws = SymWorkspace()
        self.f32 = f32_direction

    def fwd(self, model, x, y=None):
        return expected_fwd(model, x, y, sym=self.ws)

    def bwd(self, model, x, y, g_k, g_s=None):
        return expected_bwd(model, x, y, g_k, g_s, sym=self.ws, f32=self.f32)

    def diag(self, model, x, y=None):
        return expected_jacobian_diag(model, x, y, sym=self.ws, f32=self.f32)


def _residual(model, x, y, k_t, s_t, ops):
    k, s = ops.fwd(model, x, y)
    rk = (k - k_t) / k_t
    rs = None if s is None else (s - s_t) / s_t
    worst = float(rk.abs().max()) if rs is None else max(float(rk.abs().max()), float(rs.abs().max()))
    merit = float((rk * rk).sum()) + (0.0 if rs is None else float((rs * rs).sum()))
    return k, s, rk, rs, worst, merit


def _diagonal_blocks(model, x, y, n, ops):
    """Per-node d<k_i>/dtheta_i (UBCM) or the 2x2 block of d(<k_i>, <s_i>) /
    d(theta_i, phi_i) (UECM), theta = log x and phi = log y: the Jacobian
    diagonal kernel's derivatives in x and y times x_i and y_i."""
    if model == nat.MH_UBCM:
        (dk_dx,) = ops.diag(model, x, None)
        return (dk_dx * x,)
    dk_dx, dk_dy, ds_dx, ds_dy = ops.diag(model, x, y)
    return dk_dx * x, dk_dy * y, ds_dx * x, ds_dy * y


def _jvp(model, x, y, v, ops=None):
    """J v in log-parameters (J symmetric: the vector-Jacobian product)."""
    ops = ops or _LocalSums()
    if model == nat.MH_UBCM:
        gx, _ = ops.bwd(model, x, None, v[0].contiguous())
        return (gx * x,)
    gx, gy = ops.bwd(model, x, y, v[0].contiguous(), v[1].contiguous())
    return gx * x, gy * y


def _precond(blocks, r):
    """Solves each node's diagonal block against r."""
    if len(blocks) == 1:
        return (r[0] / blocks[0],)
    a11, a12, a21, a22 = blocks
    det = a11 * a22 - a12 * a21
    return (r[0] * a22 - a12 * r[1]) / det, (a11 * r[1] - a21 * r[0]) / det


def _dot(u, v):
    return float(sum((a * b).sum() for a, b in zip(u, v)))


def _newton_direction(model, x, y, blocks, b, *, rtol: float, maxiter: int, ops=None):
    """Preconditioned conjugate gradients on J d = b, started from the
    block-diagonal solution."""
    ops = ops or _LocalSums()
    d = _precond(blocks, b)
    Jd = _jvp(model, x, y, d, ops)
    r = tuple(bi - ji for bi, ji in zip(b, Jd))
    bnorm = math.sqrt(_dot(b, b))
    z = _precond(blocks, r)
    p = z
    rz = _dot(r, z)
    for _ in range(maxiter):
        if math.sqrt(_dot(r, r)) <= rtol * bnorm:
            break
        Ap = _jvp(model, x, y, p, ops)
        pAp = _dot(p, Ap)
        if not pAp > 0.0:
            break
        alpha = rz / pAp
        d = tuple(di + alpha * pi for di, pi in zip(d, p))
        r = tuple(ri - alpha * ai for ri, ai in zip(r, Ap))
        z = _precond(blocks, r)
        rz_new = _dot(r, z)
        p = tuple(zi + (rz_new / rz) * pi for zi, pi in zip(z, p))
        rz = rz_new
    return d


def fit(k_target: torch.Tensor, s_target: torch.Tensor | None = None, *, x0=None, y0=None, tol: float = 1e-8,
        adam_steps: int = 0, lr: float = 0.05, newton_steps: int = 100, cg_iters: int = 12,
        cg_rtol: float = 0.05, max_step: float = 2.0, verbose: bool = False, sums=None) -> FitResult:
    """Fit x (UBCM) or x, y (UECM) so that the expected degrees (and strengths)
    equal the targets.  Targets are float64 CUDA tensors with k_i > 0 (and
    s_i > k_i, since every weight is at least 1).

    Adam stage (optional, none by default): adam_steps steps on the mean
    squared relative residual as a warm start.  From the sparse-limit start the
    Newton stage alone reached 1e-8 on the N = 2*10^5 degree and strength
    targets in the same 11 steps as after 10 Adam steps, without their 10
    forward and 10 backward passes.
    Newton stage: each step solves J d = -(<k> - k, <s> - s) by up to
    cg_iters preconditioned conjugate-gradient iterations (relative residual
    cg_rtol), scales d to at most max_step per log-parameter, and backtracks
    on the sum of squared relative residuals.
    sums: where the Newton stage's sums, gradients and Jacobian diagonal come
    from (default: this GPU); ``distributed.ShardedSums(group)`` splits them
    by rows over the ranks of a torch.distributed group, every rank then
    taking the same steps (the Adam stage stays on each rank's GPU)."""
    ops = sums if sums is not None else _LocalSums()
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

    # --- inexact Newton (preconditioned CG), line search on the squared residuals ---
    theta = theta.detach()
    phi = None if phi is None else torch.clamp(phi.detach(), max=-1e-9)
    x = torch.exp(theta)
    y = None if phi is None else torch.exp(phi)
    k, s, rk, rs, worst, merit = _residual(model, x, y, k_t, s_t, ops)
    it = 0
    for it in range(1, newton_steps + 1):
        if worst <= tol:
            it -= 1
            break
        blocks = _diagonal_blocks(model, x, y, n, ops)
        b = (k_t - k,) if model == nat.MH_UBCM else (k_t - k, s_t - s)
        d = _newton_direction(model, x, y, blocks, b, rtol=cg_rtol, maxiter=cg_iters, ops=ops)
        biggest = max(float(di.abs().max()) for di in d)
        if biggest > max_step:
            d = tuple(di * (max_step / biggest) for di in d)
        t = 1.0
        accepted = False
        while t >= 1.0 / 256:
            th_new = theta + t * d[0]
            ph_new = None if phi is None else torch.clamp(phi + t * d[1], max=-1e-9)
            x_new = torch.exp(th_new)
            y_new = None if ph_new is None else torch.exp(ph_new)
            k_new, s_new, rk_new, rs_new, worst_new, merit_new = _residual(model, x_new, y_new, k_t, s_t, ops)
            if merit_new < (1.0 - 1e-4 * t) * merit:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            history.append(("newton-stalled", it, worst))
            break
        theta, phi, x, y = th_new, ph_new, x_new, y_new
        k, s, rk, rs, worst, merit = k_new, s_new, rk_new, rs_new, worst_new, merit_new
        history.append(("newton", it, worst, t))
        if verbose:
            print("newton", it, worst, merit, t)
    return FitResult(x=x, y=y, residual=worst, adam_steps=steps, newton_steps=it, history=history)
