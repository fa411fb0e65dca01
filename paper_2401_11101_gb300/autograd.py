"""Differentiable laminographic operators and CG least-squares reconstruction.

The backprojection L* (Eq. adj / Eq. fftadj, times pi/Ntheta) and the forward
operator L (Eq. fwd / Eq. fftfwd, the exact transpose of the chosen
backprojection without that weight) form a torch.autograd.Function pair: the
gradient of each is the other, so

    <L mu, q> * pi/Ntheta = <mu, L* q>

holds to rounding, for the direct and for the Fourier form. Both run in the CUDA
library through the binding; this module only wires them into autograd.

cg_least_squares minimises 1/2 ||L mu - d||^2 with the conjugate-gradient
iteration of the paper's Appendix A: search direction by the Dai-Yuan formula
(Eq. DaiYuan2), step length by an exact line search (the objective is
quadratic along the direction).
"""
from __future__ import annotations

import math

import torch


def _nproj(plan) -> int:
    return plan.shape_proj[0]


class _Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, plan, form):
        ctx.plan, ctx.form = plan, form
        return plan.backproject(q.detach().contiguous(), form)

    @staticmethod
    def backward(ctx, g):
        p = ctx.plan
        gq = p.project(g.detach().contiguous(), ctx.form) * (math.pi / _nproj(p))
        return gq, None, None


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, plan, form):
        ctx.plan, ctx.form = plan, form
        return plan.project(vol.detach().contiguous(), form)

    @staticmethod
    def backward(ctx, g):
        p = ctx.plan
        gv = p.backproject(g.detach().contiguous(), ctx.form) * (_nproj(p) / math.pi)
        return gv, None, None


def backproject(q: torch.Tensor, plan, form: str = "fourier") -> torch.Tensor:
    """Differentiable L* q (pi/Ntheta-weighted backprojection)."""
    return _Backproject.apply(q, plan, form)


def project(vol: torch.Tensor, plan, form: str = "fourier") -> torch.Tensor:
    """Differentiable L vol (the transpose of backproject without its weight)."""
    return _Project.apply(vol, plan, form)


def _dot(a: torch.Tensor, b: torch.Tensor) -> float:
    return float(torch.dot(a.reshape(-1).double(), b.reshape(-1).double()))


def cg_least_squares(plan, d: torch.Tensor, iters: int = 50, form: str = "fourier",
                     mu0: torch.Tensor | None = None, callback=None):
    """Minimise F(mu) = 1/2 ||L mu - d||^2 by CG (Appendix A).

    grad F = L^T (L mu - d), computed as backproject(residual) * Ntheta/pi;
    eta_0 = -grad F(mu_0); step gamma = -<grad, eta>/||L eta||^2 (exact for the
    quadratic); eta_{m+1} = -g_{m+1} + ||g_{m+1}||^2 / <g_{m+1} - g_m, eta_m> eta_m
    (Dai-Yuan). Returns (mu, history of 1/2 ||L mu - d||^2).
    """
    scale = _nproj(plan) / math.pi
    mu = torch.zeros(plan.shape_vol, dtype=torch.float32, device=d.device) if mu0 is None \
        else mu0.clone()
    r = plan.project(mu, form) - d
    g = plan.backproject(r, form) * scale
    eta = -g
    hist = [0.5 * _dot(r, r)]
    for it in range(iters):
        Le = plan.project(eta.contiguous(), form)
        den = _dot(Le, Le)
        if den <= 0.0:
            break
        gamma = -_dot(g, eta) / den
        mu.add_(eta, alpha=gamma)
        r.add_(Le, alpha=gamma)
        g_new = plan.backproject(r, form) * scale
        y = _dot(g_new - g, eta)
        beta = _dot(g_new, g_new) / y if y != 0.0 else 0.0
        eta = -g_new + beta * eta
        g = g_new
        hist.append(0.5 * _dot(r, r))
        if callback is not None:
            callback(it, mu, hist[-1])
    return mu, hist
