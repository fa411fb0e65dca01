"""TV-regularised laminographic reconstruction by ADMM (the paper's appendix on
reconstruction with regularization).

Minimises 1/2 ||L mu - d||^2 + alpha ||grad mu||_1 (Eq. mainregproblem, the
isotropic TV norm) through the augmented Lagrangian of Eq. alagr with the
splitting psi = grad mu, iterating Eqs. tomo, reg and lamd:

* mu-step (Eq. tomo): a few CG iterations on
  F(mu) = 1/2 ||L mu - d||^2 + rho/2 ||grad mu - psi + lambda/rho||^2 (Eq. tomoe),
  gradient L^T(L mu - d) - rho div(grad mu - psi + lambda/rho) (Eq. gradtomo),
  Dai-Yuan directions (Eq. DaiYuan2) and the exact step of the quadratic;
* psi-step (Eq. reg): soft thresholding of grad mu + lambda/rho at alpha/rho,
  the minimiser of Eq. alagr in psi (Eq. solreg writes this shrinkage with
  factors 2 on lambda/rho and alpha/rho, which the Lagrangian as printed does
  not give; the Lagrangian is followed here);
* lambda-step (Eq. lamd): lambda += rho (grad mu - psi).

L and L^T are the library's forward projector and its exact transpose
(backprojection times Ntheta/pi), in the direct or the Fourier form; grad is
the forward difference with a zero last difference and div = -grad^T.
"""
from __future__ import annotations

import math

import torch


def grad(u: torch.Tensor) -> torch.Tensor:
    """Forward differences of a [n2, n1, n0] volume along x3, x2, x1 -> [3, n2, n1, n0]
    (the difference across the last sample of an axis is 0)."""
    g = torch.zeros((3,) + tuple(u.shape), dtype=u.dtype, device=u.device)
    for ax in range(3):
        v, w = u.movedim(ax, 0), g[ax].movedim(ax, 0)
        if v.shape[0] > 1:
            w[:-1] = v[1:] - v[:-1]
    return g


def div(g: torch.Tensor) -> torch.Tensor:
    """The negative adjoint of grad: <grad u, g> = -<u, div g>, i.e.
    div p [i] = p[i] (i < n - 1) - p[i - 1] (i > 0) along every axis."""
    out = torch.zeros(g.shape[1:], dtype=g.dtype, device=g.device)
    for ax in range(3):
        p, o = g[ax].movedim(ax, 0), out.movedim(ax, 0)
        if p.shape[0] > 1:
            o[:-1] += p[:-1]
            o[1:] -= p[:-1]
    return out


def shrink(v: torch.Tensor, t: float) -> torch.Tensor:
    """Isotropic soft thresholding of the vector field v [3, ...] at t."""
    mag = torch.sqrt((v * v).sum(0, keepdim=True))
    return v * torch.clamp(mag - t, min=0.0) / torch.clamp(mag, min=1e-30)


def _dot(a: torch.Tensor, b: torch.Tensor) -> float:
    return float(torch.dot(a.reshape(-1).double(), b.reshape(-1).double()))


def tv_admm(plan, d: torch.Tensor, alpha: float, rho: float, outer: int = 20, inner: int = 4,
            form: str = "fourier", mu0: torch.Tensor | None = None):
    """ADMM for Eq. mainregproblem. Returns (mu, history of the objective
    1/2 ||L mu - d||^2 + alpha ||grad mu||_1 after every outer iteration)."""
    nproj = plan.shape_proj[0]
    scale = nproj / math.pi               # L^T = backprojection * Ntheta / pi

    def LT(r):
        return plan.backproject(r.contiguous(), form) * scale

    def L(u):
        return plan.project(u.contiguous(), form)

    mu = torch.zeros(plan.shape_vol, dtype=torch.float32, device=d.device) if mu0 is None \
        else mu0.clone()
    psi = torch.zeros((3,) + tuple(plan.shape_vol), dtype=torch.float32, device=d.device)
    lam = torch.zeros_like(psi)

    def objective(u):
        r = L(u) - d
        gu = grad(u)
        return 0.5 * _dot(r, r) + alpha * float(torch.sqrt((gu * gu).sum(0)).sum())

    hist = [objective(mu)]
    for _ in range(outer):
        # mu-step: CG on F (Eq. tomoe) with Dai-Yuan directions and exact steps
        b = psi - lam / rho
        r = L(mu) - d
        e = grad(mu) - b
        g = LT(r) - rho * div(e)
        eta = -g
        for _ in range(inner):
            Le, Ge = L(eta), grad(eta)
            den = _dot(Le, Le) + rho * _dot(Ge, Ge)
            if den <= 0.0:
                break
            gamma = -_dot(g, eta) / den
            mu.add_(eta, alpha=gamma)
            r.add_(Le, alpha=gamma)
            e.add_(Ge, alpha=gamma)
            g_new = LT(r) - rho * div(e)
            y = _dot(g_new - g, eta)
            beta = _dot(g_new, g_new) / y if y != 0.0 else 0.0
            eta = -g_new + beta * eta
            g = g_new
        # psi-step (Eq. reg) and dual step (Eq. lamd)
        gm = grad(mu)
        psi = shrink(gm + lam / rho, alpha / rho)
        lam = lam + rho * (gm - psi)
        hist.append(objective(mu))
    return mu, hist
