"""FP64 reference of TV-regularised laminographic reconstruction by ADMM.

TEST INFRASTRUCTURE ONLY (like everything under ``oracle/``): only the test
suite may import it. It shares no code with the product; its operators are the
oracle's exact ones (lamino_oracle: the bilinear direct form or the exact
type-1 sum of the Fourier form and their transposes), in double precision.

It follows the appendix of Nikitin et al. (arXiv 2401.11101) on reconstruction
with regularization:

* problem (Eq. mainregproblem): minimise 1/2 ||L mu - d||^2 + alpha ||grad mu||_1
  with the isotropic norm sum_x |grad mu(x)|;
* splitting psi = grad mu and the augmented Lagrangian of Eq. alagr,
  1/2 ||L mu - d||^2 + alpha ||psi||_1 + <lambda, grad mu - psi>
  + rho/2 ||grad mu - psi||^2;
* mu-step (Eq. tomo): conjugate gradients on the quadratic
  F(mu) = 1/2 ||L mu - d||^2 + rho/2 ||grad mu - psi + lambda/rho||^2
  (Eq. tomoe), gradient L^T (L mu - d) - rho div(grad mu - psi + lambda/rho)
  (Eq. gradtomo), Dai-Yuan directions (Eq. DaiYuan2) and the exact step along
  each direction (F is quadratic);
* psi-step (Eq. reg): the minimiser of the Lagrangian in psi, an isotropic soft
  threshold of grad mu + lambda/rho at alpha/rho (the reading of Eq. solreg
  that the Lagrangian gives; as printed, Eq. solreg carries factors 2 that the
  Lagrangian does not produce);
* lambda-step (Eq. lamd): lambda += rho (grad mu - psi).

grad is the forward difference along x3, x2, x1 with the difference across the
last sample set to 0; div is minus its transpose. L^T is the transpose of the
forward operator: the backprojection times Ntheta/pi.
"""
from __future__ import annotations

import math

import numpy as np

from . import lamino_oracle as O


def grad(u: np.ndarray) -> np.ndarray:
    """Forward differences of u [n2, n1, n0]: [3, n2, n1, n0], the difference
    across the last sample of each axis being 0."""
    g = np.zeros((3,) + u.shape)
    for ax in range(3):
        d = np.diff(u, axis=ax)
        sl = [slice(None)] * 3
        sl[ax] = slice(0, u.shape[ax] - 1)
        g[ax][tuple(sl)] = d
    return g


def div(p: np.ndarray) -> np.ndarray:
    """Minus the transpose of grad, written out per axis:
    (div p)[i] = p[i] (for i < n-1) - p[i-1] (for i > 0)."""
    out = np.zeros(p.shape[1:])
    for ax in range(3):
        n = p.shape[1 + ax]
        for i in range(n):
            dst = [slice(None)] * 3
            dst[ax] = i
            if i < n - 1:
                src = [slice(None)] * 3
                src[ax] = i
                out[tuple(dst)] += p[ax][tuple(src)]
            if i > 0:
                src = [slice(None)] * 3
                src[ax] = i - 1
                out[tuple(dst)] -= p[ax][tuple(src)]
    return out


def shrink(v: np.ndarray, t: float) -> np.ndarray:
    """Isotropic soft threshold of a field v [3, ...]: each vector v(x) shrunk
    towards 0 by t in length (0 if shorter than t)."""
    mag = np.sqrt((v * v).sum(axis=0))
    fac = np.where(mag > t, (mag - t) / np.where(mag > 0, mag, 1.0), 0.0)
    return v * fac[None]


def operators(geom, form: str):
    """(L, L^T) of the oracle in one form, float64."""
    if form == "fourier":
        fwd, bwd = O.project_fourier, O.backproject_fourier
    else:
        fwd, bwd = O.project_direct, O.backproject_direct
    scale = geom.nproj / math.pi
    return (lambda u: fwd(u, geom)), (lambda r: bwd(r, geom) * scale)


def objective(L, d, mu, alpha) -> float:
    r = L(mu) - d
    g = grad(mu)
    return 0.5 * float((r * r).sum()) + alpha * float(np.sqrt((g * g).sum(axis=0)).sum())


def tv_admm(d, geom, alpha: float, rho: float, outer: int, inner: int, form: str = "fourier"):
    """ADMM for Eq. mainregproblem from mu = 0, psi = 0, lambda = 0; `outer`
    iterations of Eqs. tomo, reg and lamd, `inner` CG steps each. Returns
    (mu, history of the objective after every outer iteration)."""
    L, LT = operators(geom, form)
    d = np.asarray(d, dtype=np.float64)
    mu = np.zeros((geom.n2, geom.n1, geom.n0))
    psi = np.zeros((3,) + mu.shape)
    lam = np.zeros_like(psi)
    hist = [objective(L, d, mu, alpha)]
    for _ in range(outer):
        target = psi - lam / rho                    # grad mu should approach this
        r = L(mu) - d                               # residual of the data term
        e = grad(mu) - target                       # residual of the coupling term
        g = LT(r) - rho * div(e)                    # Eq. gradtomo
        eta = -g
        for _ in range(inner):
            Le, Ge = L(eta), grad(eta)
            curv = float((Le * Le).sum()) + rho * float((Ge * Ge).sum())
            if curv <= 0.0:
                break
            step = -float((g * eta).sum()) / curv    # exact minimiser along eta
            mu = mu + step * eta
            r = r + step * Le
            e = e + step * Ge
            g_next = LT(r) - rho * div(e)
            y = float(((g_next - g) * eta).sum())
            beta = float((g_next * g_next).sum()) / y if y != 0.0 else 0.0   # Eq. DaiYuan2
            eta = -g_next + beta * eta
            g = g_next
        gm = grad(mu)
        psi = shrink(gm + lam / rho, alpha / rho)   # Eq. reg (Lagrangian reading)
        lam = lam + rho * (gm - psi)                # Eq. lamd
        hist.append(objective(L, d, mu, alpha))
    return mu, hist
