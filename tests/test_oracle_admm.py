"""Pins for the FP64 ADMM reference (oracle/lamino_admm.py): its pieces against
what the mathematics fixes, independently of the GPU path.

* grad / div: div = -grad^T (inner products), and grad of a linear ramp;
* the psi-step: the isotropic soft threshold is the proximal map of
  t |.| (closed form for a vector, and no perturbation lowers the objective);
* the whole iteration at alpha = 0: Eq. mainregproblem reduces to least
  squares, so ADMM must reach the minimum that numpy's lstsq finds on the
  explicit matrix of the oracle's direct projector.
"""
import math

import numpy as np
import pytest

from oracle import lamino_admm as A
from oracle import lamino_oracle as O
from paper_2401_11101_gb300 import inputs as I


def test_div_is_minus_grad_transpose():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((5, 6, 7))
    p = rng.standard_normal((3, 5, 6, 7))
    lhs = float((A.grad(u) * p).sum())
    rhs = -float((u * A.div(p)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_grad_of_a_ramp():
    n2, n1, n0 = 4, 5, 6
    x1 = np.arange(n0)[None, None, :] * np.ones((n2, n1, 1))
    g = A.grad(2.5 * x1)
    assert np.allclose(g[2][:, :, :-1], 2.5) and np.all(g[2][:, :, -1] == 0)
    assert np.all(g[0] == 0) and np.all(g[1] == 0)


def test_shrink_is_the_proximal_map():
    rng = np.random.default_rng(2)
    v = rng.standard_normal((3, 50))
    t = 0.7
    w = A.shrink(v, t)
    mag = np.linalg.norm(v, axis=0)
    # closed form: v (1 - t/|v|)_+
    ref = v * np.maximum(0.0, 1.0 - t / mag)[None]
    assert np.allclose(w, ref, atol=1e-14)

    def obj(z):
        return t * np.linalg.norm(z, axis=0) + 0.5 * ((z - v) ** 2).sum(axis=0)

    base = obj(w)
    for _ in range(20):
        assert np.all(obj(w + 1e-3 * rng.standard_normal(w.shape)) >= base - 1e-12)


def test_admm_without_regularisation_reaches_least_squares():
    g = I.Geometry(6, 6, 4, 8, 8, 12, math.radians(25.0))
    rng = np.random.default_rng(3)
    d = rng.standard_normal((g.nproj, g.det_h, g.det_w))
    # explicit matrix of the direct projector, column by column
    n = g.nvox
    M = np.zeros((g.nproj * g.det_h * g.det_w, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = O.project_direct(e.reshape(g.n2, g.n1, g.n0), g).ravel()
    x, *_ = np.linalg.lstsq(M, d.ravel(), rcond=None)
    best = 0.5 * float(((M @ x - d.ravel()) ** 2).sum())
    # with alpha = 0 the psi-step copies grad mu and lambda returns to 0, so the
    # outer loop is a proximal-point iteration on the data term; a small rho
    # makes each step nearly the full least-squares step
    mu, hist = A.tv_admm(d, g, alpha=0.0, rho=1e-3, outer=20, inner=40, form="direct")
    print(f"least squares minimum {best:.9e}, ADMM (alpha = 0) {hist[-1]:.9e}")
    assert abs(hist[-1] - best) <= 1e-9 * best
    assert np.linalg.norm(M @ mu.ravel() - M @ x) <= 1e-6 * np.linalg.norm(M @ x)
