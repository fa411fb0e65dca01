"""GPU checks of the forward operators and the autograd pair.

* Fourier-form projector against the oracle's exact transpose (8^3, c1 size);
* adjoint identity <L mu, q> pi/Ntheta = <mu, L* q> for both forms on the GPU;
* autograd gradient of 1/2||L mu - d||^2 against central finite differences
  (exact for a quadratic up to rounding) and against the oracle's gradient;
* CG least squares (Appendix A) decreases the residual on a c4-shaped case.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lamino_oracle as O
from paper_2401_11101_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2401_11101_gb300 import _build, lamino
    _build.build()
    lamino.load_library()
    return lamino


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def plan_for(L, g, **kw):
    return L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt, **kw)


@pytest.mark.parametrize("geom", [
    I.Geometry(8, 8, 8, 8, 8, 12, math.radians(20.0)),
    I.Geometry(16, 24, 8, 9, 11, 23, math.radians(25.0)),
    I.Geometry(16, 16, 8, 12, 10, 26, 0.0),
    I.Geometry(16, 16, 256, 4, 400, 24, math.radians(20.0)),  # Hf = M3 = 512: one warp per FFT
])
def test_fourier_projector_matches_oracle(L, geom):
    mu = I.random_volume(geom, 31).astype(np.float32)
    with plan_for(L, geom) as p:
        d = p.project(torch.as_tensor(mu).cuda(), form="fourier").cpu().numpy()
    ref = O.project_fourier(mu, geom)
    e = rel(d, ref)
    print(f"fourier projector {geom} relL2 vs exact transpose = {e:.2e}")
    assert e <= 1e-4


@pytest.mark.parametrize("form", ["direct", "fourier"])
def test_adjoint_identity_gpu(L, form):
    g, _, _ = I.make_projections("c1")
    mu = torch.as_tensor(I.random_volume(g, 32), dtype=torch.float32).cuda()
    q = torch.as_tensor(I.random_projections(g, 33), dtype=torch.float32).cuda()
    with plan_for(L, g) as p:
        lhs = float(torch.dot(p.project(mu, form).double().ravel(), q.double().ravel())) * math.pi / g.nproj
        rhs = float(torch.dot(mu.double().ravel(), p.backproject(q, form).double().ravel()))
    print(f"adjoint {form}: lhs {lhs:.8e} rhs {rhs:.8e} rel {abs(lhs - rhs) / abs(rhs):.2e}")
    assert abs(lhs - rhs) <= 2e-5 * abs(rhs)


@pytest.mark.parametrize("geom", [
    I.Geometry(8, 400, 8, 3, 150, 420, math.radians(20.0)),   # M2 = 1024 (x2 pass), Wf = 512
    I.Geometry(8, 8, 512, 4, 800, 12, math.radians(20.0)),    # Hf = M3 = 1024
])
def test_fourier_adjoint_identity_long_transforms(L, geom):
    mu = torch.as_tensor(I.random_volume(geom, 35), dtype=torch.float32).cuda()
    q = torch.as_tensor(I.random_projections(geom, 36), dtype=torch.float32).cuda()
    with plan_for(L, geom) as p:
        lhs = float(torch.dot(p.project(mu, "fourier").double().ravel(), q.double().ravel())) * math.pi / geom.nproj
        rhs = float(torch.dot(mu.double().ravel(), p.backproject(q, "fourier").double().ravel()))
    print(f"adjoint fourier {geom}: rel {abs(lhs - rhs) / abs(rhs):.2e}")
    assert abs(lhs - rhs) <= 2e-5 * abs(rhs)


@pytest.mark.parametrize("form", ["direct", "fourier"])
def test_autograd_gradient_finite_difference_and_oracle(L, form):
    from paper_2401_11101_gb300 import autograd as A
    g = I.Geometry(8, 8, 8, 8, 8, 12, math.radians(20.0))
    rng = np.random.default_rng(34)
    mu0 = rng.standard_normal((g.n2, g.n1, g.n0)).astype(np.float32)
    d = rng.standard_normal((g.nproj, g.det_h, g.det_w)).astype(np.float32)
    v = rng.standard_normal(mu0.shape).astype(np.float32)
    with plan_for(L, g) as p:
        dt = torch.as_tensor(d).cuda()
        mu = torch.as_tensor(mu0).cuda().requires_grad_(True)
        f = 0.5 * ((A.project(mu, p, form) - dt) ** 2).sum()
        f.backward()
        grad = mu.grad.detach().cpu().numpy()

        def F(x):
            r = p.project(torch.as_tensor(x).cuda(), form).double() - dt.double()
            return 0.5 * float((r * r).sum())
        eps = 1e-2
        fd = (F(mu0 + eps * v) - F(mu0 - eps * v)) / (2 * eps)
    an = float(np.vdot(grad.astype(np.float64), v))
    print(f"{form}: directional derivative autograd {an:.6e} finite difference {fd:.6e}")
    assert abs(an - fd) <= 1e-3 * abs(fd)
    # oracle gradient L^T (L mu - d)
    if form == "direct":
        r = O.project_direct(mu0, g) - d
        og = O.backproject_direct(r, g) * g.nproj / math.pi
    else:
        r = O.project_fourier(mu0, g) - d
        og = O.backproject_fourier(r, g) * g.nproj / math.pi
    e = rel(grad, og)
    print(f"{form}: gradient relL2 vs oracle = {e:.2e}")
    assert e <= (2e-5 if form == "direct" else 2e-4)


def test_autograd_backproject_gradient(L):
    from paper_2401_11101_gb300 import autograd as A
    g = I.Geometry(16, 16, 8, 12, 10, 26, math.radians(30.0))
    q0 = torch.as_tensor(I.random_projections(g, 35), dtype=torch.float32).cuda().requires_grad_(True)
    w = torch.as_tensor(I.random_volume(g, 36), dtype=torch.float32).cuda()
    with plan_for(L, g) as p:
        out = (A.backproject(q0, p, "fourier") * w).sum()
        out.backward()
        ref = p.project(w, "fourier") * (math.pi / g.nproj)
    assert rel(q0.grad.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_cg_least_squares_c4_shape(L):
    from paper_2401_11101_gb300 import autograd as A
    # c4 geometry scaled down 2x per axis (same tilt and angular density)
    g = I.Geometry(128, 128, 64, 200, 64, 192, math.radians(30.0))
    prm = I.blob_params(g, 12, seed=4, sigma=(2.0, 5.0))
    d = I.add_noise(I.project(prm, g), 0.005, 4).float().cuda()
    with plan_for(L, g) as p:
        mu, hist = A.cg_least_squares(p, d, iters=20, form="fourier")
    print("CG residuals:", ["%.3e" % h for h in hist[:5]], "...", "%.3e" % hist[-1])
    assert all(b <= a * (1 + 1e-5) for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.05 * hist[0]
    truth = I.rasterize_blobs(prm, g)
    assert float(np.corrcoef(mu.cpu().numpy().ravel(), truth.ravel())[0, 1]) > 0.9
