"""Pins for the seeded input generators (line integrals of Eq. fwd).

P1: the closed-form projections of Gaussian blobs and ellipsoids are checked
against brute-force ray marching along the beam direction w = a x b, against
the total-mass invariant (the integral of every projection equals the integral
of the phantom) and against the chord of a sphere.
"""
import math

import numpy as np
import pytest
import torch

from paper_2401_11101_gb300 import inputs as I


def _ray_points(geom, k, r, j, s):
    theta = geom.angles[k]
    a, b, w = I.geometry_vectors(np.array([theta]), geom.tilt)
    u = j - geom.det_w / 2.0
    v = r - geom.det_h / 2.0
    p = u * a[0] + v * b[0]
    return p[None, :] + s[:, None] * w[0][None, :]


def test_geometry_vectors_orthonormal():
    th = np.linspace(0, 2 * np.pi, 17)
    for tilt in (0.0, 0.3, 1.1):
        a, b, w = I.geometry_vectors(th, tilt)
        for x, y in ((a, b), (a, w), (b, w)):
            assert np.abs(np.einsum("ki,ki->k", x, y)).max() < 1e-15
        for x in (a, b, w):
            assert np.abs(np.linalg.norm(x, axis=1) - 1).max() < 1e-15
        # w is a x b (right-handed frame)
        assert np.abs(np.cross(a, b) - w).max() < 1e-15


def test_tomography_limit_of_geometry():
    # phi = 0: v = x3 and u = x1 cos t + x2 sin t (Radon transform per slice)
    th = np.linspace(0, 2 * np.pi, 9)
    a, b, w = I.geometry_vectors(th, 0.0)
    assert np.abs(b - np.array([0, 0, 1.0])).max() < 1e-15
    assert np.abs(w[:, 2]).max() < 1e-15


def test_gaussian_projection_matches_ray_marching():
    geom = I.Geometry(16, 16, 8, 7, 12, 20, math.radians(25.0))
    p = I.blob_params(geom, 3, seed=11, sigma=(1.5, 3.0))
    d = I.project(p, geom).numpy()
    s = np.linspace(-60, 60, 120001)
    rng = np.random.default_rng(0)
    for _ in range(12):
        k, r, j = rng.integers(geom.nproj), rng.integers(geom.det_h), rng.integers(geom.det_w)
        x = _ray_points(geom, k, r, j, s)
        f = np.zeros(len(s))
        for c, sg, A in zip(p["centre"], p["sigma"], p["amp"]):
            f += A * np.exp(-((x - c) ** 2).sum(1) / (2 * sg * sg))
        ref = np.trapezoid(f, s)
        assert abs(d[k, r, j] - ref) <= 1e-9 * max(1.0, abs(ref))


def test_gaussian_projection_total_mass():
    # sum over unit pixels of an untruncated projection = A (2 pi)^{3/2} s^3
    geom = I.Geometry(16, 16, 16, 5, 64, 64, math.radians(20.0))
    p = dict(kind="blobs", centre=np.array([[1.3, -0.7, 0.4]]), sigma=np.array([2.5]),
             amp=np.array([0.8]))
    d = I.project(p, geom).numpy()
    mass = 0.8 * (2 * np.pi) ** 1.5 * 2.5 ** 3
    assert np.abs(d.sum(axis=(1, 2)) / mass - 1).max() < 1e-10


def test_sphere_chord():
    geom = I.Geometry(16, 16, 16, 4, 20, 20, math.radians(30.0))
    R = 5.0
    p = dict(kind="ellipsoids", M=np.eye(3)[None] / R, centre=np.zeros((1, 3)),
             rho=np.array([1.0]))
    d = I.project(p, geom).numpy()
    u = np.arange(20) - 10.0
    v = np.arange(20) - 10.0
    rho2 = u[None, :] ** 2 + v[:, None] ** 2
    ref = 2 * np.sqrt(np.clip(R * R - rho2, 0, None))
    for k in range(geom.nproj):
        assert np.abs(d[k] - ref).max() < 1e-12


def test_ellipsoid_projection_matches_ray_marching():
    geom = I.Geometry(32, 32, 16, 6, 24, 40, math.radians(20.0))
    p = I.ellipsoid_params(geom, 4, seed=5)
    d = I.project(p, geom).numpy()
    s = np.linspace(-80, 80, 400001)
    ds = s[1] - s[0]
    rng = np.random.default_rng(1)
    checked = 0
    while checked < 10:
        k, r, j = rng.integers(geom.nproj), rng.integers(geom.det_h), rng.integers(geom.det_w)
        if d[k, r, j] == 0:
            continue
        x = _ray_points(geom, k, r, j, s)
        f = np.zeros(len(s))
        for M, c, rho in zip(p["M"], p["centre"], p["rho"]):
            y = (x - c) @ M.T
            f += rho * ((y ** 2).sum(1) <= 1.0)
        ref = f.sum() * ds
        # indicator marching: error <= (number of boundary crossings) * step
        assert abs(d[k, r, j] - ref) <= 8 * ds + 1e-9
        checked += 1


def test_ellipsoid_projection_total_mass():
    geom = I.Geometry(32, 32, 32, 3, 96, 96, math.radians(20.0))
    axes = np.array([18.0, 12.0, 9.0])
    Rm = I._random_rotation(np.random.default_rng(3))
    p = dict(kind="ellipsoids", M=(np.diag(1 / axes) @ Rm.T)[None], centre=np.array([[1.0, 2.0, -1.0]]),
             rho=np.array([0.7]))
    d = I.project(p, geom).numpy()
    mass = 0.7 * 4.0 / 3.0 * np.pi * axes.prod()
    # midpoint sums of the sqrt-edged chord function converge like h^{3/2}
    assert np.abs(d.sum(axis=(1, 2)) / mass - 1).max() < 2e-3


def test_boxed_projection_equals_dense():
    geom = I.Geometry(48, 40, 24, 9, 30, 70, math.radians(25.0))
    p = I.ellipsoid_params(geom, 7, seed=9, dense_frac=0.3)
    a = I.project(p, geom).numpy()
    b = I.project_boxed(p, geom, angle_chunk=4, batch=3).numpy()
    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def test_poisson_noise_is_seeded_and_unbiased():
    geom = I.Geometry(16, 16, 8, 4, 8, 16, 0.3)
    d = torch.full((4, 8, 16), 0.5, dtype=torch.float64)
    n1, s1 = I.add_poisson(d, 1e4, 3, mu_scale=1.0)
    n2, _ = I.add_poisson(d, 1e4, 3, mu_scale=1.0)
    assert torch.equal(n1, n2)
    assert abs(float(n1.mean()) - 0.5) < 0.01


def test_seeded_inputs_are_reproducible():
    g1, _, d1 = I.make_projections("c1")
    g2, _, d2 = I.make_projections("c1")
    assert g1 == g2
    assert d1.dtype == d2.dtype
    assert bool((d1 == d2).all())
    assert tuple(d1.shape) == (64, 64, 96)


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4"])
def test_config_shapes(name):
    g = I.CONFIGS[name]["geom"]
    assert g.n0 > 0 and g.nproj > 0 and g.det_w % 2 == 0 and g.det_h % 2 == 0
