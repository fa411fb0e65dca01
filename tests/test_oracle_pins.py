"""Pins for the FP64 oracle: each test ties it to something other than itself.

P2  filter: closed-form periodic Ram-Lak kernel; cosine eigenfunctions;
    the padded/cropped impulse response written as a plain cosine sum.
P3  direct backprojection: the phi = 0 reduction to per-slice 2D parallel-beam
    backprojection (a separately written textbook loop); the bilinear
    footprint of a single detector pixel; exact 90-degree rotation symmetry.
P4  adjoint identities <L mu, q> (pi/Ntheta) = <mu, L* q> for both forms.
P5  the four-loop Fourier sum equals the separable one; the Fourier form
    equals the direct form exactly where all nodes are integers and the data
    carry no Nyquist component.
P5b the spatial (periodic-kernel) evaluation of the Fourier form equals the
    DFT evaluation, and its kernel equals the Nyquist-free exponential sum it
    closes (a plain Python sum).
P7  FBP scale: at phi = 0 FBP reproduces an analytic Gaussian phantom, at
    phi = 40 deg it reproduces the missing-cone-filtered phantom.
P8  brute force on 8^3 inputs written as plain Python loops.
"""
import math

import numpy as np
import pytest

from oracle import lamino_oracle as O
from paper_2401_11101_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# ---------------------------------------------------------------- sizes

def test_fft_size_rule():
    assert [O.fft_size(n) for n in (1, 2, 3, 5, 7, 13, 17, 25, 97, 193)] == \
        [1, 2, 3, 6, 8, 16, 24, 32, 128, 256]


@pytest.mark.parametrize("name,expect", [
    ("c1", dict(Wp=192, Wf=96, Hf=96)),
    ("c2", dict(Wp=1536, Wf=768, Hf=512)),
    ("c3", dict(Wp=4096, Wf=3072, Hf=1536)),
    ("c4", dict(Wp=768, Wf=384, Hf=384)),
])
def test_padded_sizes_of_workloads(name, expect):
    assert O.padded_sizes(I.CONFIGS[name]["geom"]) == expect


# ---------------------------------------------------------------- P2 filter

def test_ramp_filter_impulse_is_periodic_ramlak():
    # IDFT of |m/N| on N points: 1/4 at 0, -1/(N^2 sin^2(pi n/N)) at odd n, 0 at
    # even n (sum of an arithmetic triangle wave). Times cos(phi) for the tilt.
    geom = I.Geometry(8, 8, 8, 1, 1, 96, math.radians(30.0))
    Wp = O.padded_sizes(geom)["Wp"]
    j0 = 40
    d = np.zeros((1, 1, 96))
    d[0, 0, j0] = 1.0
    q = O.filter_rows(d, geom, "ramp")[0, 0]
    n = (np.arange(96) - j0) % Wp
    with np.errstate(divide="ignore"):
        h = np.where(n % 2 == 1, -1.0 / (Wp * Wp * np.sin(np.pi * n / Wp) ** 2), 0.0)
    h[n == 0] = 0.25
    assert np.abs(q - math.cos(geom.tilt) * h).max() < 1e-14


@pytest.mark.parametrize("kind", O.FILTERS)
def test_filter_cosines_are_eigenfunctions(kind):
    # on a full periodic row the filter multiplies cos(2 pi m0 j/N) by H(m0/N)
    N, tilt = 192, 0.4
    Hr = O.filter_response(N, tilt, kind)
    j = np.arange(N)
    for m0 in (0, 1, 5, 37, 95, 96):
        x = np.cos(2 * np.pi * m0 * j / N)
        y = np.real(np.fft.ifft(np.fft.fft(x) * Hr))
        f = m0 / N
        lam = abs(f) * math.cos(tilt) * O.filter_window(np.array([f]), kind)[0]
        assert np.abs(y - lam * x).max() < 1e-12


@pytest.mark.parametrize("kind", O.FILTERS)
def test_filter_impulse_response_as_cosine_sum(kind):
    # padded-and-cropped filtering of a delta at j0 gives h[(j - j0) mod Wp] with
    # h[n] = (1/Wp) sum_m H(m/Wp) cos(2 pi m n / Wp) (H is real and even).
    geom = I.Geometry(8, 8, 8, 1, 1, 50, math.radians(15.0))
    Wp = O.padded_sizes(geom)["Wp"]
    assert Wp == 128
    m = np.arange(Wp)
    f = np.where(m < Wp // 2, m, m - Wp) / Wp
    H = np.abs(f) * math.cos(geom.tilt) * O.filter_window(f, kind)
    for j0 in (0, 7, 49):
        d = np.zeros((1, 1, 50))
        d[0, 0, j0] = 1.0
        q = O.filter_rows(d, geom, kind)[0, 0]
        for jj in range(50):
            n = (jj - j0) % Wp
            h = float(np.sum(H * np.cos(2 * np.pi * m * n / Wp))) / Wp
            assert abs(q[jj] - h) < 1e-14


def test_filter_windows_known_values():
    f = np.array([0.0, 0.25, 0.5])
    assert np.allclose(O.filter_window(f, "shepp"), [1.0, math.sin(math.pi / 4) / (math.pi / 4),
                                                   2 / math.pi], atol=1e-15)
    # Parzen: 1 - 6 z^2 + 6 z^3 up to z = 1/2, 2 (1-z)^3 beyond (z = f / 0.5)
    assert np.allclose(O.filter_window(np.array([0.0, 0.125, 0.25, 0.375, 0.5]), "parzen"),
                       [1.0, 1 - 6 / 16 + 6 / 64, 0.25, 2 / 64, 0.0], atol=1e-15)


# ---------------------------------------------------------------- P3 direct

def _textbook_parallel_bp(sino, theta, n, W):
    """2D parallel-beam backprojection of one slice, linear interpolation of
    each sinogram row at s = x.theta (standard tomography textbook loop)."""
    out = np.zeros((n, n))
    xs = np.arange(n) - n / 2.0
    X2, X1 = np.meshgrid(xs, xs, indexing="ij")
    for k, t in enumerate(theta):
        s = X1 * math.cos(t) + X2 * math.sin(t) + W / 2.0
        out += np.interp(s, np.arange(W), sino[k], left=0.0, right=0.0)
    return out * math.pi / len(theta)


def test_direct_reduces_to_2d_parallel_beam_at_phi0():
    n, nproj, W = 16, 12, 30          # W > 2*u_max + 2: nothing reaches the detector edge
    geom = I.Geometry(n, n, 6, nproj, 6, W, 0.0)
    q = I.random_projections(geom, seed=3)
    q[:, :, 0] = 0.0
    q[:, :, -1] = 0.0
    vol = O.backproject_direct(q, geom)
    for z in range(6):
        ref = _textbook_parallel_bp(q[:, z, :], geom.angles, n, W)
        assert np.abs(vol[z] - ref).max() < 1e-13


def test_direct_single_pixel_footprint():
    geom = I.Geometry(12, 10, 8, 5, 9, 14, math.radians(25.0))
    q = np.zeros((geom.nproj, geom.det_h, geom.det_w))
    k0, r0, j0 = 2, 4, 6
    q[k0, r0, j0] = 1.0
    vol = O.backproject_direct(q, geom)
    a, b, _ = I.geometry_vectors(geom.angles, geom.tilt)
    x3, x2, x1 = np.meshgrid(np.arange(8) - 4.0, np.arange(10) - 5.0, np.arange(12) - 6.0,
                             indexing="ij")
    j = a[k0, 0] * x1 + a[k0, 1] * x2 + geom.det_w / 2.0
    r = b[k0, 0] * x1 + b[k0, 1] * x2 + b[k0, 2] * x3 + geom.det_h / 2.0
    hat = lambda t: np.clip(1.0 - np.abs(t), 0.0, None)
    ref = math.pi / geom.nproj * hat(j - j0) * hat(r - r0)
    assert np.abs(vol - ref).max() < 1e-15


def test_direct_rotation_by_quarter_turn():
    # shifting the angle index by N/4 rotates the reconstruction by 90 degrees
    # about x3: vol'(x1, x2, x3) = vol(-x2, x1, x3) (interior of the grid).
    n = 12
    geom = I.Geometry(n, n, 6, 16, 10, 22, math.radians(20.0))
    q = I.random_projections(geom, seed=4)
    v = O.backproject_direct(q, geom)
    v2 = O.backproject_direct(np.roll(q, -geom.nproj // 4, axis=0), geom)
    # index of x = (i - n/2): -x2 -> i0 = n - i1
    for i1 in range(1, n):
        for i0 in range(1, n):
            assert np.abs(v2[:, i1, i0] - v[:, i0, n - i1]).max() < 1e-12


# ---------------------------------------------------------------- P4 adjoint

@pytest.mark.parametrize("n,nproj,tilt", [(8, 8, 20.0), (16, 12, 35.0), (8, 6, 0.0)])
def test_adjoint_identity_direct(n, nproj, tilt):
    geom = I.Geometry(n, n, n // 2 + 2, nproj, n, n + 6, math.radians(tilt))
    mu = I.random_volume(geom, seed=5)
    q = I.random_projections(geom, seed=6)
    lhs = np.vdot(O.project_direct(mu, geom), q) * math.pi / nproj
    rhs = np.vdot(mu, O.backproject_direct(q, geom))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


@pytest.mark.parametrize("n,nproj,tilt", [(8, 8, 20.0), (6, 5, 0.0)])
def test_adjoint_identity_fourier(n, nproj, tilt):
    geom = I.Geometry(n, n, 4, nproj, 6, 10, math.radians(tilt))
    mu = I.random_volume(geom, seed=7)
    q = I.random_projections(geom, seed=8)
    lhs = np.vdot(O.project_fourier(mu, geom), q) * math.pi / nproj
    rhs = np.vdot(mu, O.backproject_fourier(q, geom))
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


# ---------------------------------------------------------------- P5 Fourier

def test_fourier_separable_equals_four_loops():
    geom = I.Geometry(8, 8, 8, 8, 8, 12, math.radians(20.0))
    q = I.random_projections(geom, seed=9)
    a = O.backproject_fourier(q, geom)
    b = O.backproject_fourier_full4(q, geom)
    assert rel(a, b) < 1e-12


def test_fourier_equals_direct_on_integer_nodes():
    # phi = 0 and theta in {0, 90, 180, 270} deg: every node (a.x + W/2, b.x + H/2)
    # is an integer pixel. With no padding (Wf = W, Hf = H) and data whose DFT has
    # no Nyquist component, trigonometric interpolation returns the samples, as
    # does bilinear interpolation: both forms must agree to rounding.
    n = 8
    geom = I.Geometry(n, n, 8, 4, 16, 16, 0.0)
    s = O.padded_sizes(geom)
    assert (s["Wf"], s["Hf"]) == (16, 16)
    rng = np.random.default_rng(10)
    q = np.empty((4, 16, 16))
    for k in range(4):
        F = np.fft.fft2(rng.standard_normal((16, 16)))
        F[8, :] = 0
        F[:, 8] = 0
        q[k] = np.real(np.fft.ifft2(F))
    a = O.backproject_fourier(q, geom)
    b = O.backproject_direct(q, geom)
    assert rel(a, b) < 1e-13


def test_fourier_close_to_direct_on_smooth_data():
    # both forms discretise Eq. adj; on a band-limited phantom they agree to the
    # interpolation error of bilinear sampling (about 1e-2)
    geom = I.Geometry(24, 24, 16, 32, 32, 48, math.radians(20.0))
    p = I.blob_params(geom, 4, seed=12, sigma=(4.0, 5.0))
    q = O.filter_rows(I.project(p, geom).numpy(), geom, "shepp")
    assert rel(O.backproject_fourier(q, geom), O.backproject_direct(q, geom)) < 2e-2


def test_fourier_columns_match_full_volume():
    geom = I.Geometry(8, 6, 4, 5, 6, 10, math.radians(20.0))
    q = I.random_projections(geom, seed=13)
    full = O.backproject_fourier(q, geom)
    cols = np.array([[0, 0], [7, 5], [3, 2]], dtype=np.int32)
    part = O.backproject_fourier_columns(q, geom, cols)
    for c, (i0, i1) in enumerate(cols):
        assert np.abs(part[c] - full[:, i1, i0]).max() < 1e-14
    dcol = O.backproject_direct_columns(q, geom, cols)
    dfull = O.backproject_direct(q, geom)
    for c, (i0, i1) in enumerate(cols):
        assert np.abs(dcol[c] - dfull[:, i1, i0]).max() < 1e-15


def test_periodic_kernel_route_equals_dft_route():
    # two independent evaluations of the type-1 sum of Eq. fftadj: the 2D DFT
    # of every padded projection (numpy FFT) followed by the separable sum, and
    # the closed-form geometric series in detector space (no spectra)
    for g in (I.Geometry(8, 8, 8, 8, 8, 12, math.radians(20.0)),
              I.Geometry(24, 40, 12, 10, 14, 40, math.radians(33.0)),
              I.Geometry(16, 24, 8, 9, 11, 23, math.radians(-25.0)),
              I.Geometry(16, 16, 8, 12, 10, 26, 0.0)):
        q = I.random_projections(g, 41)
        cols = O.all_columns(g)
        a = O.backproject_fourier_columns(q, g, cols)
        b = O.backproject_trig_columns(q, g, cols)
        assert rel(b, a) <= 1e-12
        idx = np.array([0, 2, 5])
        a = O.backproject_fourier_columns(q[idx], g, cols[::3], angle_index=idx)
        b = O.backproject_trig_columns(q[idx], g, cols[::3], angle_index=idx)
        assert rel(b, a) <= 1e-12


def test_periodic_kernel_is_the_exponential_sum():
    # one detector pixel of value 1 at (r0, j0): the spatial route returns
    # (pi/Ntheta) K_Wf(u + W/2 - j0) K_Hf(v + H/2 - r0), K_N(t) written here as
    # the plain sum over m in (-N/2, N/2) of exp(2 pi i m t/N)/N
    g = I.Geometry(8, 8, 4, 1, 6, 10, math.radians(30.0))
    s = O.padded_sizes(g)
    q = np.zeros((1, g.det_h, g.det_w))
    r0, j0 = 2, 7
    q[0, r0, j0] = 1.0
    cols = np.array([[1, 6], [5, 2]], dtype=np.int32)
    out = O.backproject_trig_columns(q, g, cols)

    def K(t, N):
        m = np.arange(-N // 2 + 1, N // 2)
        return float(np.real(np.exp(2j * np.pi * m * t / N).sum())) / N

    sp, cp = math.sin(g.tilt), math.cos(g.tilt)
    for c, (i0, i1) in enumerate(cols):
        x1, x2 = i0 - g.n0 / 2, i1 - g.n1 / 2
        for i2 in range(g.n2):
            x3 = i2 - g.n2 / 2
            u = x1                              # theta = 0: a = (1, 0, 0)
            v = -x2 * sp + x3 * cp              # b = (0, -sin phi, cos phi)
            ref = math.pi * K(u + g.det_w / 2 - j0, s["Wf"]) * K(v + g.det_h / 2 - r0, s["Hf"])
            assert abs(out[c, i2] - ref) <= 1e-12


def test_angle_subset_is_the_zeroed_full_sum():
    # backprojection is a sum over angles: a subset of projections gives the
    # same result as the full set with the other projections zeroed
    geom = I.Geometry(12, 10, 6, 9, 8, 20, math.radians(25.0))
    q = I.random_projections(geom, 16)
    idx = np.array([1, 4, 8])
    qz = np.zeros_like(q)
    qz[idx] = q[idx]
    cols = np.array([[0, 0], [5, 7], [11, 9]], dtype=np.int32)
    for fn in (O.backproject_direct_columns, O.backproject_fourier_columns):
        full = fn(qz, geom, cols)
        sub = fn(q[idx], geom, cols, angle_index=idx)
        assert np.abs(full - sub).max() <= 1e-12 * np.abs(full).max()


# ---------------------------------------------------------------- P7 scale

def _blob_case(tilt_deg):
    geom = I.Geometry(32, 32, 32, 128, 96, 96, math.radians(tilt_deg))
    p = I.blob_params(geom, 3, 5, sigma=(3.0, 4.0), amp=(0.5, 1.0))
    p["centre"] *= 0.5
    return geom, p, I.project(p, geom).numpy()


def test_fbp_reproduces_phantom_in_tomography_limit():
    geom, p, d = _blob_case(0.0)
    truth = I.rasterize_blobs(p, geom)
    rec = O.fbp_direct(d, geom, "ramp")
    assert rel(rec, truth) < 0.02
    assert abs(np.vdot(rec, truth) / np.vdot(truth, truth) - 1) < 0.015


def test_fbp_matches_missing_cone_reference():
    # at phi = 40 deg a wrong cos(phi) factor would be off by 30 %
    geom, p, d = _blob_case(40.0)
    truth = I.rasterize_blobs(p, geom)
    ref = O.missing_cone_reference(truth, geom.tilt, pad=4)
    rec = O.fbp_direct(d, geom, "ramp")
    assert rel(rec, ref) < 0.03
    assert abs(np.vdot(rec, ref) / np.vdot(ref, ref) - 1) < 0.02
    assert rel(rec, truth) > 0.2          # the cone really is missing


# ---------------------------------------------------------------- P8 brute force

def test_direct_brute_force_python_loops():
    geom = I.Geometry(8, 8, 8, 6, 8, 12, math.radians(20.0))
    q = I.random_projections(geom, seed=14)
    vol = O.backproject_direct(q, geom)
    sp, cp = math.sin(geom.tilt), math.cos(geom.tilt)
    H, W = geom.det_h, geom.det_w

    def px(k, r, j):
        return q[k, r, j] if (0 <= r < H and 0 <= j < W) else 0.0

    for i2 in range(8):
        for i1 in range(8):
            for i0 in range(8):
                x1, x2, x3 = i0 - 4.0, i1 - 4.0, i2 - 4.0
                acc = 0.0
                for k in range(geom.nproj):
                    t = 2 * math.pi * k / geom.nproj
                    j = x1 * math.cos(t) + x2 * math.sin(t) + W / 2
                    r = x1 * math.sin(t) * sp - x2 * math.cos(t) * sp + x3 * cp + H / 2
                    j0, r0 = math.floor(j), math.floor(r)
                    fj, fr = j - j0, r - r0
                    acc += ((1 - fj) * (1 - fr) * px(k, r0, j0) + fj * (1 - fr) * px(k, r0, j0 + 1)
                            + (1 - fj) * fr * px(k, r0 + 1, j0) + fj * fr * px(k, r0 + 1, j0 + 1))
                assert abs(vol[i2, i1, i0] - acc * math.pi / geom.nproj) < 1e-13


def test_fourier_brute_force_python_loops():
    # the type-1 sum over every (k, m, l) for a handful of voxels, in Python
    geom = I.Geometry(6, 6, 4, 3, 6, 8, math.radians(20.0))
    q = I.random_projections(geom, seed=15)
    vol = O.backproject_fourier(q, geom)
    s = O.padded_sizes(geom)
    Wf, Hf = s["Wf"], s["Hf"]
    offu, offv = (Wf - 8) // 2, (Hf - 6) // 2
    sp, cp = math.sin(geom.tilt), math.cos(geom.tilt)
    for (i0, i1, i2) in [(0, 0, 0), (5, 2, 3), (3, 3, 1)]:
        x1, x2, x3 = i0 - 3.0, i1 - 3.0, i2 - 2.0
        acc = 0.0
        for k in range(geom.nproj):
            t = 2 * math.pi * k / geom.nproj
            pad = np.zeros((Hf, Wf))
            pad[offv:offv + 6, offu:offu + 8] = q[k]
            jp = x1 * math.cos(t) + x2 * math.sin(t) + 4 + offu
            rp = x1 * math.sin(t) * sp - x2 * math.cos(t) * sp + x3 * cp + 3 + offv
            for l in range(-Hf // 2 + 1, Hf // 2):
                for m in range(-Wf // 2 + 1, Wf // 2):
                    D = 0j
                    for r in range(Hf):
                        for j in range(Wf):
                            if pad[r, j] != 0.0:
                                D += pad[r, j] * complex(math.cos(-2 * math.pi * (m * j / Wf + l * r / Hf)),
                                                         math.sin(-2 * math.pi * (m * j / Wf + l * r / Hf)))
                    ang = 2 * math.pi * (m * jp / Wf + l * rp / Hf)
                    acc += (D * complex(math.cos(ang), math.sin(ang))).real
        ref = acc * (math.pi / geom.nproj) / (Wf * Hf)
        assert abs(vol[i2, i1, i0] - ref) < 1e-12 * max(1.0, abs(ref))
