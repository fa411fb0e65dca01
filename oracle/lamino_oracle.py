"""FP64 CPU oracle for laminographic filtered backprojection.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in ``oracle/``;
the product path never does. Plain and slow on purpose: numpy's FFT is used as
a library primitive for the DFT steps, and a small C library (``lamino_oracle.c``,
built by ``oracle/build.py``) holds the plain loops. Nothing here shares code
with the CUDA path.

Every function cites the passage of Nikitin et al., "Laminography as a tool for
imaging large-size samples with high resolution" (arXiv 2401.11101) it follows.
Readings of points the paper leaves open (the same ones the CUDA path uses):

* tilt phi is measured away from tomography: the formulas of Sec. 4 give the
  Radon transform at phi = 0 (the sentence about the rotation axis and the
  beam contradicts them; the formulas win);
* voxel = pixel = 1; x = i - n/2; u = j - W/2; v = r - H/2; theta_k = 2 pi k/N;
* filter (Sec. 4, after Eq. adj): rows zero-padded on the right to Wp (the
  smallest 2^k or 3*2^k >= 2W), multiplied in frequency by
  H(f) = |f| cos(phi) w(f), f = m/Wp in [-1/2, 1/2), cropped back to W;
  w = 1 (ramp), sin(pi f)/(pi f) (Shepp-Logan), Parzen with cutoff 1/2;
* direct backprojection (Eq. adj): (pi/Ntheta) sum_k bilinear(q_k), zero
  outside the detector;
* Fourier form (Eq. fftadj, Eq. uneqspace): the exact type-1 sum over all
  (m, l) of the 2D DFT of the zero-padded projection, Nyquist bins zeroed,
  i.e. trigonometric interpolation of each padded projection at (a.x, b.x).
  The USFFT of the CUDA path is a fast approximation of exactly this sum;
* padded Fourier detector: Wf >= max(W, 2 u_max + 2), Hf >= max(H, 2 v_max + 2)
  rounded up to 2^k or 3*2^k, u_max = |(n0, n1)|/2, v_max = u_max |sin phi| +
  n2 cos(phi)/2; the projection sits at offset ((Wf-W)//2, (Hf-H)//2).

Parity of the oracle is pinned by tests/test_oracle_pins.py (closed forms,
the phi = 0 reduction to 2D parallel-beam backprojection, adjoint identities,
the missing-cone reference, brute force on 8^3 inputs).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
from scipy import fft as _sfft

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        lib.orc_num_threads.restype = c_int
        lib.orc_set_num_threads.argtypes = [c_int]
        lib.orc_bp_direct.argtypes = [D, c_int, c_int, c_int, D, c_double, c_int, c_int,
                                      c_int, c_int, c_int, D]
        lib.orc_bp_direct_columns.argtypes = [D, c_int, c_int, c_int, D, c_double, c_int,
                                              c_int, c_int, I, c_int, D]
        lib.orc_splat.argtypes = [D, c_int, c_int, c_int, c_int, c_int, c_int, D, c_double, D]
        lib.orc_bp_fourier_columns.argtypes = [D, D, c_int, c_int, c_int, c_double, c_double,
                                               D, c_double, c_int, c_int, c_int, I, c_int,
                                               c_double, D]
        lib.orc_bp_fourier_full4.argtypes = [D, D, c_int, c_int, c_int, c_double, c_double, D,
                                             c_double, c_int, c_int, c_int, c_double, D]
        lib.orc_bp_trig_columns.argtypes = [D, c_int, c_int, c_int, D, c_double, c_int, c_int,
                                            c_int, c_int, c_int, I, c_int, c_double, D]
        lib.orc_fourier_adjoint_coeffs.argtypes = [D, c_int, c_int, c_int, c_int, c_int, c_int,
                                                   c_double, c_double, D, c_double, D, D]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    """OpenMP threads the C loops use."""
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the C loops and of the row filter's FFTs from now on."""
    global _workers
    _load().orc_set_num_threads(int(n))
    _workers = int(n)


_workers = os.cpu_count() or 1


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _theta(geom, angle_index=None) -> np.ndarray:
    idx = np.arange(geom.nproj) if angle_index is None else np.asarray(angle_index)
    return np.ascontiguousarray(2.0 * np.pi * idx.astype(np.float64) / geom.nproj)


# ----------------------------------------------------------------------------
# sizes
# ----------------------------------------------------------------------------

def fft_size(n: float) -> int:
    """Smallest integer of the form 2^k or 3*2^k that is >= n."""
    best = None
    p = 1
    while p <= 4 * max(1.0, n) + 4:
        for c in (p, 3 * p):
            if c >= n and (best is None or c < best):
                best = c
        p *= 2
    return int(best)


def padded_sizes(geom) -> dict:
    """Filter length Wp and Fourier detector grid Wf x Hf (plan rule above)."""
    W, H = geom.det_w, geom.det_h
    umax = 0.5 * math.hypot(geom.n0, geom.n1)
    vmax = umax * abs(math.sin(geom.tilt)) + 0.5 * geom.n2 * math.cos(geom.tilt)
    Wp = fft_size(2 * W)
    Wf = fft_size(max(W, 2.0 * umax + 2.0))
    Hf = fft_size(max(H, 2.0 * vmax + 2.0))
    return dict(Wp=Wp, Wf=Wf, Hf=Hf)


# ----------------------------------------------------------------------------
# filter W (Sec. 4, after Eq. adj)
# ----------------------------------------------------------------------------

FILTERS = ("ramp", "shepp", "parzen")


def filter_window(f: np.ndarray, kind: str) -> np.ndarray:
    """Low-pass window w(f) on top of the ramp; f in cycles per pixel."""
    af = np.abs(f)
    if kind == "ramp":
        return np.ones_like(f)
    if kind == "shepp":
        return np.sinc(f)  # sin(pi f)/(pi f)
    if kind == "parzen":
        z = af / 0.5
        return np.where(z <= 0.5, 1 - 6 * z ** 2 + 6 * z ** 3,
                        np.where(z <= 1.0, 2 * (1 - z) ** 3, 0.0))
    raise ValueError(kind)


def filter_response(Wp: int, tilt: float, kind: str) -> np.ndarray:
    """H(f) = |f| cos(phi) w(f) at the Wp DFT frequencies (numpy FFT order).

    Sec. 4: the transfer function of W is a scaled |sigma| cos(phi); with unit
    pixels and the rectangle rule over theta the scale is 1 (the pi/Ntheta of
    the backprojection carries the rest).
    """
    f = np.fft.fftfreq(Wp)
    return np.abs(f) * math.cos(tilt) * filter_window(f, kind)


def filter_rows(d, geom, kind: str = "ramp") -> np.ndarray:
    """Apply W along detector rows: pad to Wp, DFT, x H(f), inverse DFT, crop.

    The rows are real and H(f) is real and even, so the half spectrum of a
    real-input FFT (scipy.fft on all host threads; the Nyquist bin at
    f = +1/2 carries H(1/2) = H(-1/2)) gives the same filtered rows."""
    d = _f64(d)
    W = d.shape[-1]
    Wp = padded_sizes(geom)["Wp"]
    Hf = filter_response(Wp, geom.tilt, kind)[: Wp // 2 + 1]
    Hf[-1] = filter_response(Wp, geom.tilt, kind)[Wp // 2]
    workers = _workers
    spec = _sfft.rfft(d, n=Wp, axis=-1, workers=workers)
    spec *= Hf
    return np.ascontiguousarray(_sfft.irfft(spec, n=Wp, axis=-1, workers=workers)[..., :W])


# ----------------------------------------------------------------------------
# direct form (Eq. adj with linear interpolation)
# ----------------------------------------------------------------------------

def backproject_direct(q, geom, z0: int = 0, z1: int | None = None) -> np.ndarray:
    """(pi/Ntheta) sum_k bilinear(q_k; a_k.x + W/2, b_k.x + H/2) on slices [z0, z1)."""
    q = _f64(q)
    z1 = geom.n2 if z1 is None else z1
    out = np.zeros((z1 - z0, geom.n1, geom.n0))
    _load().orc_bp_direct(_dp(q), geom.nproj, geom.det_h, geom.det_w, _dp(_theta(geom)),
                          float(geom.tilt), geom.n0, geom.n1, geom.n2, z0, z1, _dp(out))
    return out


def backproject_direct_columns(q, geom, cols, angle_index=None) -> np.ndarray:
    """Direct backprojection on whole columns cols[c] = (i0, i1): out [ncol, n2].

    With angle_index, q holds only the projections with those indices of the
    equispaced set of geom.nproj angles and the result is their contribution
    (weight pi/geom.nproj): the backprojection is a sum over angles."""
    q = _f64(q)
    nq = q.shape[0]
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((cols.shape[0], geom.n2))
    _load().orc_bp_direct_columns(_dp(q), nq, geom.det_h, geom.det_w,
                                  _dp(_theta(geom, angle_index)), float(geom.tilt), geom.n0,
                                  geom.n1, geom.n2, _ip(cols), cols.shape[0], _dp(out))
    return out * (nq / geom.nproj)


def project_direct(vol, geom) -> np.ndarray:
    """Exact transpose of the bilinear backprojection sum (no pi/Ntheta)."""
    vol = _f64(vol)
    d = np.zeros((geom.nproj, geom.det_h, geom.det_w))
    _load().orc_splat(_dp(vol), geom.n0, geom.n1, geom.n2, geom.nproj, geom.det_h,
                      geom.det_w, _dp(_theta(geom)), float(geom.tilt), _dp(d))
    return d


# ----------------------------------------------------------------------------
# Fourier form (Eq. fftadj with the grid of Eq. uneqspace), exact definition
# ----------------------------------------------------------------------------

def _fourier_frame(geom):
    s = padded_sizes(geom)
    Wf, Hf = s["Wf"], s["Hf"]
    offu = (Wf - geom.det_w) // 2
    offv = (Hf - geom.det_h) // 2
    joff = geom.det_w / 2.0 + offu   # j' = a.x + joff
    roff = geom.det_h / 2.0 + offv   # r' = b.x + roff
    return Wf, Hf, offu, offv, joff, roff


def fourier_spectra(q, geom):
    """2D DFT of every zero-padded projection with the Nyquist row and column
    zeroed (the F_2D of Eq. fftadj). Returns D [len(q), Hf, Wf] complex128."""
    q = _f64(q)
    Wf, Hf, offu, offv, _, _ = _fourier_frame(geom)
    pad = np.zeros((q.shape[0], Hf, Wf))
    pad[:, offv:offv + geom.det_h, offu:offu + geom.det_w] = q
    D = np.fft.fft2(pad, axes=(1, 2))
    D[:, Hf // 2, :] = 0.0
    D[:, :, Wf // 2] = 0.0
    return D


def _fourier_scale(geom, Wf, Hf):
    return (math.pi / geom.nproj) / (Wf * Hf)


def backproject_fourier_columns(q, geom, cols, angle_index=None) -> np.ndarray:
    """Fourier-form backprojection (exact type-1 sum) on columns: out [ncol, n2].
    angle_index as for backproject_direct_columns."""
    Wf, Hf, _, _, joff, roff = _fourier_frame(geom)
    D = fourier_spectra(q, geom)
    Dre = np.ascontiguousarray(D.real)
    Dim = np.ascontiguousarray(D.imag)
    del D
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((cols.shape[0], geom.n2))
    _load().orc_bp_fourier_columns(_dp(Dre), _dp(Dim), Dre.shape[0], Hf, Wf, joff, roff,
                                   _dp(_theta(geom, angle_index)), float(geom.tilt), geom.n0,
                                   geom.n1, geom.n2, _ip(cols), cols.shape[0],
                                   _fourier_scale(geom, Wf, Hf), _dp(out))
    return out


def backproject_trig_columns(q, geom, cols, angle_index=None) -> np.ndarray:
    """The same sum as backproject_fourier_columns, evaluated in detector space:
    (pi/Ntheta) sum_k sum_{r,j} q_k(r, j) K_Wf(a_k.x + W/2 - j) K_Hf(b_k.x + H/2 - r)
    with the periodic kernel K_N(t) = (1/N) sum over |m| < N/2 of exp(2 pi i m t/N)
    (the geometric series of the type-1 sum of Eq. fftadj over the Nyquist-free
    frequencies, summed in closed form). Needs no padded spectra, so it serves
    paper-size projections; angle_index as for backproject_direct_columns.
    Columns cols[c] = (i0, i1); returns [ncol, n2]."""
    q = _f64(q)
    Wf, Hf, _, _, _, _ = _fourier_frame(geom)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((cols.shape[0], geom.n2))
    _load().orc_bp_trig_columns(_dp(q), q.shape[0], geom.det_h, geom.det_w,
                                _dp(_theta(geom, angle_index)), float(geom.tilt), Wf, Hf,
                                geom.n0, geom.n1, geom.n2, _ip(cols), cols.shape[0],
                                math.pi / geom.nproj, _dp(out))
    return out


def all_columns(geom) -> np.ndarray:
    i1, i0 = np.meshgrid(np.arange(geom.n1), np.arange(geom.n0), indexing="ij")
    return np.stack([i0.ravel(), i1.ravel()], axis=1).astype(np.int32)


def backproject_fourier(q, geom) -> np.ndarray:
    """Fourier-form backprojection of the whole volume: [n2, n1, n0]."""
    cols = all_columns(geom)
    out = backproject_fourier_columns(q, geom, cols)       # [n1*n0, n2]
    return np.ascontiguousarray(out.T.reshape(geom.n2, geom.n1, geom.n0))


def backproject_fourier_full4(q, geom) -> np.ndarray:
    """The same sum with four plain loops per voxel (tiny volumes only)."""
    Wf, Hf, _, _, joff, roff = _fourier_frame(geom)
    D = fourier_spectra(q, geom)
    Dre = np.ascontiguousarray(D.real)
    Dim = np.ascontiguousarray(D.imag)
    out = np.zeros((geom.n2, geom.n1, geom.n0))
    _load().orc_bp_fourier_full4(_dp(Dre), _dp(Dim), geom.nproj, Hf, Wf, joff, roff,
                                 _dp(_theta(geom)), float(geom.tilt), geom.n0, geom.n1,
                                 geom.n2, _fourier_scale(geom, Wf, Hf), _dp(out))
    return out


def project_fourier(vol, geom) -> np.ndarray:
    """Exact transpose of backproject_fourier divided by pi/Ntheta (the Fourier
    form of the forward operator, Eq. fftfwd): detector data [nproj, H, W]."""
    vol = _f64(vol)
    Wf, Hf, offu, offv, joff, roff = _fourier_frame(geom)
    Are = np.zeros((geom.nproj, Hf, Wf))
    Aim = np.zeros((geom.nproj, Hf, Wf))
    _load().orc_fourier_adjoint_coeffs(_dp(vol), geom.n0, geom.n1, geom.n2, geom.nproj, Hf,
                                       Wf, joff, roff, _dp(_theta(geom)), float(geom.tilt),
                                       _dp(Are), _dp(Aim))
    A = Are + 1j * Aim
    A[:, Hf // 2, :] = 0.0
    A[:, :, Wf // 2] = 0.0
    P = np.real(np.fft.fft2(A, axes=(1, 2))) / (Wf * Hf)
    return np.ascontiguousarray(P[:, offv:offv + geom.det_h, offu:offu + geom.det_w])


# ----------------------------------------------------------------------------
# FBP (Eq. recon) and the missing-cone reference (Sec. 4, Fig. undersampling)
# ----------------------------------------------------------------------------

def fbp_direct(d, geom, kind: str = "ramp") -> np.ndarray:
    return backproject_direct(filter_rows(d, geom, kind), geom)


def fbp_fourier(d, geom, kind: str = "ramp") -> np.ndarray:
    return backproject_fourier(filter_rows(d, geom, kind), geom)


def missing_cone_reference(vol: np.ndarray, tilt: float, pad: int = 2) -> np.ndarray:
    """What full-circle laminographic FBP recovers of a volume: its 3D spectrum
    restricted to |xi3| tan(phi) <= |(xi1, xi2)| (the sampled region of
    Eq. uneqspace; outside it lies the missing cone of Fig. undersampling).
    Computed on a `pad`-times zero-padded grid; returns [n2, n1, n0]."""
    vol = _f64(vol)
    n2, n1, n0 = vol.shape
    big = np.zeros((pad * n2, pad * n1, pad * n0))
    big[:n2, :n1, :n0] = vol
    F = np.fft.fftn(big)
    k3 = np.fft.fftfreq(pad * n2)[:, None, None]
    k2 = np.fft.fftfreq(pad * n1)[None, :, None]
    k1 = np.fft.fftfreq(pad * n0)[None, None, :]
    mask = np.abs(k3) * math.tan(tilt) <= np.sqrt(k1 ** 2 + k2 ** 2)
    return np.real(np.fft.ifftn(F * mask))[:n2, :n1, :n0]
