"""Paper-scale slab (2048x2048x512, 1800 angles, detector 512x2048, tilt 18 deg,
Sec. 5 Table perf scale) with projections stored in FP16 or BF16 and all
arithmetic in FP32, on the full data.

The exact Fourier-form oracle through padded spectra would need about 136 GB
here, so the oracle evaluates the same sum in detector space
(backproject_trig_columns: periodic-kernel interpolation, pinned against the
spectral evaluation) and, since backprojection is a sum over angles, in chunks
of 60 projections (filter, then both forms' contributions on whole sampled
columns). The GPU reconstructs the full data with the Fourier form z-chunked
in 64 k_v planes (Sec. 5 chunking) and with the direct form in 64-slice
launches; both are compared with the oracle on the same columns. This puts
the fixed-point gridding under the band loads of the real data.
"""
import math
import time

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


@pytest.fixture(scope="module")
def c3_data():
    t0 = time.time()
    g, prm, d = I.make_projections("c3", device="cuda")
    print(f"c3 inputs generated in {time.time() - t0:.1f} s")
    return g, prm, d


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _columns(g, n, seed):
    rng = np.random.default_rng(seed)
    # half inside the central disc where most ellipsoids overlap, half anywhere
    c = rng.integers(0, g.n0, (n, 2))
    c[: n // 2] = g.n0 // 2 + rng.integers(-g.n0 // 4, g.n0 // 4, (n // 2, 2))
    return c.astype(np.int32)


def _oracle_columns(d_stored, g, cols, chunk=60):
    """Both forms' FP64 FBP on whole columns, summed over chunks of angles."""
    of = np.zeros((len(cols), g.n2))
    od = np.zeros((len(cols), g.n2))
    for k0 in range(0, g.nproj, chunk):
        idx = np.arange(k0, min(g.nproj, k0 + chunk))
        q = O.filter_rows(d_stored[k0:k0 + len(idx)].float().cpu().numpy(), g, "shepp")
        of += O.backproject_trig_columns(q, g, cols, angle_index=idx)
        od += O.backproject_direct_columns(q, g, cols, angle_index=idx)
    return of, od


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_c3_full_data_parity(L, c3_data, dtype):
    g, _, d = c3_data
    ds = d.to(dtype)
    cols = _columns(g, 6, 77 if dtype == torch.float16 else 78)
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt, z_chunk=64) as p:
        print(f"Fourier workspace, z_chunk=64: {p.workspace_bytes('fourier') / 2**30:.1f} GiB "
              f"({p.info['planes']} planes in chunks of {p.info['plane_chunk']})")
        out = {}
        for form in ("fourier", "direct"):
            v = p.fbp(ds, form=form, kind="shepp")
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            p.fbp(ds, form=form, kind="shepp", out=v)
            b.record()
            b.synchronize()
            p.status()
            ms = a.elapsed_time(b)
            print(f"c3 {form} FBP, {dtype}: {ms:.1f} ms, {g.nvox / ms / 1e6:.2f} GVox/s")
            assert torch.isfinite(v).all()
            out[form] = np.stack([v[:, i1, i0].cpu().numpy() for i0, i1 in cols])
            del v
    t0 = time.time()
    of, od = _oracle_columns(ds, g, cols)
    ef, ed = rel(out["fourier"], of), rel(out["direct"], od)
    print(f"c3 full data {dtype}, {len(cols)} columns x {g.n2} slices (oracle {time.time() - t0:.0f} s): "
          f"Fourier relL2 {ef:.2e}, direct relL2 {ed:.2e}; forms' gap: GPU {rel(out['fourier'], out['direct']):.3f}, "
          f"oracle {rel(of, od):.3f}")
    assert ef <= 1e-4
    assert ed <= 1e-5


def test_4096_wide_slab_fourier_parity(L):
    # the width of the paper's largest case (Table perf, N = 4096) on a
    # 256-slice slab: 8192-point x1/x2 grids and 8192-point filter rows, the
    # Fourier form z-chunked in 64 k_v planes (about 160 GB of workspace),
    # 1000 FP16 projections of 256 x 4096, tilt 10 deg; the oracle in chunks
    # of 50 angles on sampled whole columns
    g = I.Geometry(4096, 4096, 256, 1000, 256, 4096, math.radians(10.0))
    t0 = time.time()
    prm = I.ellipsoid_params(g, 600, seed=41, max_axis=40.0)
    d = I.project_boxed(prm, g, device="cuda", dtype=torch.float32).half()
    print(f"4096-wide inputs generated in {time.time() - t0:.1f} s")
    rng = np.random.default_rng(42)
    cols = np.stack([g.n0 // 2 + rng.integers(-1200, 1200, 4), g.n1 // 2 + rng.integers(-1200, 1200, 4)],
                    axis=1).astype(np.int32)
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt, z_chunk=64) as p:
        info = p.info
        print(f"grids M1 = {info['m1']}, Wp = {info['wp']}, Wf = {info['wf']}, Hf = {info['hf']}; "
              f"Fourier workspace {p.workspace_bytes('fourier') / 2**30:.1f} GiB")
        v = p.fbp(d, form="fourier", kind="shepp")
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        p.fbp(d, form="fourier", kind="shepp", out=v)
        b.record()
        b.synchronize()
        p.status()
        ms = a.elapsed_time(b)
        print(f"4096x4096x256 Fourier FBP, 1000 FP16 projections: {ms:.0f} ms, {g.nvox / ms / 1e6:.2f} GVox/s")
        assert torch.isfinite(v).all()
        gf = np.stack([v[:, i1, i0].cpu().numpy() for i0, i1 in cols])
        del v
    of = np.zeros((len(cols), g.n2))
    for k0 in range(0, g.nproj, 50):
        idx = np.arange(k0, min(g.nproj, k0 + 50))
        q = O.filter_rows(d[k0:k0 + len(idx)].float().cpu().numpy(), g, "shepp")
        of += O.backproject_trig_columns(q, g, cols, angle_index=idx)
    e = rel(gf, of)
    print(f"4096-wide slab: Fourier relL2 vs FP64 oracle on {len(cols)} columns = {e:.2e}")
    assert e <= 1e-4
