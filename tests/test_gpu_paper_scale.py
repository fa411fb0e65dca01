"""Paper-scale slab (2048x2048x512, 1800 angles, detector 512x2048, tilt 18 deg)
with projections stored in FP16 and all arithmetic in FP32.

The exact oracle of the Fourier form needs every padded spectrum (about 136 GB
here), so parity at full size uses linearity: the GPU reconstructs FP16 inputs
in which only a few angles are non-zero, and the oracle computes exactly the
contribution of those angles on sampled columns (both forms). The full FP16
data are then reconstructed by both forms to check that they run at this size.
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_c3_fp16_paper_scale(L):
    t0 = time.time()
    g, _, d = I.make_projections("c3", device="cuda")
    d16 = d.to(I.storage_dtype("c3"))
    del d
    print(f"c3 inputs generated in {time.time() - t0:.1f} s")
    idx = np.array([0, 451, 900, 1349])
    dz = torch.zeros_like(d16)
    dz[torch.as_tensor(idx, device="cuda")] = d16[torch.as_tensor(idx, device="cuda")]
    rng = np.random.default_rng(77)
    cols = np.stack([rng.integers(0, g.n0, 4), rng.integers(0, g.n1, 4)], 1).astype(np.int32)
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        print(f"Fourier workspace {p.workspace_bytes('fourier') / 2**30:.1f} GiB")
        vf = p.fbp(dz, form="fourier", kind="shepp")
        vd = p.fbp(dz, form="direct", kind="shepp")
        p.status()
        gf = np.stack([vf[:, i1, i0].cpu().numpy() for i0, i1 in cols])
        gd = np.stack([vd[:, i1, i0].cpu().numpy() for i0, i1 in cols])
        # full data, both forms
        for form, v in (("fourier", vf), ("direct", vd)):
            p.fbp(d16, form=form, kind="shepp", out=v)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            p.fbp(d16, form=form, kind="shepp", out=v)
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
            print(f"c3 {form} FBP on FP16 projections: {ms:.1f} ms, {g.nvox / ms / 1e6:.2f} GVox/s")
            assert torch.isfinite(v).all()
        p.status()
    q = O.filter_rows(d16[torch.as_tensor(idx, device="cuda")].float().cpu().numpy(), g, "shepp")
    of = O.backproject_fourier_columns(q, g, cols, angle_index=idx)
    od = O.backproject_direct_columns(q, g, cols, angle_index=idx)
    ef, ed = rel(gf, of), rel(gd, od)
    print(f"c3 sparse-angle parity: fourier relL2 {ef:.2e}, direct relL2 {ed:.2e}")
    assert ef <= 1e-4
    assert ed <= 1e-5
