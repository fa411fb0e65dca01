"""Z chunking (Sec. 5: the 2D USFFT of the split Eq. fftfwdsplit by chunks of
k_v slices, the 1D USFFT by chunks of columns, the direct form by chunks of
x3 slices).

Every plane, column and voxel tile is computed by the same arithmetic whether
or not the work is chunked, so chunked results must equal the unchunked ones
bit for bit; the chunked Fourier workspace must be smaller wherever the
x1-pass planes dominate it.
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


# few projections and wide planes: the x1-pass planes V dominate workspace A
WIDE = I.Geometry(128, 128, 64, 90, 64, 192, math.radians(20.0))


@pytest.mark.parametrize("geom,zc", [
    (WIDE, 16),
    (WIDE, 7),                                                   # chunks that do not divide the planes
    (I.Geometry(24, 40, 12, 10, 14, 40, math.radians(33.0)), 5),  # 3*2^k grids
    (I.CONFIGS["c1"]["geom"], 13),
])
def test_chunked_fourier_equals_unchunked(L, geom, zc):
    d = torch.as_tensor(I.random_projections(geom, 81), dtype=torch.float32).cuda()
    with plan_for(L, geom) as p, plan_for(L, geom, z_chunk=zc) as pc:
        assert pc.info["z_chunk"] == zc and pc.info["plane_chunk"] == min(zc, pc.info["planes"])
        v = p.fbp(d, form="fourier", kind="shepp")
        vc = pc.fbp(d, form="fourier", kind="shepp")
        bp = p.backproject_fourier(d)
        bpc = pc.backproject_fourier(d)
        pc.status()
    print(f"{geom} z_chunk={zc}: planes {pc.info['planes']}, chunked vs unchunked "
          f"max |diff| {float((vc - v).abs().max()):.1e}")
    assert torch.equal(v, vc)
    assert torch.equal(bp, bpc)


def test_chunked_workspace_is_smaller_and_parity_holds(L):
    g = WIDE
    q = I.random_projections(g, 82).astype(np.float32)
    with plan_for(L, g) as p, plan_for(L, g, z_chunk=16) as pc:
        full, chunked = p.workspace_bytes("fourier"), pc.workspace_bytes("fourier")
        free0 = torch.cuda.mem_get_info()[0]
        v = pc.backproject_fourier(torch.as_tensor(q).cuda())
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        v = v.cpu().numpy()
    print(f"Fourier workspace: unchunked {full / 2**20:.2f} MiB, z_chunk=16 {chunked / 2**20:.2f} MiB, "
          f"device memory taken by the chunked call {used / 2**20:.2f} MiB")
    assert chunked < 0.9 * full
    e = rel(v, O.backproject_fourier(q, g))
    print(f"chunked Fourier backprojection relL2 vs exact sum = {e:.2e}")
    assert e <= 1e-4


def test_chunked_projector_equals_unchunked(L):
    g = WIDE
    mu = torch.as_tensor(I.random_volume(g, 83), dtype=torch.float32).cuda()
    with plan_for(L, g) as p, plan_for(L, g, z_chunk=9) as pc:
        a = p.project(mu, form="fourier")
        b = pc.project(mu, form="fourier")
    assert torch.equal(a, b)


@pytest.mark.parametrize("zc", [16, 40, 64])
def test_chunked_direct_equals_unchunked(L, zc):
    g = I.Geometry(40, 24, 90, 9, 60, 50, math.radians(33.0))   # 90 slices: a ragged last slab
    d = torch.as_tensor(I.random_projections(g, 84), dtype=torch.float32).cuda()
    with plan_for(L, g) as p, plan_for(L, g, z_chunk=zc) as pc:
        v = p.fbp(d, form="direct", kind="ramp")
        pc.profile(True)
        vc = pc.fbp(d, form="direct", kind="ramp")
        launches = [n for n, _ in pc.profile_read() if n == "direct"]
        pc.status()
    slab = (zc + 31) // 32 * 32                     # whole 32-slice tiles per launch
    assert len(launches) == math.ceil(g.n2 / slab)
    assert torch.equal(v, vc)


def test_set_z_chunk_reallocates(L):
    g = WIDE
    d = torch.as_tensor(I.random_projections(g, 85), dtype=torch.float32).cuda()
    with plan_for(L, g) as p:
        v = p.fbp(d, form="fourier")
        full = p.workspace_bytes("fourier")
        p.set_z_chunk(8)
        assert p.info["plane_chunk"] == 8
        assert p.workspace_bytes("fourier") < full
        assert torch.equal(p.fbp(d, form="fourier"), v)
        p.set_z_chunk(0)
        assert p.workspace_bytes("fourier") == full
        assert torch.equal(p.fbp(d, form="fourier"), v)
        with pytest.raises(L.LaminoError):
            p.set_z_chunk(-1)


def test_chunked_host_pipeline(L):
    g = I.Geometry(64, 64, 32, 40, 32, 96, math.radians(20.0))
    d = torch.as_tensor(I.random_projections(g, 86), dtype=torch.float32)
    with plan_for(L, g, z_chunk=6) as p:
        out = torch.empty(p.shape_vol, dtype=torch.float32).pin_memory()
        dev = p.fbp(d.cuda(), form="fourier", kind="shepp").cpu()
        p.fbp_host(d.pin_memory(), out, form="fourier", kind="shepp")
    assert rel(out.numpy(), dev.numpy()) < 1e-6


def test_lent_workspace_gives_identical_results_and_allocates_nothing(L):
    g = I.Geometry(64, 64, 32, 40, 32, 98, math.radians(20.0))    # 98 columns: the padded TMA copy too
    d = torch.as_tensor(I.random_projections(g, 87), dtype=torch.float32).cuda()
    with plan_for(L, g) as own, plan_for(L, g, z_chunk=8) as p:
        ref_f = own.fbp(d, form="fourier")
        ref_d = own.fbp(d, form="direct")
        need = max(p.workspace_bytes("fourier"), p.workspace_bytes("direct"))
        arena = torch.empty(need, dtype=torch.uint8, device="cuda")
        p.set_workspace(arena)
        out = torch.empty(p.shape_vol, dtype=torch.float32, device="cuda")
        p.fbp(d, form="fourier", out=out)                  # loads the kernels of both forms
        p.fbp(d, form="direct", out=out)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for form, ref in (("fourier", ref_f), ("direct", ref_d), ("fourier", ref_f)):
            p.fbp(d, form=form, out=out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), form
        assert torch.cuda.mem_get_info()[0] == free0
        assert p.device_bytes() < 1 << 20                  # tables only
        # too small a buffer: a clean ENOMEM naming both sizes
        p.set_workspace(arena[: 256 * 16])
        with pytest.raises(L.LaminoError) as e:
            p.fbp(d, form="fourier", out=out)
        assert e.value.code == L.ENOMEM and "lent workspace" in str(e.value)
        with pytest.raises(L.LaminoError) as e:
            p.set_workspace(arena[8:])                       # not 256-byte aligned
        assert e.value.code == L.EINVAL
        p.set_workspace(None)                                # back to plan-owned workspaces
        assert torch.equal(p.fbp(d, form="fourier"), ref_f)
