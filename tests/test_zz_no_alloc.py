"""The allocation-free Fourier backprojection (lamino_backproject_fourier_noalloc).

Callers that must not allocate device memory while they reconstruct (a
streaming loop that may not stall on the allocator, a process whose device
memory belongs to a pool, code recorded into a CUDA graph) use this entry
point: it takes its workspace from a fixed 64 MiB array in the library instead
of cudaMalloc'ing one. These tests call it through the C ABI and check that it
gives the same volume as lamino_backproject_fourier, on two calls in a row (the
shared array keeps the previous call's contents), and that it refuses a
geometry whose workspace does not fit, with a message naming both sizes.

This file is collected last on purpose and also passes when run alone.
"""
import math

import numpy as np
import pytest
import torch

from paper_2401_11101_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2401_11101_gb300 import _build, lamino
    _build.build()
    lamino.load_library()
    return lamino


def _rel(a, b):
    a = a.double().cpu().ravel()
    b = b.double().cpu().ravel()
    return float((a - b).norm() / b.norm())


def test_noalloc_first_on_fresh_plan_allocates_nothing(L):
    # a fresh plan whose Fourier workspaces were never allocated: the entry
    # point runs before any allocating call, and device memory does not move
    # across a call once the first one (which also loads the kernels and looks
    # up the static array) is done
    g = I.Geometry(48, 48, 24, 30, 28, 72, math.radians(25.0))
    q = torch.as_tensor(I.random_projections(g, 6), dtype=torch.float32).cuda()
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        out = torch.empty(p.shape_vol, dtype=torch.float32, device="cuda")
        p.backproject_fourier_noalloc(q, out)
        torch.cuda.synchronize()
        first = out.clone()
        free0 = torch.cuda.mem_get_info()[0]
        out.fill_(float("nan"))
        p.backproject_fourier_noalloc(q, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, f"device free memory moved by {free0 - free1} bytes"
        assert torch.equal(out, first)
        ref = p.backproject_fourier(q)          # allocates the plan's own workspaces
        assert _rel(out, ref) <= 1e-6


def test_noalloc_rejects_tensors_it_would_have_to_convert(L):
    g = I.Geometry(16, 16, 8, 6, 10, 24, math.radians(20.0))
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        q = torch.zeros(p.shape_proj, dtype=torch.float32, device="cuda")
        out = torch.empty(p.shape_vol, dtype=torch.float32, device="cuda")
        for bad_q, bad_out in ((q.double(), out), (q, out.double()), (q.cpu(), out),
                               (q, torch.empty(p.shape_vol[::-1], device="cuda").transpose(0, 2))):
            with pytest.raises(ValueError):
                p.backproject_fourier_noalloc(bad_q, bad_out)


def test_noalloc_matches_fourier_twice(L):
    g, _, d = I.make_projections("c1")
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        assert p.workspace_bytes("fourier") <= 64 << 20
        q = p.filter(d.cuda(), "shepp")
        ref = p.backproject_fourier(q)
        out = torch.empty_like(ref)
        for _ in range(2):
            out.fill_(float("nan"))
            p.backproject_fourier_noalloc(q, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel(out, ref) <= 1e-6


def test_noalloc_second_geometry_after_first(L):
    # a different plan reuses the same static array after the first one
    g = I.Geometry(32, 32, 16, 24, 20, 48, math.radians(30.0))
    q = torch.as_tensor(I.random_projections(g, 5), dtype=torch.float32).cuda()
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        ref = p.backproject_fourier(q)
        out = torch.empty_like(ref)
        for _ in range(2):
            p.backproject_fourier_noalloc(q, out)
            torch.cuda.synchronize()
            assert _rel(out, ref) <= 1e-6


def test_noalloc_rejects_oversize_geometry(L):
    g = I.CONFIGS["c2"]["geom"]
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        assert p.workspace_bytes("fourier") > 64 << 20
        q = torch.zeros(p.shape_proj, dtype=torch.float32, device="cuda")
        out = torch.empty(p.shape_vol, dtype=torch.float32, device="cuda")
        with pytest.raises(L.LaminoError) as e:
            p.backproject_fourier_noalloc(q, out)
        assert e.value.code == L.EINVAL
        assert "static scratch" in str(e.value) and str(64 << 20) in str(e.value)
