"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/lamino.h declares, and rejects bad arguments before touching
the device."""
import ctypes
import math
import os
import re

import pytest

from paper_2401_11101_gb300 import _build
from paper_2401_11101_gb300 import lamino as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return L.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "lamino.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lamino_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lamino_plan", "lamino_filter", "lamino_backproject_direct",
                     "lamino_backproject_fourier", "lamino_project"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert set(names) == set(L.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def _plan(lib, *args):
    h = ctypes.c_void_p()
    rc = lib.lamino_plan(ctypes.byref(h), *args, None, None)
    return rc, lib.lamino_last_error(None).decode()


@pytest.mark.parametrize("args", [
    (0, 64, 64, 64, 96, 64, 0.3),         # empty volume
    (64, 64, 64, 0, 96, 64, 0.3),         # no projections
    (64, 64, 64, 64, 20000, 64, 0.3),     # detector too wide
    (64, 64, 64, 64, 96, 0, 0.3),         # empty detector
    (64, 64, 64, 64, 96, 64, math.pi / 2),  # tilt at 90 degrees
    (64, 64, 64, 64, 96, 64, float("nan")),
    (9000, 64, 64, 64, 96, 64, 0.3),      # above the size limit
])
def test_plan_rejects_bad_geometry(lib, args):
    rc, msg = _plan(lib, *args)
    assert rc == L.EINVAL
    assert msg


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.lamino_filter(None, None, 0, None, 0, None) == L.EINVAL
    assert lib.lamino_backproject_direct(None, None, None, None) == L.EINVAL
    assert lib.lamino_backproject_fourier(None, None, 0, None, None) == L.EINVAL
    assert lib.lamino_project(None, 0, None, None, None) == L.EINVAL
    assert lib.lamino_destroy(None) == L.OK
    b = ctypes.c_size_t()
    assert lib.lamino_workspace_bytes(None, 0, ctypes.byref(b)) == L.EINVAL


def test_plan_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, msg = _plan(lib, 64, 64, 64, 64, 96, 64, 0.35)
    assert rc == L.ECUDA and "device" in msg


def test_binding_rejects_wrong_angle_count():
    # checked before the library or the device is touched: a shorter list
    # would otherwise reach lamino_plan zero-padded
    with pytest.raises(ValueError, match="angles"):
        L.Plan(8, 8, 8, 4, 12, 8, 0.3, angles=[0.0, 1.0, 2.0])
    with pytest.raises(ValueError, match="angles"):
        L.Plan(8, 8, 8, 2, 12, 8, 0.3, angles=[0.0, 1.0, 2.0])


@pytest.mark.parametrize("bad", ["Fourier", "auto", "fft", ""])
def test_binding_rejects_unknown_form_and_filter(bad):
    with pytest.raises(ValueError, match="form"):
        L._form(bad)
    with pytest.raises(ValueError, match="filter"):
        L._filter(bad)
    assert L._form("direct") == L.DIRECT and L._form("fourier") == L.FOURIER
    assert L._filter("parzen") == L.PARZEN
