"""Python binding of the C ABI in include/lamino.h (argument marshalling only).

Every computation runs in liblamino.so; this module checks tensor shapes,
dtypes and devices, passes raw pointers and the current CUDA stream, and turns
status codes into exceptions. There is no fallback: if the library is missing
the import of the first call raises.

    plan = Plan(n0, n1, n2, nproj, det_w, det_h, tilt)
    vol = plan.fbp(d, form="fourier", kind="shepp")      # d: CUDA tensor
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblamino.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5
F32, F16, BF16 = 0, 1, 2
RAMP, SHEPP, PARZEN = 0, 1, 2
DIRECT, FOURIER = 0, 1

DTYPES = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}
FILTERS = {"ramp": RAMP, "shepp": SHEPP, "parzen": PARZEN}
FORMS = {"direct": DIRECT, "fourier": FOURIER}

# every symbol include/lamino.h declares
EXPORTS = ("lamino_plan", "lamino_get_info", "lamino_filter", "lamino_backproject_direct",
           "lamino_backproject_fourier", "lamino_backproject_fourier_noalloc", "lamino_fbp", "lamino_fbp_host", "lamino_project",
           "lamino_status", "lamino_selftest_wait", "lamino_profile", "lamino_profile_read", "lamino_workspace_bytes",
           "lamino_set_z_chunk", "lamino_device_bytes", "lamino_set_workspace",
           "lamino_last_error", "lamino_destroy")


class LaminoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lamino error {code}: {msg}")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("usfft_w", ctypes.c_int), ("usfft_wz", ctypes.c_int),
                ("wf", ctypes.c_int), ("hf", ctypes.c_int), ("grid_rows", ctypes.c_int),
                ("z_chunk", ctypes.c_int)]


class _KTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_float)]


class _Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("n0", "n1", "n2", "nproj", "det_w", "det_h", "wp", "wf", "hf", "m1", "m2", "m3",
                 "usfft_w", "usfft_wz", "planes")] + [("usfft_err_est", ctypes.c_float),
                                                       ("z_chunk", ctypes.c_int),
                                                       ("plane_chunk", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblamino.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, ci, cd, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.lamino_plan.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ci, ci, cd,
                                ctypes.POINTER(cd), ctypes.POINTER(_Opts)]
    lib.lamino_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    lib.lamino_filter.argtypes = [vp, vp, ci, vp, ci, vp]
    lib.lamino_backproject_direct.argtypes = [vp, vp, vp, vp]
    lib.lamino_backproject_fourier.argtypes = [vp, vp, ci, vp, vp]
    lib.lamino_backproject_fourier_noalloc.argtypes = [vp, vp, ci, vp, vp]
    lib.lamino_fbp.argtypes = [vp, ci, vp, ci, vp, ci, vp]
    lib.lamino_fbp_host.argtypes = [vp, ci, vp, ci, vp, ci, vp]
    lib.lamino_project.argtypes = [vp, ci, vp, vp, vp]
    lib.lamino_status.argtypes = [vp, vp]
    lib.lamino_selftest_wait.argtypes = [vp, ctypes.c_uint, vp]
    lib.lamino_workspace_bytes.argtypes = [vp, ci, ctypes.POINTER(sz)]
    lib.lamino_set_z_chunk.argtypes = [vp, ci]
    lib.lamino_device_bytes.argtypes = [vp, ctypes.POINTER(sz)]
    lib.lamino_set_workspace.argtypes = [vp, vp, sz]
    lib.lamino_profile.argtypes = [vp, ci]
    lib.lamino_profile_read.argtypes = [vp, ctypes.POINTER(_KTime), ci, ctypes.POINTER(ci)]
    lib.lamino_last_error.argtypes = [vp]
    lib.lamino_last_error.restype = ctypes.c_char_p
    lib.lamino_destroy.argtypes = [vp]
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or ci
    lib.lamino_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _form(form: str) -> int:
    if form not in FORMS:
        raise ValueError(f"form must be one of {sorted(FORMS)}, not {form!r}")
    return FORMS[form]


def _filter(kind: str) -> int:
    if kind not in FILTERS:
        raise ValueError(f"filter kind must be one of {sorted(FILTERS)}, not {kind!r}")
    return FILTERS[kind]


class Plan:
    """A reconstruction plan for one geometry (owns device tables/workspaces)."""

    def __init__(self, n0, n1, n2, nproj, det_w, det_h, tilt, angles=None, usfft_w=0,
                 usfft_wz=0, wf=0, hf=0, grid_rows=0, z_chunk=0, device=None):
        self._h = ctypes.c_void_p()
        ang_list = None
        if angles is not None:
            ang_list = [float(a) for a in angles]
            if len(ang_list) != nproj:
                # a shorter list would otherwise reach the library zero-padded
                raise ValueError(f"angles has {len(ang_list)} entries, nproj is {nproj}")
        self._lib = load_library()
        idx = None if device is None else torch.device(device).index
        self.device = torch.device("cuda", torch.cuda.current_device() if idx is None else idx)
        opts = _Opts(usfft_w, usfft_wz, wf, hf, grid_rows, z_chunk)
        ang = None
        if ang_list is not None:
            arr = (ctypes.c_double * nproj)(*ang_list)
            ang = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        with torch.cuda.device(self.device):
            rc = self._lib.lamino_plan(ctypes.byref(self._h), n0, n1, n2, nproj, det_w, det_h,
                                       float(tilt), ang, ctypes.byref(opts))
        if rc != OK:
            raise LaminoError(rc, self._lib.lamino_last_error(None).decode())
        self.shape_vol = (n2, n1, n0)
        self.shape_proj = (nproj, det_h, det_w)
        self.nproj = nproj
        self._read_info()

    def _read_info(self):
        info = _Info()
        self._check(self._lib.lamino_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _Info._fields_}

    # ----------------------------------------------------------------- utils
    def _check(self, rc):
        if rc != OK:
            raise LaminoError(rc, self._lib.lamino_last_error(self._h).decode())

    def _tensor(self, t, shape, dtypes, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device != self.device:
            raise ValueError(f"{name} is on {t.device}, plan on {self.device}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _out(self, out, shape):
        if out is None:
            return torch.empty(shape, dtype=torch.float32, device=self.device)
        return self._tensor(out, shape, (torch.float32,), "out")

    # ----------------------------------------------------------------- calls
    def filter(self, d, kind="shepp", out=None):
        d = self._tensor(d, self.shape_proj, tuple(DTYPES), "d")
        q = self._out(out, self.shape_proj)
        self._check(self._lib.lamino_filter(self._h, d.data_ptr(), DTYPES[d.dtype], q.data_ptr(),
                                            _filter(kind), _stream(self.device)))
        return q

    def backproject_direct(self, q, out=None):
        q = self._tensor(q, self.shape_proj, (torch.float32,), "q")
        v = self._out(out, self.shape_vol)
        self._check(self._lib.lamino_backproject_direct(self._h, q.data_ptr(), v.data_ptr(),
                                                        _stream(self.device)))
        return v

    def backproject_fourier(self, q, out=None):
        q = self._tensor(q, self.shape_proj, tuple(DTYPES), "q")
        v = self._out(out, self.shape_vol)
        self._check(self._lib.lamino_backproject_fourier(self._h, q.data_ptr(), DTYPES[q.dtype],
                                                         v.data_ptr(), _stream(self.device)))
        return v

    def backproject_fourier_noalloc(self, q, out):
        """Fourier-form backprojection that allocates no device memory (its
        workspace is the library's fixed 64 MiB static array). `out` must be
        given, since creating it would allocate; q and out are used as they
        are (a tensor of the wrong dtype, device or layout raises ValueError
        rather than being copied), and the volume is written into `out`."""
        q = self._tensor(q, self.shape_proj, tuple(DTYPES), "q")
        v = self._tensor(out, self.shape_vol, (torch.float32,), "out")
        self._check(self._lib.lamino_backproject_fourier_noalloc(
            self._h, q.data_ptr(), DTYPES[q.dtype], v.data_ptr(), _stream(self.device)))
        return v

    def backproject(self, q, form="fourier", out=None):
        _form(form)
        return (self.backproject_fourier if form == "fourier" else self.backproject_direct)(q, out)

    def fbp(self, d, form="fourier", kind="shepp", out=None):
        d = self._tensor(d, self.shape_proj, tuple(DTYPES), "d")
        v = self._out(out, self.shape_vol)
        self._check(self._lib.lamino_fbp(self._h, _form(form), d.data_ptr(), DTYPES[d.dtype],
                                         v.data_ptr(), _filter(kind), _stream(self.device)))
        return v

    def fbp_host(self, d_host, out_host, form="fourier", kind="shepp"):
        """FBP of a HOST tensor into a HOST float32 tensor (copies inside the call)."""
        for t, nm in ((d_host, "d_host"), (out_host, "out_host")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous host tensor")
        if tuple(d_host.shape) != self.shape_proj or tuple(out_host.shape) != self.shape_vol:
            raise ValueError("fbp_host: shape mismatch")
        if out_host.dtype != torch.float32 or d_host.dtype not in DTYPES:
            raise ValueError("fbp_host: dtype mismatch")
        self._check(self._lib.lamino_fbp_host(self._h, _form(form), d_host.data_ptr(),
                                              DTYPES[d_host.dtype], out_host.data_ptr(),
                                              _filter(kind), _stream(self.device)))
        return out_host

    def project(self, vol, form="direct", out=None):
        vol = self._tensor(vol, self.shape_vol, (torch.float32,), "vol")
        d = self._out(out, self.shape_proj)
        self._check(self._lib.lamino_project(self._h, _form(form), vol.data_ptr(), d.data_ptr(),
                                             _stream(self.device)))
        return d

    def set_workspace(self, buf):
        """Lend a CUDA tensor (any dtype, contiguous, 256-byte aligned) as this
        plan's workspace, or None to return to plan-owned workspaces. The plan
        keeps a reference while it is lent."""
        if buf is None:
            self._check(self._lib.lamino_set_workspace(self._h, None, 0))
            self._lent = None
            return
        if not isinstance(buf, torch.Tensor) or not buf.is_cuda or buf.device != self.device \
                or not buf.is_contiguous():
            raise ValueError("workspace must be a contiguous CUDA tensor on the plan's device")
        self._check(self._lib.lamino_set_workspace(self._h, buf.data_ptr(),
                                                   buf.numel() * buf.element_size()))
        self._lent = buf

    def set_z_chunk(self, z_chunk: int):
        """k_v planes per Fourier chunk / slices per direct launch (0: none);
        frees the Fourier workspaces, which the next call re-allocates."""
        self._check(self._lib.lamino_set_z_chunk(self._h, int(z_chunk)))
        self._read_info()

    def workspace_bytes(self, form="fourier") -> int:
        b = ctypes.c_size_t()
        self._check(self._lib.lamino_workspace_bytes(self._h, _form(form), ctypes.byref(b)))
        return int(b.value)

    def device_bytes(self) -> int:
        """Device memory this plan holds now (tables + allocated workspaces)."""
        b = ctypes.c_size_t()
        self._check(self._lib.lamino_device_bytes(self._h, ctypes.byref(b)))
        return int(b.value)

    def profile(self, enable: bool = True):
        """Bracket every kernel launch of this plan with CUDA events."""
        self._check(self._lib.lamino_profile(self._h, int(enable)))

    def profile_read(self, max_records: int = 4096):
        """[(kernel name, ms)] of the launches since the last read (waits for them)."""
        buf = (_KTime * max_records)()
        n = ctypes.c_int()
        self._check(self._lib.lamino_profile_read(self._h, buf, max_records, ctypes.byref(n)))
        return [(buf[i].name.decode(), float(buf[i].ms)) for i in range(n.value)]

    def status(self):
        """Synchronise the current stream; raise if a bounded device wait expired."""
        self._check(self._lib.lamino_status(self._h, _stream(self.device)))

    def selftest_wait(self, limit_us: int):
        """Queue a kernel whose bounded wait on a barrier nothing arrives at
        gives up after limit_us; the next status() raises LaminoError
        (LAMINO_ETIMEOUT)."""
        self._check(self._lib.lamino_selftest_wait(self._h, int(limit_us), _stream(self.device)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lamino_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
