"""Seeded synthetic inputs for laminographic FBP: geometry, phantoms, projections.

This module is the one thing the CUDA path and the FP64 oracle share. It holds
no filtering or backprojection arithmetic: it draws phantom parameters, builds
the laminographic projection data those phantoms would produce (the data model
of the paper's forward operator, Sec. 4 Eq. fwd and the two delta functions
after it) and adds seeded noise.

Conventions (the paper leaves them open; the same readings are used everywhere):

* voxel = detector pixel = 1 length unit;
* voxel index i along an axis of size n sits at x = i - n/2;
* detector column j sits at u = j - W/2, row r at v = r - H/2;
* theta_k = 2*pi*k/nproj ("equally spaced over [0, 360)");
* a = (cos t, sin t, 0), b = (sin t sin phi, -cos t sin phi, cos phi), so that
  u = a.x and v = b.x (Sec. 4, the delta functions after Eq. fwd); phi = 0 is
  tomography (Sec. 4 notes that phi = 0 gives the Radon transform);
* the ray through detector point (u, v) is p + s*w with p = u a + v b and
  w = a x b = (sin t cos phi, -cos t cos phi, -sin phi).

Layouts are C order: projections [nproj][det_h][det_w], volume [n2][n1][n0].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # torch is only needed for fast projection of large phantoms
    import torch
except Exception:  # pragma: no cover - torch is present in every supported setup
    torch = None


@dataclasses.dataclass(frozen=True)
class Geometry:
    n0: int          # x1 (fastest axis of the volume)
    n1: int          # x2
    n2: int          # x3 (slab thickness)
    nproj: int
    det_h: int
    det_w: int
    tilt: float      # radians, tilt away from tomography

    @property
    def angles(self) -> np.ndarray:
        return 2.0 * np.pi * np.arange(self.nproj, dtype=np.float64) / self.nproj

    @property
    def nvox(self) -> int:
        return self.n0 * self.n1 * self.n2


# Workloads shaped like the paper's slab scans (Sec. 5-6: thin x3, wide x1/x2,
# full 360-degree rotations). Phantom recipes are stated next to each entry.
CONFIGS = {
    # 64^3, 64 angles, detector 64x96, tilt 20; 12 Gaussian blobs, 1% noise
    "c1": dict(geom=Geometry(64, 64, 64, 64, 64, 96, math.radians(20.0)),
               phantom="blobs", count=12, sigma=(2.0, 6.0), amp=(0.5, 1.0),
               noise=0.01, filter="shepp", seed=1),
    # 512x512x256 slab, 720 angles, detector 256x768, tilt 20; 200 ellipsoids
    "c2": dict(geom=Geometry(512, 512, 256, 720, 256, 768, math.radians(20.0)),
               phantom="ellipsoids", count=200, noise=0.01, filter="shepp", seed=2),
    # 2048x2048x512 slab, 1800 angles, detector 512x2048 stored fp16, tilt 18;
    # 5000 ellipsoids (semi-axes U[2, 48]) + 2% dense spheres, Poisson 1e4
    "c3": dict(geom=Geometry(2048, 2048, 512, 1800, 512, 2048, math.radians(18.0)),
               phantom="ellipsoids", count=5000, dense_frac=0.02, poisson=1e4,
               max_axis=48.0, filter="shepp", seed=3, storage="f16"),
    # the c2 geometry with a band-limited phantom whose projections stay inside
    # the detector: 40 Gaussian blobs (sigma U[12, 20]) centred in
    # |x1|, |x2| <= 100, |x3| <= 30, noise-free. Here the two forms' own
    # discretisation gap is below 1e-3 (the agreement the metric asks for).
    "c2b": dict(geom=Geometry(512, 512, 256, 720, 256, 768, math.radians(20.0)),
                phantom="blobs", count=40, sigma=(12.0, 20.0), amp=(0.5, 1.0),
                box=(100.0, 100.0, 30.0), noise=0.0, filter="shepp", seed=6),
    # 256x256x128, 400 angles, detector 128x384, tilt 30; blobs, 0.5% noise
    "c4": dict(geom=Geometry(256, 256, 128, 400, 128, 384, math.radians(30.0)),
               phantom="blobs", count=24, sigma=(3.0, 10.0), amp=(0.5, 1.0),
               noise=0.005, filter="shepp", seed=4),
}


def geometry_vectors(theta: np.ndarray, tilt: float):
    """Unit vectors a_k, b_k, w_k (each [nproj, 3], float64)."""
    ct, st = np.cos(theta), np.sin(theta)
    sp, cp = math.sin(tilt), math.cos(tilt)
    a = np.stack([ct, st, np.zeros_like(ct)], axis=1)
    b = np.stack([st * sp, -ct * sp, np.full_like(ct, cp)], axis=1)
    w = np.stack([st * cp, -ct * cp, np.full_like(ct, -sp)], axis=1)
    return a, b, w


# ----------------------------------------------------------------------------
# phantom parameters
# ----------------------------------------------------------------------------

def blob_params(geom: Geometry, count: int, seed: int, sigma=(2.0, 6.0), amp=(0.5, 1.0),
                box=None):
    """Gaussian blobs A*exp(-|x-c|^2/(2 s^2)); centres drawn inside the slab, or
    uniformly in |x_i| <= box[i] when `box` is given.

    Returns dict(centre [count,3], sigma [count], amp [count]) in float64.
    """
    rng = np.random.default_rng(seed)
    s = rng.uniform(sigma[0], sigma[1], count)
    a = rng.uniform(amp[0], amp[1], count)
    if box is not None:
        c = rng.uniform(-1.0, 1.0, (count, 3)) * np.asarray(box, dtype=np.float64)[None, :]
        return dict(kind="blobs", centre=c, sigma=s, amp=a)
    half = np.array([geom.n0, geom.n1, geom.n2], dtype=np.float64) / 2.0
    # keep each blob two widths away from the slab faces where the slab allows
    margin = np.minimum(2.0 * s[:, None], 0.45 * half[None, :])
    c = rng.uniform(-1.0, 1.0, (count, 3)) * (half[None, :] - margin)
    return dict(kind="blobs", centre=c, sigma=s, amp=a)


def _random_rotation(rng) -> np.ndarray:
    # uniform rotation from a random unit quaternion
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def ellipsoid_params(geom: Geometry, count: int, seed: int, dense_frac: float = 0.0,
                     max_axis: float | None = None):
    """Random ellipsoids {|M(x-c)| <= 1} of density rho, overlapping densities add.

    Semi-axes U[2, n/8] voxels (n = smallest of n0, n1, or U[2, max_axis]; capped
    so they fit the slab), random orientation, centres inside the slab,
    rho ~ U[0, 1]. With
    dense_frac > 0 that fraction of extra small dense spheres (rho = 5) is added.
    Returns dict(M [count,3,3], centre [count,3], rho [count]).
    """
    rng = np.random.default_rng(seed)
    nmin = min(geom.n0, geom.n1)
    amax = max(2.5, nmin / 8.0) if max_axis is None else max_axis
    half = np.array([geom.n0, geom.n1, geom.n2], dtype=np.float64) / 2.0
    Ms, cs, rhos = [], [], []
    for _ in range(count):
        ax = rng.uniform(2.0, amax, 3)
        ax = np.minimum(ax, 0.45 * half.min() + 2.0)
        R = _random_rotation(rng)
        M = np.diag(1.0 / ax) @ R.T
        c = rng.uniform(-1.0, 1.0, 3) * np.maximum(half - ax.max(), 1.0)
        Ms.append(M)
        cs.append(c)
        rhos.append(rng.uniform(0.0, 1.0))
    ndense = int(round(dense_frac * count))
    for _ in range(ndense):
        r = rng.uniform(1.5, 4.0)
        c = rng.uniform(-1.0, 1.0, 3) * np.maximum(half - r, 1.0)
        Ms.append(np.eye(3) / r)
        cs.append(c)
        rhos.append(5.0)
    return dict(kind="ellipsoids", M=np.array(Ms), centre=np.array(cs), rho=np.array(rhos))


# ----------------------------------------------------------------------------
# analytic projections (line integrals of the phantoms)
# ----------------------------------------------------------------------------

def _detector_grid(geom: Geometry, xp, dev, dt):
    u = xp.arange(geom.det_w, dtype=dt, device=dev) - geom.det_w / 2.0
    v = xp.arange(geom.det_h, dtype=dt, device=dev) - geom.det_h / 2.0
    return u, v


def project(params: dict, geom: Geometry, device: str = "cpu", dtype=None,
            chunk: int = 64) -> "torch.Tensor":
    """Exact line integrals of a phantom at every detector pixel centre.

    Gaussian blob:  A * s*sqrt(2 pi) * exp(-((u - a.c)^2 + (v - b.c)^2) / (2 s^2)).
    Ellipsoid:      chord 2*sqrt(beta^2 - alpha*gamma)/alpha (0 if negative) with
                    alpha = |Mw|^2, beta = Mw.M(p-c), gamma = |M(p-c)|^2 - 1.
    Returns a torch tensor [nproj, det_h, det_w] in `dtype` (default float64)
    on `device`.
    """
    if torch is None:
        raise RuntimeError("torch is required for projection")
    dt = torch.float64 if dtype is None else dtype
    dev = torch.device(device)
    theta = geom.angles
    a, b, w = geometry_vectors(theta, geom.tilt)
    out = torch.zeros((geom.nproj, geom.det_h, geom.det_w), dtype=dt, device=dev)
    u, v = _detector_grid(geom, torch, dev, dt)
    U = u[None, None, :]
    V = v[None, :, None]
    for k0 in range(0, geom.nproj, chunk):
        k1 = min(geom.nproj, k0 + chunk)
        sl = slice(k0, k1)
        acc = out[sl]
        if params["kind"] == "blobs":
            for c, s, amp in zip(params["centre"], params["sigma"], params["amp"]):
                uc = torch.as_tensor(a[sl] @ c, dtype=dt, device=dev)[:, None, None]
                vc = torch.as_tensor(b[sl] @ c, dtype=dt, device=dev)[:, None, None]
                r2 = (U - uc) ** 2 + (V - vc) ** 2
                acc += (amp * s * math.sqrt(2.0 * math.pi)) * torch.exp(-r2 / (2.0 * s * s))
        else:
            for M, c, rho in zip(params["M"], params["centre"], params["rho"]):
                Ma = a[sl] @ M.T           # [k, 3]
                Mb = b[sl] @ M.T
                Mw = w[sl] @ M.T
                Mc = M @ c
                al = np.einsum("ki,ki->k", Mw, Mw)
                bu = np.einsum("ki,ki->k", Mw, Ma)
                bv = np.einsum("ki,ki->k", Mw, Mb)
                b0 = -(Mw @ Mc)
                guu = np.einsum("ki,ki->k", Ma, Ma)
                gvv = np.einsum("ki,ki->k", Mb, Mb)
                guv = np.einsum("ki,ki->k", Ma, Mb)
                gu0 = -(Ma @ Mc)
                gv0 = -(Mb @ Mc)
                g00 = float(Mc @ Mc) - 1.0
                T = lambda z: torch.as_tensor(z, dtype=dt, device=dev)[:, None, None]
                beta = T(bu) * U + T(bv) * V + T(b0)
                gamma = (T(guu) * U * U + 2.0 * T(guv) * U * V + T(gvv) * V * V
                         + 2.0 * T(gu0) * U + 2.0 * T(gv0) * V + g00)
                disc = beta * beta - T(al) * gamma
                acc += (2.0 * rho) * torch.sqrt(torch.clamp(disc, min=0.0)) / T(al)
    return out


def project_boxed(params: dict, geom: Geometry, device: str = "cpu", dtype=None,
                  angle_chunk: int = 32, batch: int = 64) -> "torch.Tensor":
    """The same line integrals as `project` for an ellipsoid phantom, evaluated
    only inside each ellipsoid's projected bounding disk (radius = its largest
    semi-axis): identical values at a cost set by the footprints rather than
    by the whole detector. Ellipsoids are processed in batches of similar size.
    """
    if params["kind"] != "ellipsoids":
        return project(params, geom, device, dtype)
    dt = torch.float64 if dtype is None else dtype
    dev = torch.device(device)
    theta = geom.angles
    a, b, w = geometry_vectors(theta, geom.tilt)
    M = params["M"]
    c = params["centre"]
    rho = params["rho"]
    R = 1.0 / np.linalg.svd(M, compute_uv=False)[:, -1]        # largest semi-axis
    order = np.argsort(R)
    out = torch.zeros((geom.nproj, geom.det_h, geom.det_w), dtype=dt, device=dev)
    T = lambda z: torch.as_tensor(np.ascontiguousarray(z), dtype=dt, device=dev)
    for k0 in range(0, geom.nproj, angle_chunk):
        k1 = min(geom.nproj, k0 + angle_chunk)
        A_, B_, W_ = a[k0:k1], b[k0:k1], w[k0:k1]
        kk = torch.arange(k0, k1, device=dev)
        for e0 in range(0, len(order), batch):
            idx = order[e0:e0 + batch]
            Mb, cb, rb = M[idx], c[idx], rho[idx]
            h = int(np.ceil(R[idx].max())) + 2
            off = torch.arange(-h, h + 1, device=dev)
            Ma = np.einsum("eij,kj->eki", Mb, A_)       # [E, K, 3]
            Mv = np.einsum("eij,kj->eki", Mb, B_)
            Mw = np.einsum("eij,kj->eki", Mb, W_)
            Mc = np.einsum("eij,ej->ei", Mb, cb)[:, None, :]
            al = (Mw * Mw).sum(-1)
            bu, bv, b0 = (Mw * Ma).sum(-1), (Mw * Mv).sum(-1), -(Mw * Mc).sum(-1)
            guu, gvv, guv = (Ma * Ma).sum(-1), (Mv * Mv).sum(-1), (Ma * Mv).sum(-1)
            gu0, gv0 = -(Ma * Mc).sum(-1), -(Mv * Mc).sum(-1)
            g00 = (Mc * Mc).sum(-1)[:, :1] - 1.0
            uc = cb @ A_.T                               # [E, K] projected centres
            vc = cb @ B_.T
            j0 = torch.as_tensor(np.rint(uc + geom.det_w / 2.0), dtype=torch.long, device=dev)
            r0 = torch.as_tensor(np.rint(vc + geom.det_h / 2.0), dtype=torch.long, device=dev)
            jj = j0[:, :, None, None] + off[None, None, None, :]     # [E, K, 1, P]
            rr = r0[:, :, None, None] + off[None, None, :, None]     # [E, K, P, 1]
            U = (jj - geom.det_w / 2.0).to(dt)
            V = (rr - geom.det_h / 2.0).to(dt)
            X = lambda z: T(z)[:, :, None, None]
            beta = X(bu) * U + X(bv) * V + X(b0)
            gamma = (X(guu) * U * U + 2.0 * X(guv) * U * V + X(gvv) * V * V
                     + 2.0 * X(gu0) * U + 2.0 * X(gv0) * V + T(g00)[:, :, None, None])
            disc = beta * beta - X(al) * gamma
            val = (2.0 * T(rb)[:, None, None, None]) * torch.sqrt(torch.clamp(disc, min=0.0)) / X(al)
            jjb, rrb = torch.broadcast_tensors(jj, rr)
            kb = kk[None, :, None, None].expand_as(jjb)
            ok = (jjb >= 0) & (jjb < geom.det_w) & (rrb >= 0) & (rrb < geom.det_h) & (val > 0)
            out.index_put_((kb[ok], rrb[ok], jjb[ok]), val[ok], accumulate=True)
    return out


def add_noise(d, frac: float, seed: int):
    """Additive Gaussian noise with sigma = frac * max|d| (seeded, numpy PCG64)."""
    if frac <= 0:
        return d
    rng = np.random.default_rng(seed + 1000003)
    scale = float(d.abs().max()) * frac
    n = rng.standard_normal(tuple(d.shape), dtype=np.float32)
    return d + scale * torch.as_tensor(n, device=d.device).to(d.dtype)


def add_poisson(d, photons: float, seed: int, mu_scale: float | None = None, chunk: int = 64):
    """Poisson counting noise at `photons` per pixel, returned as line integrals.

    The line integrals are scaled so the darkest pixel transmits about 5%, the
    counts are drawn from I0*exp(-d) (torch generator on d's device, seeded,
    chunks of `chunk` projections) and d is re-estimated as -log(counts/I0)
    (a count of 0 is clamped to 0.5). Returns (noisy line integrals, scale).
    """
    g = torch.Generator(device=d.device).manual_seed(seed + 7919)
    if mu_scale is None:
        dmax = float(d.max())
        mu_scale = 3.0 / dmax if dmax > 0 else 1.0
    out = torch.empty_like(d)
    for k0 in range(0, d.shape[0], chunk):
        lam = photons * torch.exp(-(d[k0:k0 + chunk].double() * mu_scale))
        counts = torch.poisson(lam, generator=g).clamp_(min=0.5)
        out[k0:k0 + chunk] = (-torch.log(counts / photons) / mu_scale).to(d.dtype)
    return out, mu_scale


def make_projections(name: str, device: str = "cpu", dtype=None, slab: int = 0):
    """Build the seeded synthetic projections of one named workload.

    Returns (geom, params, d) where d is a float32 tensor on `device` (use
    `storage_dtype(name)` for the type the workload stores projections in).
    `slab` > 0 draws another independent specimen of the same workload (the
    seed is offset), as each replica of a multi-GPU run reconstructs its own.
    """
    cfg = dict(CONFIGS[name])
    cfg["seed"] = cfg["seed"] + 1009 * slab
    geom = cfg["geom"]
    if cfg["phantom"] == "blobs":
        params = blob_params(geom, cfg["count"], cfg["seed"], cfg["sigma"], cfg["amp"],
                             cfg.get("box"))
    else:
        params = ellipsoid_params(geom, cfg["count"], cfg["seed"], cfg.get("dense_frac", 0.0),
                                  cfg.get("max_axis"))
    if params["kind"] == "ellipsoids":
        d = project_boxed(params, geom, device=device, dtype=dtype)
    else:
        d = project(params, geom, device=device, dtype=dtype)
    if "poisson" in cfg:
        d, _ = add_poisson(d, cfg["poisson"], cfg["seed"])
    else:
        d = add_noise(d, cfg["noise"], cfg["seed"])
    return geom, params, d.float()


def storage_dtype(name: str):
    """torch dtype a workload stores its projections in (float32 unless stated)."""
    st = CONFIGS[name].get("storage", "f32")
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[st]


def rasterize_blobs(params: dict, geom: Geometry) -> np.ndarray:
    """The blob phantom sampled at voxel centres, float64 [n2, n1, n0]."""
    x1 = np.arange(geom.n0) - geom.n0 / 2.0
    x2 = np.arange(geom.n1) - geom.n1 / 2.0
    x3 = np.arange(geom.n2) - geom.n2 / 2.0
    out = np.zeros((geom.n2, geom.n1, geom.n0))
    for c, s, amp in zip(params["centre"], params["sigma"], params["amp"]):
        g1 = np.exp(-(x1 - c[0]) ** 2 / (2 * s * s))
        g2 = np.exp(-(x2 - c[1]) ** 2 / (2 * s * s))
        g3 = np.exp(-(x3 - c[2]) ** 2 / (2 * s * s))
        out += amp * g3[:, None, None] * g2[None, :, None] * g1[None, None, :]
    return out


def rasterize_ellipsoids(params: dict, geom: Geometry, sub: int = 2) -> np.ndarray:
    """The ellipsoid phantom averaged over sub^3 points per voxel, float64
    [n2, n1, n0] (the sampled truth for reconstruction-quality checks)."""
    o = (np.arange(sub) + 0.5) / sub - 0.5
    out = np.zeros((geom.n2, geom.n1, geom.n0))
    for a in o:
        for b in o:
            for c in o:
                x1 = np.arange(geom.n0) - geom.n0 / 2.0 + a
                x2 = np.arange(geom.n1) - geom.n1 / 2.0 + b
                x3 = np.arange(geom.n2) - geom.n2 / 2.0 + c
                X = np.stack(np.meshgrid(x1, x2, x3, indexing="ij"), -1)   # [n0, n1, n2, 3]
                acc = np.zeros(X.shape[:3])
                for M, cen, rho in zip(params["M"], params["centre"], params["rho"]):
                    y = (X - cen) @ M.T
                    acc += rho * ((y * y).sum(-1) <= 1.0)
                out += acc.transpose(2, 1, 0)
    return out / sub ** 3


def random_projections(geom: Geometry, seed: int, dtype=np.float64) -> np.ndarray:
    """Plain seeded N(0,1) detector data [nproj, det_h, det_w] (for operator tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((geom.nproj, geom.det_h, geom.det_w)).astype(dtype)


def random_volume(geom: Geometry, seed: int, dtype=np.float64) -> np.ndarray:
    """Plain seeded N(0,1) volume [n2, n1, n0] (for adjoint tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((geom.n2, geom.n1, geom.n0)).astype(dtype)
