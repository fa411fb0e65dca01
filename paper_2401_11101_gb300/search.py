"""Alignment searches of the paper's reconstruction pipeline (Sec. 6.1, Steps 1
and 2): one-slab reconstructions over candidate rotation centres, then over
candidate tilt angles, each scored by sparsity.

Each candidate reconstructs a thin slab around x3 = 0 (`slab` slices) with the
library's FBP. The paper picks the best slice by eye; here every slab gets a
sparsity score, ||mu||_1 / ||mu||_2 over a region (lower is better): a wrong
centre or tilt spreads every feature along arcs of backprojection lines,
which makes the image less sparse. As the paper observes, the middle of the
slice is hardly affected by a tilt error and its border is, so the centre is
scored on the central half of (x1, x2) and the tilt on the rest. The centre is
searched by moving the projections along u by -s before the reconstruction
(linear interpolation, zero outside the detector), the tilt with one plan per
candidate angle. The score is a heuristic: it needs features that are sparse
in the scored region.
"""
from __future__ import annotations

import torch

from . import lamino as L


def region_mask(n1: int, n0: int, region: str, device) -> torch.Tensor:
    """(x1, x2) mask: everything ("all"), the central half ("center") or the rest ("border")."""
    mask = torch.ones((n1, n0), dtype=torch.bool, device=device)
    if region != "all":
        inner = torch.zeros_like(mask)
        inner[n1 // 4:n1 - n1 // 4, n0 // 4:n0 - n0 // 4] = True
        mask = inner if region == "center" else ~inner
    return mask


def sparsity(vol: torch.Tensor, region: str = "all") -> float:
    """||mu||_1 / ||mu||_2 of the slab over the region (lower: sparser)."""
    v = vol.double()[:, region_mask(vol.shape[1], vol.shape[2], region, vol.device)]
    return float(v.abs().sum()) / max(float(torch.sqrt((v * v).sum())), 1e-300)


def shift_u(d: torch.Tensor, s: float) -> torch.Tensor:
    """Projections moved by s detector columns along u: out(j) = d(j - s),
    linear interpolation, zero outside the detector."""
    W = d.shape[-1]
    j = torch.arange(W, device=d.device, dtype=torch.float64) - s
    j0 = torch.floor(j)
    w = (j - j0).to(d.dtype)
    i0 = j0.long()
    out = torch.zeros_like(d)
    for off, wt in ((0, 1.0 - w), (1, w)):
        idx = i0 + off
        ok = (idx >= 0) & (idx < W)
        out[..., ok] += d[..., idx[ok]] * wt[ok]
    return out


class _Plans:
    def __init__(self):
        self.cache = {}

    def get(self, n0, n1, n2, nproj, det_w, det_h, tilt):
        key = (n0, n1, n2, nproj, det_w, det_h, round(float(tilt), 12))
        if key not in self.cache:
            self.cache[key] = L.Plan(n0, n1, n2, nproj, det_w, det_h, tilt)
        return self.cache[key]

    def close(self):
        for p in self.cache.values():
            p.close()
        self.cache.clear()


def center_search(d: torch.Tensor, n0: int, n1: int, tilt: float, shifts, slab: int = 2,
                  form: str = "fourier", kind: str = "shepp"):
    """Score every candidate centre offset s (detector columns; the axis sits at
    u = s): reconstruct the slab from the projections moved by -s. Returns
    (best s, list of (s, score)); the best has the lowest score."""
    nproj, det_h, det_w = d.shape
    plans = _Plans()
    try:
        p = plans.get(n0, n1, slab, nproj, det_w, det_h, tilt)
        scores = []
        for s in shifts:
            v = p.fbp(shift_u(d, -float(s)).contiguous(), form=form, kind=kind)
            scores.append((float(s), sparsity(v, "center")))
        p.status()
    finally:
        plans.close()
    return min(scores, key=lambda t: t[1])[0], scores


def tilt_search(d: torch.Tensor, n0: int, n1: int, tilts, slab: int = 2, form: str = "fourier",
                kind: str = "shepp"):
    """Score every candidate tilt (radians) by the sparsity of its slab's
    border. Returns (best tilt, list of (tilt, score)); the best has the
    lowest score."""
    nproj, det_h, det_w = d.shape
    plans = _Plans()
    try:
        scores = []
        for t in tilts:
            p = plans.get(n0, n1, slab, nproj, det_w, det_h, float(t))
            v = p.fbp(d, form=form, kind=kind)
            p.status()
            scores.append((float(t), sparsity(v, "border")))
    finally:
        plans.close()
    return min(scores, key=lambda t: t[1])[0], scores
