#!/usr/bin/env python
"""Laminographic FBP throughput on GB300: Fourier form vs direct form.

Workload (default): 512x512x256 slab, 720 projections over 360 degrees,
detector 256 rows x 768 columns, tilt 20 degrees, 200 random ellipsoids with
densities U[0,1], float32 projections with 1% Gaussian noise, Shepp-Logan
filter. Inputs are seeded and synthetic (paper_2401_11101_gb300.inputs).

One step = one pass of the whole hot path over the HBM-resident projections:
  Fourier FBP: filter fused into the row FFT, column FFT (half spectrum),
               Gaussian gridding + x1 inverse FFT, x2 inverse FFT, x3 USFFT;
  direct FBP:  row filter, TMA-staged bilinear backprojection.
`value` is the Fourier-form FBP throughput in GVox/s (the volume size over the
Fourier part of the step); the direct form's figure is reported beside it,
with the two forms' relative L2 gap. The metric's qualifier (the forms agree
to relL2 <= 1e-3) is shown on a band-limited input of the same geometry
(`qualifier`: c2b, whose own discretisation gap is below 1e-3).

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (torchrun): every rank reconstructs its own slab (independent
problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2401_11101_gb300 import inputs as I  # noqa: E402

METRIC = "lamino FBP GVox/s, Fourier vs direct on 1 GB300 @relL2<=1e-3; serve p50/p99 ms"
WORKLOADS = {
    "c2": "512x512x256 slab, 720 projections over 360 deg, detector 256x768, tilt 20 deg, "
          "200 random ellipsoids rho~U[0,1], float32 projections + 1% noise, Shepp-Logan",
    "c1": "64^3, 64 projections over 360 deg, detector 64x96, tilt 20 deg, 12 Gaussian blobs, "
          "1% noise, Shepp-Logan",
    "c4": "256x256x128, 400 projections over 360 deg, detector 128x384, tilt 30 deg, Gaussian "
          "blobs, 0.5% noise, Shepp-Logan",
    "c3": "2048x2048x512 slab, 1800 projections over 360 deg, detector 512x2048 stored FP16, "
          "tilt 18 deg, 5000 ellipsoids + 2% dense spheres, Poisson 1e4 photons, Shepp-Logan",
    "c2b": "512x512x256 slab, 720 projections over 360 deg, detector 256x768, tilt 20 deg, "
           "40 Gaussian blobs sigma~U[12,20] inside the detector's field of view, noise-free, "
           "Shepp-Logan (band-limited: the forms' own gap is below 1e-3)",
}
# shared-memory reduction pipe: 32 banks, one 32-bit reduction per bank and
# clock; a complex tap of the gridding is two of them (real, imaginary)
SMEM_RED_LANES_PER_CLK = 32
FP32_LANES_PER_SM = 128
N_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-columns", type=int, default=16)
    ap.add_argument("--z-chunk", type=int, default=0)
    ap.add_argument("--no-qualifier", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--cg-iters", type=int, default=50)
    return ap.parse_args()


# --------------------------------------------------------------------- utils

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, device):
    """Element-wise maximum over ranks of per-rank timings: the slowest rank
    sets the job's time (identity on one process)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()) \
            or torch.distributed.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_gvox_s(nvox_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the voxels all ranks reconstructed over the job time."""
    return world * nvox_per_rank / (ms * 1e-3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"lamino_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def grid_taps(p_info, g, planes=None) -> int:
    """Complex taps the gridding spreads per launch: every point (angle k,
    column frequency m, the Nyquist column dropped) of every plane it grids
    reaches (2w)^2 cells of the oversampled plane."""
    L = p_info["planes"] if planes is None else planes
    return L * g.nproj * (p_info["wf"] - 1) * (2 * p_info["usfft_w"]) ** 2


def kernel_algorithmic(p_info, g, esz_in=4):
    """Algorithmic bytes (one read of each input, one write of each output) or
    FP32 flops per launch of every kernel of the hot path."""
    nproj, H, W = g.nproj, g.det_h, g.det_w
    Wf, L = p_info["wf"], p_info["planes"]
    M2, n0, n1, n2 = p_info["m2"], g.n0, g.n1, g.n2
    c = 8  # complex64
    # row spectra R hold the frequencies m in [0, Wf/2) (real rows: -m is the
    # conjugate); the column pass writes both signs of m (all but the Nyquist)
    return {
        "filter_rowfft": ("hbm", nproj * H * W * esz_in + nproj * H * (Wf // 2) * c),
        "colfft": ("hbm", nproj * H * (Wf // 2) * c + L * nproj * (Wf - 1) * c),
        "grid": ("hbm", L * nproj * Wf * c + L * n0 * M2 * c),
        "colifft": ("hbm", L * n0 * M2 * c + L * n1 * n0 * c),
        "zusfft": ("hbm", L * n1 * n0 * c + n0 * n1 * n2 * 4),
        "filter": ("hbm", nproj * H * W * (esz_in + 4)),
        # bilinear update: 3 lerps (3 flops each) + accumulate = 10 flops
        "direct": ("alu", 10 * n0 * n1 * n2 * nproj),
    }


def src_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2401_11101_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if not os.path.exists(path):
        return {}
    out, digest = {}, None
    for line in open(path):
        line = line.strip()
        if line.startswith("# sources"):
            digest = line.split()[-1]
        elif line and not line.startswith("#"):
            parts = line.split()
            if len(parts) >= 2:
                out[parts[0]] = float(parts[1])
    return out if digest == src_digest() else {}


# --------------------------------------------------------------------- CPU oracle

def sample_columns(g, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, g.n0, n), rng.integers(0, g.n1, n)], 1).astype(np.int32)


def oracle_sample(d_cpu: np.ndarray, g, ncols: int, seed: int = 7, threads: int | None = None):
    """The FP64 oracle's FBP of both forms on a bounded sample: the row filter
    of every projection (a fixed cost), then the Fourier form (the exact sum,
    evaluated in detector space) and the direct form on ncols whole columns.
    Returns the times, the columns and both forms' values."""
    from oracle import lamino_oracle as O
    O.set_num_threads(threads or os.cpu_count() or 1)
    cols = sample_columns(g, ncols, seed)
    t0 = time.perf_counter()
    q = O.filter_rows(d_cpu, g, "shepp")
    t1 = time.perf_counter()
    of = O.backproject_trig_columns(q, g, cols)
    t2 = time.perf_counter()
    od = O.backproject_direct_columns(q, g, cols)
    t3 = time.perf_counter()
    out = {"fixed_s": t1 - t0, "fourier_col_s": (t2 - t1) / ncols, "direct_col_s": (t3 - t2) / ncols,
           "threads": O.num_threads(), "cols": cols, "fourier": of, "direct": od}
    O.set_num_threads(os.cpu_count() or 1)
    return out


def oracle_baseline(d_cpu: np.ndarray, g, ncols: int) -> dict:
    """cpu_baseline: the oracle's Fourier-form FBP throughput extrapolated to
    the whole volume from its fixed cost and its cost per column (all host
    threads), with the single-thread time and the direct form beside it."""
    s = oracle_sample(d_cpu, g, ncols)
    ncol_all = g.n0 * g.n1
    full_f = s["fixed_s"] + s["fourier_col_s"] * ncol_all
    full_d = s["fixed_s"] + s["direct_col_s"] * ncol_all
    one = oracle_sample(d_cpu, g, 1, seed=8, threads=1)
    full_f1 = one["fixed_s"] + one["fourier_col_s"] * ncol_all
    return {"value": g.nvox / full_f / 1e9, "unit": "GVox/s", "cores": s["threads"], "kind": "oracle",
            "sample": (f"FP64 oracle, Fourier form (exact type-1 sum, detector-space evaluation): filter "
                       f"of all {g.nproj * g.det_h} rows ({s['fixed_s']:.2f} s) + {ncols} whole columns "
                       f"x {g.n2} slices ({s['fourier_col_s']:.3f} s per column), extrapolated to all "
                       f"{ncol_all} columns = {full_f:.0f} s"),
            "fixed_s": s["fixed_s"], "per_column_s": s["fourier_col_s"], "full_volume_s": full_f,
            "single_thread": {"fixed_s": one["fixed_s"], "per_column_s": one["fourier_col_s"],
                              "full_volume_s": full_f1, "gvox_s": g.nvox / full_f1 / 1e9},
            "direct_form": {"per_column_s": s["direct_col_s"], "full_volume_s": full_d,
                            "gvox_s": g.nvox / full_d / 1e9},
            "_sample": s}


# --------------------------------------------------------------------- serving

def run_serving(n: int, rate: float, device: int, seed: int = 5) -> dict:
    """Mixed stream of FBP requests with Poisson arrivals, served live: a client
    thread submits each request at its arrival time to a running server
    (Server.start / submit / stop). Volumes from {128^3, 256^2x128, 512^2x256,
    1024^2x256}, 180-1800 angles, tilt U[10,40] deg, detector width 1.5 x volume
    width, FP16 projections on pinned host memory, Fourier form, volumes copied
    back to pinned host buffers. Each request's input is the first nproj
    projections of one pinned projection set per size class (1800 angles of 40
    ellipsoids): the shapes, transfers and work of the mixed stream, without
    pinning separate data for every request (about 70 GB for 200)."""
    from paper_2401_11101_gb300 import serve as S
    reqs = S.mixed_requests(n, rate, seed)
    t0 = time.perf_counter()
    tmpl = {}
    for r in reqs:
        cls = (r.n0, r.n1, r.n2)
        if cls not in tmpl:
            g = I.Geometry(r.n0, r.n1, r.n2, 1800, r.n2, r.det_w, math.radians(25.0))
            prm = I.ellipsoid_params(g, 40, seed=1000 + len(tmpl), max_axis=max(4.0, r.n2 / 8.0))
            d = I.project_boxed(prm, g, device=f"cuda:{device}", dtype=torch.float32)
            tmpl[cls] = d.half().cpu().pin_memory()
            del d
        r.d = tmpl[cls][: r.nproj]
        r.form = "fourier"
    gen_s = time.perf_counter() - t0
    backend = S.CudaBackend(device, slots=4, keep_volumes=False)
    srv = S.Server(backend, slots=4)
    srv.start()
    start = time.perf_counter()
    for r in reqs:
        wait = r.arrival - (time.perf_counter() - start)
        if wait > 0:
            time.sleep(wait)
        srv.submit(r)
    rep = srv.stop()
    out = rep.summary(reqs)
    out.update({"rate_req_s": rate, "slots": 4, "form": "fourier", "input_generation_s": gen_s,
                "budget_gb": srv.budget / 1e9,
                "mode": "live: a client thread submits at Poisson arrival times while the loop thread runs",
                "workload": "mixed volumes {128^3, 256^2x128, 512^2x256, 1024^2x256}, "
                            "180-1800 angles, tilt U[10,40] deg, det 1.5 n0 x n2, FP16"})
    return out


# --------------------------------------------------------------------- CG

def run_cg(iters: int, device: int) -> dict:
    """CG least squares (Dai-Yuan directions, exact steps) with the Fourier-form
    projector pair on the c4 workload: 256x256x128, 400 angles, det 128x384,
    tilt 30 deg, Gaussian blobs, 0.5 % noise."""
    from paper_2401_11101_gb300 import autograd as A, lamino as L
    g, prm, d = I.make_projections("c4", device=f"cuda:{device}")
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p:
        A.cg_least_squares(p, d, iters=2, form="fourier")        # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mu, hist = A.cg_least_squares(p, d, iters=iters, form="fourier")
        b.record()
        b.synchronize()
        p.status()
        ms = a.elapsed_time(b)
    truth = torch.as_tensor(I.rasterize_blobs(prm, g), dtype=torch.float32, device=mu.device)
    err = float((mu - truth).norm() / truth.norm())
    return {"workload": "c4: " + WORKLOADS["c4"], "form": "fourier", "iterations": len(hist) - 1,
            "ms_total": ms, "ms_per_iter": ms / max(1, len(hist) - 1),
            "residual_ratio": hist[-1] / hist[0], "relL2_vs_phantom": err}


# --------------------------------------------------------------------- arms

def run_reference(args, geom, d):
    """The oracle as it stands on a bounded sample per step (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    d_cpu = d.cpu().numpy()
    ncols = 4
    for _ in range(args.warmup):
        oracle_sample(d_cpu, geom, ncols)
    times, thr = [], 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s = oracle_sample(d_cpu, geom, ncols)
        times.append(time.perf_counter() - t0)
        thr = s["threads"]
    t = sum(times) / len(times)
    vox = ncols * geom.n2
    val = vox / t / 1e9
    sample = (f"FBP of both forms by the FP64 oracle: filter of all {geom.nproj * geom.det_h} rows, "
              f"then the Fourier form (exact type-1 sum) and the direct form on {ncols} whole columns x "
              f"{geom.n2} slices = {vox} voxels per step")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GVox/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": val, "unit": "GVox/s", "cores": thr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GVox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gvox_gap(a: torch.Tensor, b: torch.Tensor) -> float:
    return float((a - b).double().norm() / a.double().norm())


def run_qualifier(plan_kw, dev) -> dict:
    """The metric's qualifier on the band-limited c2b input: both forms on the
    GPU (full volume) and the FP64 oracle's own gap on sampled columns."""
    from paper_2401_11101_gb300 import lamino as L
    g, _, d = I.make_projections("c2b", device=str(dev))
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt, **plan_kw) as p:
        vf = p.fbp(d, form="fourier", kind="shepp")
        vd = p.fbp(d, form="direct", kind="shepp")
        p.status()
    out = {"workload": "c2b: " + WORKLOADS["c2b"], "gap_relL2_gpu": gvox_gap(vf, vd)}
    s = oracle_sample(d.cpu().numpy(), g, 16, seed=43)
    cols = s["cols"]
    gf = np.stack([vf[:, i1, i0].cpu().numpy() for i0, i1 in cols])
    gd = np.stack([vd[:, i1, i0].cpu().numpy() for i0, i1 in cols])
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(a))
    out.update({"gap_relL2_gpu_sampled": rel(gf, gd), "gap_relL2_oracle_sampled": rel(s["fourier"], s["direct"]),
                "fourier_vs_oracle_sampled": rel(s["fourier"], gf), "direct_vs_oracle_sampled": rel(s["direct"], gd),
                "sampled_columns": len(cols)})
    return out


def run_ours(args, geom, d):
    from paper_2401_11101_gb300 import lamino as L
    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    plan_kw = {"z_chunk": args.z_chunk} if args.z_chunk else {}
    plan = L.Plan(geom.n0, geom.n1, geom.n2, geom.nproj, geom.det_w, geom.det_h, geom.tilt, **plan_kw)
    info = plan.info
    vol_f = torch.empty(plan.shape_vol, dtype=torch.float32, device=dev)
    vol_d = torch.empty(plan.shape_vol, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        plan.fbp(d, form="fourier", kind="shepp", out=vol_f)
        if ev:
            ev[1].record(stream)
        plan.fbp(d, form="direct", kind="shepp", out=vol_d)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    plan.status()
    torch.cuda.synchronize(dev)

    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or local) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    clocks = ClockSampler(gpu_index)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    plan.profile(True)
    for i in range(args.steps):
        flush.fill_(1.0)            # L2 flush between timed iterations (outside the events)
        step(evs[i])
    torch.cuda.synchronize(dev)
    recs = plan.profile_read()
    plan.profile(False)
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    plan.status()

    t_f = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    t_d = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    t_f, t_d = max_over_ranks([t_f, t_d], dev)
    nvox = geom.nvox
    value = job_gvox_s(nvox, ws, t_f)
    value_d = job_gvox_s(nvox, ws, t_d)
    gap_gpu = gvox_gap(vol_f, vol_d)

    # per-kernel live timing and roofline
    per = {}
    for name, ms in recs:
        per.setdefault(name, []).append(ms)
    peaks, peaks_src = measured_peaks()
    sm_mhz_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = N_SMS * FP32_LANES_PER_SM * 2 * sm_mhz_max * 1e6 / 1e12  # TFLOP/s
    alg = kernel_algorithmic(info, geom, d.element_size())
    traffic = ncu_traffic(args.workload)
    kernels = {}
    total = sum(sum(v) for v in per.values())
    for name, v in per.items():
        avg = sum(v) / len(v)
        kind, amount = alg.get(name, ("hbm", 0))
        # a z-chunked form launches a kernel once per chunk: the amounts are per step
        steps_launches = len(v) / args.steps
        amount_l = amount / steps_launches
        if kind == "hbm":
            ach = amount_l / (avg * 1e-3) / 1e9
            peak = float(peaks.get("hbm_gbs", 6800.0))
            unit = "GB/s"
        else:
            ach = amount_l / (avg * 1e-3) / 1e12
            peak = alu_peak
            unit = "TFLOP/s"
        kernels[name] = {"launches": len(v), "avg_ms": round(avg, 4), "share": round(sum(v) / total, 4),
                         "bound": kind, "achieved": round(ach, 2), "peak": round(peak, 1), "unit": unit,
                         "frac": round(ach / peak, 4), "algorithmic": amount_l}

    def roof(name):
        k = kernels[name]
        tr = traffic.get(name)
        return {"kernel": name, "bound": k["bound"], "achieved": k["achieved"], "peak": k["peak"],
                "unit": k["unit"], "frac": k["frac"], "traffic": tr,
                "peak_source": f"{peaks_src} ({'hbm_gbs' if k['bound'] == 'hbm' else 'SMs x 128 FP32 lanes x 2 x sm_max_mhz'})"}

    # the headline path is the Fourier form: its dominant kernel is the gridding
    fourier_names = [n for n in kernels if n in ("filter_rowfft", "colfft", "grid", "colifft", "zusfft")]
    dom_f = max(fourier_names, key=lambda n: kernels[n]["share"])
    roofline = roof(dom_f)
    if "grid" in kernels:
        g_ms = kernels["grid"]["avg_ms"]
        taps = grid_taps(info, geom) / (len(per["grid"]) / args.steps)
        red_peak = N_SMS * SMEM_RED_LANES_PER_CLK / 2 * sm_mhz_max * 1e6       # complex taps / s
        ach_taps = taps / (g_ms * 1e-3)
        roofline["bounds"] = {
            "hbm": {"achieved": kernels["grid"]["achieved"], "peak": kernels["grid"]["peak"], "unit": "GB/s",
                    "frac": kernels["grid"]["frac"], "per_launch_bytes": kernels["grid"]["algorithmic"]},
            "smem_reduction": {"achieved": round(ach_taps / 1e9, 1), "peak": round(red_peak / 1e9, 1),
                               "unit": "Gtap/s", "frac": round(ach_taps / red_peak, 4),
                               "per_launch_taps": taps,
                               "peak_source": "152 SMs x 32 shared-memory banks x sm_max_mhz / 2 "
                                              "(one 32-bit reduction per bank and clock; two per complex tap)"}}
    roofline_direct = roof("direct") if "direct" in kernels else None

    # end to end through the C ABI on host buffers (Fourier form)
    e2e = None
    if not args.no_e2e:
        d_host = d.cpu().pin_memory()
        v_host = torch.empty(plan.shape_vol, dtype=torch.float32).pin_memory()
        for _ in range(2):
            plan.fbp_host(d_host, v_host, form="fourier", kind="shepp")
        ts = []
        for _ in range(max(3, min(args.steps, 20))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.fbp_host(d_host, v_host, form="fourier", kind="shepp")
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        # the median of the calls (the metric's statistic): a call now and then
        # stalls on the host side for tens of ms, which the mean would carry
        te, tmean = max_over_ranks([statistics.median(ts), sum(ts) / len(ts)], dev)
        e2e = {"value": job_gvox_s(nvox, ws, te), "unit": "GVox/s",
               "h2d_bytes_per_step": int(d_host.numel() * d_host.element_size()),
               "d2h_bytes_per_step": int(v_host.numel() * v_host.element_size()),
               "ms_per_step": te, "ms_mean": tmean, "calls": len(ts), "statistic": "median"}

    serve = None
    if not args.no_serve:
        serve = run_serving(args.serve_requests, args.serve_rate, local)
    cg = None
    if not args.no_cg:
        cg = run_cg(args.cg_iters, local)
    qual = None
    if not args.no_qualifier and args.workload in ("c2", "c2b"):
        qual = run_qualifier(plan_kw, dev)

    cpu = None
    gap_oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(d.cpu().numpy(), geom, args.cpu_columns)
        s = cpu.pop("_sample")
        cols = s["cols"]
        vf = np.stack([vol_f[:, i1, i0].cpu().numpy() for i0, i1 in cols])
        vd = np.stack([vol_d[:, i1, i0].cpu().numpy() for i0, i1 in cols])
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(a))
        gap_oracle = {"gap_relL2_oracle_sampled": rel(s["fourier"], s["direct"]),
                      "gap_relL2_gpu_sampled": rel(vf, vd),
                      "fourier_vs_oracle_sampled": rel(s["fourier"], vf),
                      "direct_vs_oracle_sampled": rel(s["direct"], vd), "sampled_columns": len(cols)}

    if rank == 0:
        forms = {"fourier": {"gvox_s": value, "ms": t_f},
                 "direct": {"gvox_s": value_d, "ms": t_d, "roofline": roofline_direct},
                 "fourier_over_direct": t_d / t_f,
                 "gap_relL2": gap_gpu}
        if gap_oracle:
            forms.update(gap_oracle)
        line = {"metric": METRIC, "value": value, "unit": "GVox/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_f + t_d, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "storage": str(d.dtype).replace("torch.", ""),
                "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                           "parallelism": f"replicas x{ws} (independent slabs)",
                           "l2": "inputs larger than L2 and a 256 MB L2 flush between steps",
                           "usfft": {"R": 2, "w_xy": info["usfft_w"], "w_z": info["usfft_wz"],
                                     "err_est": info["usfft_err_est"]},
                           "z_chunk": info["z_chunk"], "plane_chunk": info["plane_chunk"]},
                "forms": forms, "qualifier": qual,
                "roofline": roofline,
                "kernels": kernels, "gpu_launches": len(recs),
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "serve": serve, "cg": cg}
        print(json.dumps(line), flush=True)
    plan.close()


def main():
    args = parse()
    ws, rank, local = dist_env()
    if ws > 1:
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    cfg = I.CONFIGS[args.workload]
    if args.impl == "reference":
        if rank == 0:
            dev = "cuda" if torch.cuda.is_available() else "cpu"
            geom, _, d = I.make_projections(args.workload, device=dev)
            run_reference(args, geom, d)
    else:
        torch.cuda.set_device(local)
        # every replica reconstructs its own specimen (seed offset by rank)
        geom, _, d = I.make_projections(args.workload, device=f"cuda:{local}", slab=rank)
        d = d.to(I.storage_dtype(args.workload)).contiguous()
        run_ours(args, geom, d)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
