"""Continuous-batching reconstruction server for laminographic FBP requests.

Requests (projections of one slab, any size, angle count and tilt) arrive over
time. The server admits a waiting request as soon as an execution slot (a CUDA
stream) is free and its HBM footprint fits the budget (plan tables + the
form's workspace from lamino_workspace_bytes + input + output), backfilling
past a request that does not fit yet. Admitted requests run concurrently on
their slot streams, so the kernels of different requests overlap on the GPU.
Plans (with their device tables and workspaces) stay resident in a cache keyed
by geometry and are evicted least-recently-used when memory is needed.
Completion is detected by polling CUDA events; a request that does not finish
within `timeout_s` is reported as timed out instead of blocking the loop.

The scheduling logic is independent of CUDA: `Server` drives a backend with
`footprint / submit / poll / collect / release`; `CudaBackend` is the real one.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    n0: int
    n1: int
    n2: int
    nproj: int
    det_w: int
    det_h: int
    tilt: float
    arrival: float                 # seconds after the start of the run
    d: object = None               # projections (host tensor, ideally pinned)
    form: str = "fourier"          # "fourier", "direct", or "auto" (Fourier if it fits the budget)
    kind: str = "shepp"

    @property
    def key(self):
        return (self.n0, self.n1, self.n2, self.nproj, self.det_w, self.det_h, round(self.tilt, 12))

    @property
    def nvox(self) -> int:
        return self.n0 * self.n1 * self.n2


@dataclasses.dataclass
class Outcome:
    rid: int
    status: str                    # "ok", "rejected", "timeout", "error"
    arrival: float
    admitted: float = float("nan")
    done: float = float("nan")
    volume: object = None
    message: str = ""

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclasses.dataclass
class Report:
    outcomes: list
    wall_s: float
    busy_s: float

    def latencies_ms(self):
        return np.array([o.latency * 1e3 for o in self.outcomes if o.status == "ok"])

    def summary(self, requests) -> dict:
        lat = self.latencies_ms()
        vox = sum(r.nvox for r, o in zip(requests, self.outcomes) if o.status == "ok")
        return {
            "requests": len(self.outcomes),
            "ok": int(sum(o.status == "ok" for o in self.outcomes)),
            "rejected": int(sum(o.status == "rejected" for o in self.outcomes)),
            "timeout": int(sum(o.status == "timeout" for o in self.outcomes)),
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_ms": float(lat.mean()) if len(lat) else None,
            "gvox_s": vox / self.wall_s / 1e9 if self.wall_s > 0 else None,
            "wall_s": self.wall_s,
        }


class Server:
    """Admission, scheduling and completion tracking (backend-agnostic)."""

    def __init__(self, backend, slots: int = 4, budget_bytes: int | None = None,
                 timeout_s: float = 120.0, poll_s: float = 2e-4, clock=time.perf_counter,
                 sleep=time.sleep):
        self.backend = backend
        self.slots = slots
        self.budget = budget_bytes if budget_bytes is not None else backend.default_budget()
        if hasattr(backend, "budget"):
            backend.budget = self.budget      # lets "auto" requests choose a form that fits
        self.timeout_s = timeout_s
        self.poll_s = poll_s
        self.clock = clock
        self.sleep = sleep

    def run(self, requests) -> Report:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        order = {r.rid: i for i, r in enumerate(requests)}
        outcomes = [Outcome(r.rid, "pending", r.arrival) for r in requests]
        waiting = collections.deque()
        inflight = []                   # (request, handle, slot, bytes)
        free = list(range(self.slots))
        used = 0
        t0 = self.clock()
        busy = 0.0
        last = t0
        while pending or waiting or inflight:
            now = self.clock() - t0
            if inflight:
                busy += (self.clock() - last)
            last = self.clock()
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                need = self.backend.footprint(r)
                if need > self.budget:
                    o = outcomes[order[r.rid]]
                    o.status, o.done = "rejected", now
                    o.message = f"needs {need} bytes, budget {self.budget}"
                else:
                    waiting.append(r)
            # admit: first waiting request that fits (backfill)
            progressed = True
            while progressed and waiting and free:
                progressed = False
                for i, r in enumerate(waiting):
                    need = self.backend.footprint(r)
                    if used + need <= self.budget or (not inflight and need <= self.budget):
                        if used + need > self.budget:
                            self.backend.evict(self.budget - need)
                        del waiting[i]
                        slot = free.pop()
                        try:
                            h = self.backend.submit(r, slot)
                        except Exception as e:          # pragma: no cover - reported, not raised
                            o = outcomes[order[r.rid]]
                            o.status, o.done, o.message = "error", self.clock() - t0, str(e)
                            free.append(slot)
                            progressed = True
                            break
                        outcomes[order[r.rid]].admitted = self.clock() - t0
                        inflight.append((r, h, slot, need))
                        used += need
                        progressed = True
                        break
            # completions
            still = []
            for r, h, slot, need in inflight:
                o = outcomes[order[r.rid]]
                tnow = self.clock() - t0
                if self.backend.poll(h):
                    o.volume = self.backend.collect(h)
                    o.status, o.done = "ok", self.clock() - t0
                elif tnow - o.admitted > self.timeout_s:
                    o.status, o.done = "timeout", tnow
                    o.message = f"not complete after {self.timeout_s} s"
                else:
                    still.append((r, h, slot, need))
                    continue
                self.backend.release(h)
                free.append(slot)
                used -= need
            inflight = still
            if inflight or (waiting and not free):
                self.sleep(self.poll_s)
            elif pending and not waiting:
                # idle until the next arrival
                self.sleep(max(0.0, min(self.poll_s * 50, pending[0].arrival - (self.clock() - t0))))
        return Report(outcomes, self.clock() - t0, busy)


class CudaBackend:
    """Runs requests with liblamino on one GPU, one CUDA stream per slot.

    A request with form "auto" runs the Fourier form when its HBM footprint
    fits the server's budget and falls back to the direct form (projections,
    filtered rows and volume only) when it does not."""

    def __init__(self, device: int = 0, slots: int = 4, keep_volumes: bool = True):
        import torch
        from . import lamino as L
        self.torch, self.L = torch, L
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.idle = collections.OrderedDict()     # key -> [Plan] (LRU order)
        self.keep_volumes = keep_volumes
        self.budget = None                         # set by the Server
        self._ws = {}
        self.draining = []                         # handles released before their work finished

    def default_budget(self) -> int:
        free, total = self.torch.cuda.mem_get_info(self.device)
        return int(0.8 * free)

    def _to_idle(self, key, plan):
        self.idle.setdefault(key, []).append(plan)
        self.idle.move_to_end(key)

    def _drain(self):
        # plans of timed-out requests rejoin the pool once their work has finished
        still = []
        for h in self.draining:
            if h["ev"].query():
                self._to_idle(h["req"].key, h["plan"])
            else:
                still.append(h)
        self.draining = still

    def _plan(self, r: Request):
        self._drain()
        lst = self.idle.get(r.key)
        if lst:
            p = lst.pop()
            self.idle.move_to_end(r.key)
            return p
        with self.torch.cuda.device(self.device):
            return self.L.Plan(r.n0, r.n1, r.n2, r.nproj, r.det_w, r.det_h, r.tilt)

    def _form_bytes(self, r: Request, form: str) -> int:
        esz = 2 if r.d is None else r.d.element_size()
        key = (r.key, form, esz)
        if key not in self._ws:
            with self.torch.cuda.device(self.device):
                p = self._plan(r)
                ws = p.workspace_bytes(form)
                self.idle.setdefault(r.key, []).append(p)
            self._ws[key] = ws + r.nproj * r.det_h * r.det_w * (esz + 4) + 4 * r.nvox
        return self._ws[key]

    def form_of(self, r: Request) -> str:
        """The form a request runs in ("auto": Fourier unless it exceeds the budget)."""
        if r.form != "auto":
            return r.form
        if self.budget is None or self._form_bytes(r, "fourier") <= self.budget:
            return "fourier"
        return "direct"

    def footprint(self, r: Request) -> int:
        return self._form_bytes(r, self.form_of(r))

    def evict(self, target_free: int):
        # drop idle plans (tables + workspaces) least recently used first
        while self.idle:
            key, lst = next(iter(self.idle.items()))
            while lst:
                lst.pop().close()
            del self.idle[key]
            free, _ = self.torch.cuda.mem_get_info(self.device)
            if free >= target_free:
                break

    def submit(self, r: Request, slot: int):
        torch = self.torch
        s = self.streams[slot]
        p = self._plan(r)
        with torch.cuda.device(self.device), torch.cuda.stream(s):
            d = r.d.to(self.device, non_blocking=True)
            vol = torch.empty(p.shape_vol, dtype=torch.float32, device=self.device)
            p.fbp(d, form=self.form_of(r), kind=r.kind, out=vol)
            host = None
            if self.keep_volumes:
                host = torch.empty(p.shape_vol, dtype=torch.float32, pin_memory=True)
                host.copy_(vol, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return {"req": r, "plan": p, "ev": ev, "d": d, "vol": vol, "host": host, "stream": s}

    def poll(self, h) -> bool:
        return h["ev"].query()

    def collect(self, h):
        h["plan"].status()          # raises if a bounded device wait expired
        return h["host"]

    def release(self, h):
        h["d"].record_stream(h["stream"])
        h["vol"].record_stream(h["stream"])
        if not h["ev"].query():
            # a timed-out request: its kernels may still use the plan's
            # workspaces, so the plan stays out of the pool until they finish
            self.draining.append(h)
            return
        self._to_idle(h["req"].key, h["plan"])


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process with `rate` requests per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def mixed_requests(n: int, rate: float, seed: int, sizes=((128, 128, 128), (256, 256, 128),
                                                          (512, 512, 256), (1024, 1024, 256)),
                   nproj=(180, 1800), tilt_deg=(10.0, 40.0)):
    """A stream shaped like the mixed serving workload: volume sizes drawn
    uniformly from `sizes`, angle counts U{nproj}, tilts U[tilt_deg], detector
    width 1.5 x volume width and height = slab thickness (projections attached
    by the caller)."""
    rng = np.random.default_rng(seed + 1)
    t = poisson_arrivals(n, rate, seed)
    out = []
    for i in range(n):
        n0, n1, n2 = sizes[rng.integers(len(sizes))]
        k = int(rng.integers(nproj[0], nproj[1] + 1))
        phi = math.radians(float(rng.uniform(*tilt_deg)))
        out.append(Request(i, n0, n1, n2, k, int(1.5 * n0) // 2 * 2, n2, phi, float(t[i])))
    return out
