"""Continuous-batching reconstruction server for laminographic FBP requests.

Requests (projections of one slab, any size, angle count and tilt) arrive over
time. The server admits a waiting request as soon as an execution slot (a CUDA
stream) is free and its HBM footprint fits the budget (plan tables + the
form's workspace from lamino_workspace_bytes + input + output), backfilling
past a request that does not fit yet. Admitted requests run concurrently on
their slot streams, so the kernels of different requests overlap on the GPU.

Each slot owns a workspace arena that it lends to the plan it runs
(lamino_set_workspace), so plans allocate no workspace of their own: plans
(device tables only) stay resident in a pool keyed by geometry after their
request finishes, and an arena grows only when a larger request comes. Idle
plans and the arenas of idle slots count against the budget: when a request
would not fit, idle plans are closed least recently used first (never the one
the request is about to reuse), then idle arenas are released, and the pool is
capped in size. Apart from closing a plan, nothing in the loop frees device
memory or waits for the whole device. A request in form "auto" runs the
Fourier form, z-chunked (Sec. 5: k_v-plane chunks of the 2D USFFT) as finely
as needed to fit the budget, and falls back to the direct form only if no
chunking fits.

Completion is detected by polling CUDA events. A request that does not finish
within `timeout_s` is reported as timed out at once, but its slot and its
bytes stay charged until its device work has actually finished (the kernels
may still be using its buffers).

Two ways to drive it: `run(requests)` replays a list of requests with given
arrival times; `start()`, `submit(request)` (from any thread, while others run)
and `stop()` serve a live stream from a background loop thread, and every
`submit` returns the request's Outcome, whose `wait()` blocks until it is
decided. The scheduling logic is independent of CUDA: the server drives a
backend with `footprint / submit / poll / collect / release` (plus the
optional `idle_bytes / evict`); `CudaBackend` is the real one.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
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
    form: str = "fourier"          # "fourier", "direct", or "auto" (Fourier, z-chunked to fit)
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
    status: str                    # "pending", "ok", "rejected", "timeout", "error"
    arrival: float
    admitted: float = float("nan")
    done: float = float("nan")
    volume: object = None
    message: str = ""
    form: str = ""                 # the form it ran in ("fourier/z64": z-chunked by 64 planes)
    _event: threading.Event = dataclasses.field(default_factory=threading.Event, repr=False)

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def finish(self):
        self._event.set()

    def wait(self, timeout: float | None = None) -> bool:
        """Block until the outcome is decided (True) or `timeout` passes."""
        return self._event.wait(timeout)


@dataclasses.dataclass
class Report:
    outcomes: list
    wall_s: float
    busy_s: float
    timeline: list = dataclasses.field(default_factory=list)   # (t, queued, inflight, draining, GB charged, GB idle)

    def latencies_ms(self):
        return np.array([o.latency * 1e3 for o in self.outcomes if o.status == "ok"])

    def summary(self, requests) -> dict:
        lat = self.latencies_ms()
        vox = sum(r.nvox for r, o in zip(requests, self.outcomes) if o.status == "ok")
        tl = self.timeline
        step = max(1, len(tl) // 40)
        return {
            "requests": len(self.outcomes),
            "ok": int(sum(o.status == "ok" for o in self.outcomes)),
            "rejected": int(sum(o.status == "rejected" for o in self.outcomes)),
            "timeout": int(sum(o.status == "timeout" for o in self.outcomes)),
            "error": int(sum(o.status == "error" for o in self.outcomes)),
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p90_ms": float(np.percentile(lat, 90)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_ms": float(lat.mean()) if len(lat) else None,
            "queue_wait_p50_ms": float(np.percentile([(o.admitted - o.arrival) * 1e3 for o in self.outcomes
                                                      if o.status == "ok"], 50)) if len(lat) else None,
            "gvox_s": vox / self.wall_s / 1e9 if self.wall_s > 0 else None,
            # the stream's own rate: all requests' voxels over the arrival span
            # (a server that keeps up delivers about this much)
            "offered_gvox_s": (sum(r.nvox for r in requests) / max(o.arrival for o in self.outcomes) / 1e9
                               if self.outcomes and max(o.arrival for o in self.outcomes) > 0 else None),
            "wall_s": self.wall_s,
            "busy_s": self.busy_s,
            "queued_max": max((s[1] for s in tl), default=0),
            "inflight_max": max((s[2] for s in tl), default=0),
            "forms": dict(collections.Counter(o.form for o in self.outcomes if o.status == "ok")),
            "timeline": [[round(s[0], 3), s[1], s[2], s[3], round(s[4], 3), round(s[5], 3)] for s in tl[::step]],
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
        self._lock = threading.Lock()
        self._incoming = collections.deque()
        self._thread = None
        self._stopping = False
        self._live = []
        self._reset()

    # ------------------------------------------------------------ state
    def _reset(self):
        self.t0 = self.clock()
        self.waiting = collections.deque()     # (request, outcome)
        self.inflight = []                     # (request, handle, slot, bytes, outcome)
        self.draining = []                     # timed out, device work still running
        self.free = list(range(self.slots))
        self.used = 0                          # bytes charged to admitted requests
        self.busy = 0.0
        self._last = self.t0
        self.timeline = []

    def _now(self) -> float:
        return self.clock() - self.t0

    def _idle(self, r=None) -> int:
        f = getattr(self.backend, "idle_bytes", None)
        return f(r) if f else 0

    def _sample(self):
        s = (self._now(), len(self.waiting), len(self.inflight), len(self.draining),
             self.used / 1e9, self._idle() / 1e9)
        if not self.timeline or self.timeline[-1][1:] != s[1:]:
            self.timeline.append(s)

    # ------------------------------------------------------------ steps
    def _arrive(self, r, o):
        need = self.backend.footprint(r)
        if need > self.budget:
            o.status, o.done = "rejected", self._now()
            o.message = f"needs {need} bytes, budget {self.budget}"
            o.finish()
        else:
            self.waiting.append((r, o))

    def _admit(self):
        # the first waiting request that fits (backfill past those that do not)
        progressed = True
        while progressed and self.waiting and self.free:
            progressed = False
            for i, (r, o) in enumerate(self.waiting):
                need = self.backend.footprint(r)
                if self.used + need + self._idle(r) > self.budget and hasattr(self.backend, "evict"):
                    # close idle plans, least recently used first, keeping the one r reuses
                    self.backend.evict(self.budget - self.used - need, r)
                if self.used + need + self._idle(r) > self.budget:
                    continue
                del self.waiting[i]
                slot = self.free.pop()
                try:
                    h = self.backend.submit(r, slot)
                except Exception as e:          # reported, not raised
                    o.status, o.done, o.message = "error", self._now(), str(e)
                    o.finish()
                    self.free.append(slot)
                    progressed = True
                    break
                o.admitted = self._now()
                o.form = h.get("form", r.form) if isinstance(h, dict) else r.form
                self.inflight.append((r, h, slot, need, o))
                self.used += need
                progressed = True
                break

    def _complete(self):
        still = []
        for r, h, slot, need, o in self.inflight:
            tnow = self._now()
            if self.backend.poll(h):
                try:
                    o.volume = self.backend.collect(h)
                    o.status = "ok"
                except Exception as e:          # e.g. a bounded device wait expired
                    o.status, o.message = "error", str(e)
                o.done = self._now()
                o.finish()
                self.backend.release(h)
                self.free.append(slot)
                self.used -= need
            elif tnow - o.admitted > self.timeout_s:
                o.status, o.done = "timeout", tnow
                o.message = f"not complete after {self.timeout_s} s"
                o.finish()
                # its kernels may still use its buffers: slot and bytes stay charged
                self.draining.append((r, h, slot, need, o))
            else:
                still.append((r, h, slot, need, o))
        self.inflight = still
        still = []
        for r, h, slot, need, o in self.draining:
            if self.backend.poll(h):
                self.backend.release(h)
                self.free.append(slot)
                self.used -= need
            else:
                still.append((r, h, slot, need, o))
        self.draining = still

    def _tick(self):
        now = self.clock()
        if self.inflight:
            self.busy += now - self._last
        self._last = now
        self._admit()
        self._complete()
        self._sample()

    # ------------------------------------------------------------ replay
    def run(self, requests) -> Report:
        """Serve a scripted stream: each request enters at its `arrival` time.
        Returns when every request is decided (timed-out work may still be
        draining; see `draining`)."""
        self._reset()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        outcomes = [Outcome(r.rid, "pending", r.arrival) for r in requests]
        by_rid = {r.rid: o for r, o in zip(requests, outcomes)}
        while pending or self.waiting or self.inflight:
            now = self._now()
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                self._arrive(r, by_rid[r.rid])
            self._tick()
            if self.inflight or (self.waiting and not self.free):
                self.sleep(self.poll_s)
            elif pending and not self.waiting:
                # idle until the next arrival
                self.sleep(max(0.0, min(self.poll_s * 50, pending[0].arrival - self._now())))
        return Report(outcomes, self._now(), self.busy, list(self.timeline))

    # ------------------------------------------------------------ live
    def start(self):
        """Start the loop thread; requests then enter through submit()."""
        if self._thread is not None:
            raise RuntimeError("server already running")
        self._reset()
        self._stopping = False
        self._live = []
        self._thread = threading.Thread(target=self._serve, name="lamino-serve", daemon=True)
        self._thread.start()

    def submit(self, r: Request) -> Outcome:
        """Enqueue a request now (any thread); its arrival time is set to now."""
        if self._thread is None:
            raise RuntimeError("server not started")
        with self._lock:
            r.arrival = self._now()
            o = Outcome(r.rid, "pending", r.arrival)
            self._incoming.append((r, o))
            self._live.append((r, o))
        return o

    def stop(self, timeout: float | None = None) -> Report:
        """Finish every submitted request, stop the loop thread and report."""
        self._stopping = True
        self._thread.join(timeout)
        self._thread = None
        outs = [o for _, o in self._live]
        return Report(outs, self._now(), self.busy, list(self.timeline))

    def _serve(self):
        while True:
            with self._lock:
                batch = list(self._incoming)
                self._incoming.clear()
            for r, o in batch:
                self._arrive(r, o)
            self._tick()
            with self._lock:
                idle = not self._incoming
            if self._stopping and idle and not self.waiting and not self.inflight:
                return
            self.sleep(self.poll_s if (self.inflight or self.waiting) else self.poll_s * 10)


class CudaBackend:
    """Runs requests with liblamino on one GPU, one CUDA stream per slot.

    Plans stay in an idle pool (LRU, at most `max_idle_plans`) between
    requests; their workspaces are the slots' arenas. With `keep_volumes` every
    result is copied into its own pinned host tensor; otherwise into a pinned
    buffer owned by the request's slot, valid until that slot's next request."""

    def __init__(self, device: int = 0, slots: int = 4, keep_volumes: bool = True,
                 max_idle_plans: int = 1024):
        import torch
        from . import lamino as L
        self.torch, self.L = torch, L
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.idle = collections.OrderedDict()     # geometry key -> [Plan] (LRU order)
        self.keep_volumes = keep_volumes
        self.max_idle_plans = max_idle_plans
        self.slot_out = [None] * slots
        self.arena = [None] * slots                # per-slot workspace lent to the running plan
        self.busy_slots = set()
        self.budget = None                         # set by the Server
        self._ws = {}
        self._planes = {}
        self.draining = []                         # handles released before their work finished

    def default_budget(self) -> int:
        free, total = self.torch.cuda.mem_get_info(self.device)
        return int(0.8 * free)

    # ------------------------------------------------------------ plan pool
    def _to_idle(self, pk, plan):
        self.idle.setdefault(pk, []).append(plan)
        self.idle.move_to_end(pk)
        while sum(len(v) for v in self.idle.values()) > self.max_idle_plans:
            self._close_lru()

    def _close_lru(self, keep=None):
        for pk, lst in self.idle.items():
            if pk == keep and len(lst) <= 1:
                continue
            lst.pop(0).close()
            if not lst:
                del self.idle[pk]
            return True
        return False

    def _drain(self):
        # plans of requests released with work in flight rejoin the pool once it has finished
        still = []
        for h in self.draining:
            if h["ev"].query():
                self._idle_plan(h)
            else:
                still.append(h)
        self.draining = still

    def _new_plan(self, r: Request):
        with self.torch.cuda.device(self.device):
            return self.L.Plan(r.n0, r.n1, r.n2, r.nproj, r.det_w, r.det_h, r.tilt)

    def _plan(self, r: Request, zc: int):
        """An idle plan of r's geometry (or a new one) set to z chunking zc;
        plans hold no workspace (the slots lend theirs), so the chunking
        changes without freeing anything."""
        self._drain()
        lst = self.idle.get(r.key)
        if lst:
            p = lst.pop()
            if not lst:
                del self.idle[r.key]
        else:
            p = self._new_plan(r)
        if p.info["z_chunk"] != zc:
            p.set_z_chunk(zc)
        return p

    def _idle_arenas(self) -> int:
        return sum(a.numel() for i, a in enumerate(self.arena) if a is not None and i not in self.busy_slots)

    def idle_bytes(self, r: Request | None = None) -> int:
        """Device bytes held by idle plans (not counting one plan that `r` would
        reuse) and by the arenas of idle slots."""
        keep = r.key if r is not None else None
        total, skipped = 0, False
        for pk, lst in self.idle.items():
            for p in lst:
                if pk == keep and not skipped:
                    skipped = True
                    continue
                total += p.device_bytes()
        return total + self._idle_arenas()

    def evict(self, target_idle: int, r: Request | None = None):
        """Close idle plans, least recently used first, then release the arenas
        of idle slots, until the idle bytes (without the plan `r` would reuse)
        are at most `target_idle`."""
        keep = r.key if r is not None else None
        while self.idle and self.idle_bytes(r) > max(0, target_idle):
            if not self._close_lru(keep):
                break
        for i in sorted(range(len(self.arena)), key=lambda i: -(self.arena[i].numel() if self.arena[i] is not None else 0)):
            if self.idle_bytes(r) <= max(0, target_idle):
                break
            if i not in self.busy_slots:
                self.arena[i] = None

    # ------------------------------------------------------------ footprints
    def _form_bytes(self, r: Request, form: str, zc: int = 0) -> int:
        """Footprint of r in one form: plan tables + workspace + input + output.
        The plan that answers joins the idle pool for r to use (creating and
        closing a plan here would wait for the whole device)."""
        esz = 2 if r.d is None else r.d.element_size()
        key = (r.key, form, zc, esz)
        if key not in self._ws:
            lst = self.idle.get(r.key)
            p = lst[-1] if lst else None
            if p is None:
                p = self._new_plan(r)
                self._to_idle(r.key, p)
            keep = p.info["z_chunk"]
            p.set_z_chunk(zc)                # no workspace is held: nothing is freed
            ws = p.workspace_bytes(form)
            p.set_z_chunk(keep)
            self._planes[r.key] = p.info["planes"]
            self._ws[key] = p.device_bytes() + ws + r.nproj * r.det_h * r.det_w * (esz + 4) + 4 * r.nvox
        return self._ws[key]

    def form_of(self, r: Request):
        """(form, z_chunk) a request runs with. "auto": the Fourier form,
        unchunked if it fits the budget, else in the largest k_v-plane chunks
        (halving down to 8 planes) that fit, else the direct form."""
        if r.form != "auto":
            return r.form, 0
        if self.budget is None or self._form_bytes(r, "fourier") <= self.budget:
            return "fourier", 0
        zc = self._planes.get(r.key) or 0
        while zc > 8:
            zc //= 2
            if self._form_bytes(r, "fourier", zc) <= self.budget:
                return "fourier", zc
        return "direct", 0

    def footprint(self, r: Request) -> int:
        form, zc = self.form_of(r)
        return self._form_bytes(r, form, zc)

    # ------------------------------------------------------------ execution
    def _out_buffer(self, slot: int, shape):
        torch = self.torch
        n = math.prod(shape)
        buf = self.slot_out[slot]
        if buf is None or buf.numel() < n:
            buf = torch.empty(n, dtype=torch.float32, pin_memory=True)
            self.slot_out[slot] = buf
        return buf[:n].view(shape)

    def _arena_for(self, slot: int, nbytes: int):
        a = self.arena[slot]
        if a is None or a.numel() < nbytes:
            # the slot's previous request has finished (its slot was free): the old
            # arena goes back to the allocator before the larger one is taken
            self.arena[slot] = None
            with self.torch.cuda.device(self.device), self.torch.cuda.stream(self.streams[slot]):
                a = self.torch.empty(max(nbytes, 256), dtype=self.torch.uint8, device=self.device)
            self.arena[slot] = a
        return a

    def submit(self, r: Request, slot: int):
        torch = self.torch
        s = self.streams[slot]
        form, zc = self.form_of(r)
        p = self._plan(r, zc)
        self.busy_slots.add(slot)
        p.set_workspace(self._arena_for(slot, p.workspace_bytes(form)))
        with torch.cuda.device(self.device), torch.cuda.stream(s):
            d = r.d.to(self.device, non_blocking=True)
            vol = torch.empty(p.shape_vol, dtype=torch.float32, device=self.device)
            p.fbp(d, form=form, kind=r.kind, out=vol)
            if self.keep_volumes:
                host = torch.empty(p.shape_vol, dtype=torch.float32, pin_memory=True)
            else:
                host = self._out_buffer(slot, p.shape_vol)
            host.copy_(vol, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return {"req": r, "plan": p, "pkey": r.key, "ev": ev, "d": d, "vol": vol, "host": host,
                "stream": s, "slot": slot, "form": form if not zc else f"{form}/z{zc}"}

    def poll(self, h) -> bool:
        return h["ev"].query()

    def collect(self, h):
        h["plan"].status()          # raises if a bounded device wait expired
        return h["host"]

    def release(self, h):
        h["d"].record_stream(h["stream"])
        h["vol"].record_stream(h["stream"])
        if not h["ev"].query():
            # work still in flight may use the plan's tables and the slot's
            # arena: both stay out of reuse until it has finished
            self.draining.append(h)
            return
        self._idle_plan(h)

    def _idle_plan(self, h):
        if hasattr(h["plan"], "set_workspace"):
            h["plan"].set_workspace(None)          # the arena stays with the slot
        self.busy_slots.discard(h.get("slot"))
        self._to_idle(h["pkey"], h["plan"])


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
