"""Serving: admission by HBM footprint, backfill, slots, timeouts, idle-plan
eviction and live submission (CPU, with fake backends) and, on the GPU, that
every request's result is the same alone and in a mixed stream and that an
"auto" request is z-chunked to fit the budget."""
import collections
import math
import threading
import time

import numpy as np
import pytest
import torch

from paper_2401_11101_gb300 import serve as S


class FakeBackend:
    """Jobs finish a fixed number of polls after submission; never = stuck;
    `unstick_after` polls of a stuck job end it anyway (work that outlives its
    timeout)."""

    def __init__(self, sizes, durations, stuck=(), unstick_after=None):
        self.sizes, self.durations, self.stuck = sizes, durations, set(stuck)
        self.unstick_after = unstick_after
        self.log = []
        self.concurrent = 0
        self.max_concurrent = 0

    def default_budget(self):
        return 100

    def footprint(self, r):
        return self.sizes[r.rid]

    def evict(self, target, r=None):
        self.log.append(("evict", target))

    def submit(self, r, slot):
        self.concurrent += 1
        self.max_concurrent = max(self.max_concurrent, self.concurrent)
        self.log.append(("submit", r.rid, slot))
        return {"r": r, "left": self.durations[r.rid]}

    def poll(self, h):
        if h["r"].rid in self.stuck:
            h["polls"] = h.get("polls", 0) + 1
            return self.unstick_after is not None and h["polls"] >= self.unstick_after
        h["left"] -= 1
        return h["left"] <= 0

    def collect(self, h):
        return f"vol{h['r'].rid}"

    def release(self, h):
        self.concurrent -= 1
        self.log.append(("release", h["r"].rid))


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


def _req(i, arrival):
    return S.Request(i, 8, 8, 8, 4, 12, 8, 0.3, arrival)


def test_fifo_slots_and_completion():
    clk = FakeClock()
    be = FakeBackend(sizes=[10] * 6, durations=[3] * 6)
    srv = S.Server(be, slots=2, budget_bytes=100, clock=clk, sleep=clk.sleep)
    rep = srv.run([_req(i, 0.0) for i in range(6)])
    assert [o.status for o in rep.outcomes] == ["ok"] * 6
    assert be.max_concurrent == 2
    assert [o.volume for o in rep.outcomes] == [f"vol{i}" for i in range(6)]


def test_admission_by_memory_and_backfill():
    clk = FakeClock()
    # request 0 holds 70 of 100 bytes; request 1 (50) must wait, request 2 (20) backfills
    be = FakeBackend(sizes=[70, 50, 20], durations=[20, 2, 2])
    srv = S.Server(be, slots=3, budget_bytes=100, clock=clk, sleep=clk.sleep)
    rep = srv.run([_req(0, 0.0), _req(1, 0.0), _req(2, 0.0)])
    subs = [e[1] for e in be.log if e[0] == "submit"]
    assert subs == [0, 2, 1]
    assert all(o.status == "ok" for o in rep.outcomes)
    assert rep.outcomes[1].admitted >= rep.outcomes[0].done


def test_oversize_request_rejected_and_timeout_reported():
    clk = FakeClock()
    be = FakeBackend(sizes=[10, 500, 10], durations=[1, 1, 1], stuck={2})
    srv = S.Server(be, slots=2, budget_bytes=100, timeout_s=0.05, clock=clk, sleep=clk.sleep)
    rep = srv.run([_req(0, 0.0), _req(1, 0.001), _req(2, 0.002)])
    st = [o.status for o in rep.outcomes]
    assert st == ["ok", "rejected", "timeout"]
    assert "budget" in rep.outcomes[1].message
    # the stuck job is reported at its deadline, but its slot and bytes stay
    # charged (its kernels may still use its buffers)
    assert be.concurrent == 1 and srv.used == 10 and len(srv.draining) == 1


def test_timed_out_bytes_stay_charged_until_the_work_finishes():
    clk = FakeClock()
    # job 0 (60 of 100 bytes) times out after 0.05 s but runs until its 2000th
    # poll; job 1 (60 bytes) arrives after the timeout and must wait for it
    be = FakeBackend(sizes=[60, 60], durations=[1, 1], stuck={0}, unstick_after=2000)
    srv = S.Server(be, slots=2, budget_bytes=100, timeout_s=0.05, clock=clk, sleep=clk.sleep)
    rep = srv.run([_req(0, 0.0), _req(1, 0.1)])
    assert [o.status for o in rep.outcomes] == ["timeout", "ok"]
    released = [i for i, e in enumerate(be.log) if e == ("release", 0)]
    submitted = [i for i, e in enumerate(be.log) if e[0] == "submit" and e[1] == 1]
    assert released and submitted and released[0] < submitted[0]
    assert srv.used == 0 and not srv.draining


def test_timed_out_plan_rejoins_the_pool_only_after_its_work_finishes():
    # CudaBackend.release without a GPU: events and tensors are stand-ins
    import collections

    class Ev:
        def __init__(self):
            self.done = False

        def query(self):
            return self.done

    class Buf:
        def record_stream(self, s):
            pass

    b = S.CudaBackend.__new__(S.CudaBackend)
    b.idle, b.draining, b.max_idle_plans, b.busy_slots = collections.OrderedDict(), [], 16, set()
    r = S.Request(0, 8, 8, 8, 4, 12, 8, 0.3, 0.0)
    pk = (r.key, 0)
    ev, plan = Ev(), object()
    b.release({"req": r, "plan": plan, "pkey": pk, "ev": ev, "d": Buf(), "vol": Buf(), "host": None,
               "stream": None})
    assert pk not in b.idle and len(b.draining) == 1
    b._drain()
    assert pk not in b.idle
    ev.done = True
    b._drain()
    assert b.idle[pk] == [plan] and not b.draining
    ev2 = Ev()
    ev2.done = True
    plan2 = object()
    b.release({"req": r, "plan": plan2, "pkey": pk, "ev": ev2, "d": Buf(), "vol": Buf(), "host": None,
               "stream": None})
    assert b.idle[pk] == [plan, plan2]


class PoolBackend(FakeBackend):
    """A fake backend whose finished jobs leave a plan of `plan_bytes` idle per
    distinct geometry key (like CudaBackend's plan pool)."""

    def __init__(self, sizes, durations, plan_bytes):
        super().__init__(sizes, durations)
        self.plan_bytes = plan_bytes
        self.idle = collections.OrderedDict()    # key -> bytes
        self.closed = []

    def release(self, h):
        super().release(h)
        self.idle[h["r"].key] = self.plan_bytes
        self.idle.move_to_end(h["r"].key)

    def idle_bytes(self, r=None):
        return sum(b for k, b in self.idle.items() if r is None or k != r.key)

    def evict(self, target, r=None):
        for k in list(self.idle):
            if self.idle_bytes(r) <= max(0, target):
                break
            if r is not None and k == r.key:
                continue
            del self.idle[k]
            self.closed.append(k)


def test_idle_plans_count_against_the_budget_and_are_evicted_lru():
    clk = FakeClock()
    # every request has a new geometry; each finished one leaves a 30-byte
    # plan idle. With a 100-byte budget and 40-byte requests at most one
    # older plan can stay: the least recently used ones are closed.
    reqs = [S.Request(i, 8 + 2 * i, 8, 8, 4, 12, 8, 0.3, 0.01 * i) for i in range(6)]
    be = PoolBackend(sizes=[40] * 6, durations=[2] * 6, plan_bytes=30)
    srv = S.Server(be, slots=1, budget_bytes=100, clock=clk, sleep=clk.sleep)
    rep = srv.run(reqs)
    assert all(o.status == "ok" for o in rep.outcomes)
    assert be.closed == [r.key for r in reqs[:len(be.closed)]]      # oldest first
    assert len(be.closed) >= 3
    for t, queued, inflight, draining, used_gb, idle_gb in rep.timeline:
        assert used_gb * 1e9 + idle_gb * 1e9 <= 100 + 30 + 1e-6        # + the plan being reused


def test_live_submission_from_another_thread():
    be = FakeBackend(sizes=[10] * 12, durations=[30] * 12)
    srv = S.Server(be, slots=3, budget_bytes=100, poll_s=1e-4)
    srv.start()
    outs = []

    def client():
        for i in range(12):
            outs.append(srv.submit(_req(i, 0.0)))
            time.sleep(0.002)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    assert outs[-1].wait(10.0)
    rep = srv.stop(timeout=10.0)
    assert [o.status for o in rep.outcomes] == ["ok"] * 12
    assert all(o.wait(0) for o in outs)
    # requests entered while earlier ones were still running
    assert any(o2.arrival < o1.done for o1, o2 in zip(rep.outcomes, rep.outcomes[1:]))
    assert be.max_concurrent >= 2


def test_arrivals_are_honoured():
    clk = FakeClock()
    be = FakeBackend(sizes=[1] * 4, durations=[1] * 4)
    srv = S.Server(be, slots=4, budget_bytes=100, clock=clk, sleep=clk.sleep)
    arr = [0.0, 0.01, 0.02, 0.5]
    rep = srv.run([_req(i, a) for i, a in enumerate(arr)])
    for o, a in zip(rep.outcomes, arr):
        assert o.admitted >= a


def test_poisson_and_mixed_stream_shape():
    t = S.poisson_arrivals(2000, 20.0, 1)
    assert abs(np.mean(np.diff(t)) - 0.05) < 0.005
    reqs = S.mixed_requests(40, 20.0, 2)
    for r in reqs:
        assert (r.n0, r.n1, r.n2) in {(128, 128, 128), (256, 256, 128), (512, 512, 256), (1024, 1024, 256)}
        assert 180 <= r.nproj <= 1800 and math.radians(10) <= r.tilt <= math.radians(40)
        assert r.det_w == int(1.5 * r.n0) and r.det_h == r.n2


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    from paper_2401_11101_gb300 import _build, inputs as I, lamino as L
    _build.build()
    sizes = ((32, 32, 32), (64, 64, 32), (48, 48, 48))
    reqs = S.mixed_requests(12, 400.0, 9, sizes=sizes, nproj=(24, 96))
    for r in reqs:
        g = I.Geometry(r.n0, r.n1, r.n2, r.nproj, r.det_h, r.det_w, r.tilt)
        prm = I.ellipsoid_params(g, 6, seed=100 + r.rid)
        r.d = I.project_boxed(prm, g, device="cuda").half().cpu().pin_memory()
        r.form = "fourier" if r.rid % 3 else "direct"
    be = S.CudaBackend(0, slots=3)
    rep = S.Server(be, slots=3).run(reqs)
    summ = rep.summary(reqs)
    print("serve summary:", summ)
    assert summ["ok"] == len(reqs)
    # at some point more than one request was in flight
    spans = [(o.admitted, o.done) for o in rep.outcomes]
    assert any(a2 < d1 and a1 < d2 for i, (a1, d1) in enumerate(spans)
               for (a2, d2) in spans[i + 1:])
    for r, o in zip(reqs, rep.outcomes):
        with L.Plan(r.n0, r.n1, r.n2, r.nproj, r.det_w, r.det_h, r.tilt) as p:
            alone = p.fbp(r.d.cuda(), form=r.form, kind=r.kind).cpu()
        err = float((o.volume - alone).norm() / alone.norm())
        assert err <= 1e-6, (r.rid, err)


@pytest.mark.gpu
def test_auto_form_is_z_chunked_to_fit_then_falls_back_to_direct():
    from paper_2401_11101_gb300 import _build, inputs as I, lamino as L
    _build.build()
    # few projections, wide planes: the x1-pass planes dominate the Fourier workspace
    r = S.Request(0, 128, 128, 64, 40, 192, 64, 0.35, 0.0)
    g = I.Geometry(r.n0, r.n1, r.n2, r.nproj, r.det_h, r.det_w, r.tilt)
    r.d = I.project_boxed(I.ellipsoid_params(g, 8, seed=70), g, device="cuda").half().cpu().pin_memory()
    r.form = "auto"
    be = S.CudaBackend(0, slots=1)
    direct = be._form_bytes(r, "direct")
    full = be._form_bytes(r, "fourier")
    z16 = be._form_bytes(r, "fourier", 16)
    z8 = be._form_bytes(r, "fourier", 8)
    print(f"footprints: direct {direct}, Fourier {full}, z16 {z16}, z8 {z8}")
    assert direct < z8 <= z16 < full
    with L.Plan(r.n0, r.n1, r.n2, r.nproj, r.det_w, r.det_h, r.tilt) as p:
        alone_f = p.fbp(r.d.cuda(), form="fourier", kind=r.kind).cpu()
        alone_d = p.fbp(r.d.cuda(), form="direct", kind=r.kind).cpu()
    # a budget below the unchunked Fourier footprint: z-chunked Fourier form
    rep = S.Server(be, slots=1, budget_bytes=z16).run([r])
    o = rep.outcomes[0]
    assert o.status == "ok" and o.form == "fourier/z16" and be.form_of(r) == ("fourier", 16)
    assert float((o.volume - alone_f).norm() / alone_f.norm()) <= 1e-6
    # below every chunked footprint: the direct form
    be2 = S.CudaBackend(0, slots=1)
    rep = S.Server(be2, slots=1, budget_bytes=(direct + z8) // 2).run([r])
    o = rep.outcomes[0]
    assert o.status == "ok" and o.form == "direct"
    assert float((o.volume - alone_d).norm() / alone_d.norm()) <= 1e-6
    # with room, the unchunked Fourier form
    be2.budget = full * 2
    assert be2.form_of(r) == ("fourier", 0)
