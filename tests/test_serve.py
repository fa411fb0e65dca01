"""Serving: admission by HBM footprint, backfill, slots, timeouts (CPU, with a
fake backend) and, on the GPU, that every request's result is the same alone
and in a mixed stream."""
import math

import numpy as np
import pytest
import torch

from paper_2401_11101_gb300 import serve as S


class FakeBackend:
    """Jobs finish a fixed number of polls after submission; never = stuck."""

    def __init__(self, sizes, durations, stuck=()):
        self.sizes, self.durations, self.stuck = sizes, durations, set(stuck)
        self.log = []
        self.concurrent = 0
        self.max_concurrent = 0

    def default_budget(self):
        return 100

    def footprint(self, r):
        return self.sizes[r.rid]

    def evict(self, target):
        self.log.append(("evict", target))

    def submit(self, r, slot):
        self.concurrent += 1
        self.max_concurrent = max(self.max_concurrent, self.concurrent)
        self.log.append(("submit", r.rid, slot))
        return {"r": r, "left": self.durations[r.rid]}

    def poll(self, h):
        if h["r"].rid in self.stuck:
            return False
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
    # the stuck job's slot and memory were returned
    assert be.concurrent == 0


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
    b.idle, b.draining = collections.OrderedDict(), []
    r = S.Request(0, 8, 8, 8, 4, 12, 8, 0.3, 0.0)
    ev, plan = Ev(), object()
    b.release({"req": r, "plan": plan, "ev": ev, "d": Buf(), "vol": Buf(), "host": None, "stream": None})
    assert r.key not in b.idle and len(b.draining) == 1
    b._drain()
    assert r.key not in b.idle
    ev.done = True
    b._drain()
    assert b.idle[r.key] == [plan] and not b.draining
    ev2 = Ev()
    ev2.done = True
    plan2 = object()
    b.release({"req": r, "plan": plan2, "ev": ev2, "d": Buf(), "vol": Buf(), "host": None, "stream": None})
    assert b.idle[r.key] == [plan, plan2]


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
def test_auto_form_falls_back_to_direct_when_short_of_memory():
    from paper_2401_11101_gb300 import _build, inputs as I, lamino as L
    _build.build()
    be = S.CudaBackend(0, slots=1)
    r = S.Request(0, 64, 64, 32, 48, 96, 32, 0.35, 0.0)
    g = I.Geometry(r.n0, r.n1, r.n2, r.nproj, r.det_h, r.det_w, r.tilt)
    r.d = I.project_boxed(I.ellipsoid_params(g, 8, seed=70), g, device="cuda").half().cpu().pin_memory()
    r.form = "auto"
    direct = be._form_bytes(r, "direct")
    fourier = be._form_bytes(r, "fourier")
    assert direct < fourier
    # a budget between the two footprints: admitted, in the direct form
    rep = S.Server(be, slots=1, budget_bytes=(direct + fourier) // 2).run([r])
    assert rep.outcomes[0].status == "ok" and be.form_of(r) == "direct"
    with L.Plan(r.n0, r.n1, r.n2, r.nproj, r.det_w, r.det_h, r.tilt) as p:
        alone = p.fbp(r.d.cuda(), form="direct", kind=r.kind).cpu()
    assert float((rep.outcomes[0].volume - alone).norm() / alone.norm()) <= 1e-6
    # with room for both, the same request runs in the Fourier form
    be.budget = fourier * 2
    assert be.form_of(r) == "fourier"
