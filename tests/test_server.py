"""Request server: admission, continuous batching in priority lanes and
time-to-result.

The policy is tested on the CPU with a stand-in backend: a simulated device
runs the work queued on its streams at one cell-update per nanosecond, always
from the highest-priority stream that has work (as tiles of a higher-priority
stream take the SMs first), while the host side of the stand-in keeps step
counters, fences and read-outs the way the library does. The GPU tests check
that every served result equals the same request solved alone."""
from collections import deque

import numpy as np
import pytest

from paper_2007_07760_gb300 import server as S


class FakeDevice:
    """Streams of queued work items [seconds left, fence id or None], earlier
    streams first; the device runs up to the fake clock's time when asked."""

    def __init__(self, clock):
        self.clock = clock
        self.t = 0.0
        self.streams = []
        self.done = {}          # fence id -> device time it was passed
        self.next_id = 1

    def stream(self) -> int:
        self.streams.append(deque())
        return len(self.streams) - 1

    def push(self, s, seconds, kind="work"):
        self.streams[s].append([seconds, None, kind])

    def mark(self, s) -> int:
        fid = self.next_id
        self.next_id += 1
        self.streams[s].append([0.0, fid, "fence"])
        return fid

    def queued(self, s, kind) -> int:
        return sum(1 for it in self.streams[s] if it[2] == kind)

    def sync(self):
        while True:
            for q in self.streams:
                while q and q[0][0] <= 0.0:
                    it = q.popleft()
                    if it[1] is not None:
                        self.done[it[1]] = self.t
            q = next((q for q in self.streams if q), None)
            if q is None:
                self.t = max(self.t, self.clock.t)
                return
            if self.t >= self.clock.t:
                return
            dt = min(q[0][0], self.clock.t - self.t)
            q[0][0] -= dt
            self.t += dt


class FakeBatch:
    """Batch interface on a FakeDevice stream: steps cost cells * 1 ns. The
    blocking read-out is refused: the server must not use it."""

    def __init__(self, clock, device=None):
        self.clock = clock
        self.dev = device or FakeDevice(clock)
        self.s = self.dev.stream()
        self.grids = {}          # gid -> [step, target, cells, retire fence]
        self.next = 0
        self.live_bytes = 0
        self.max_live_bytes = 0
        self.max_queued_steps = 0
        self.ready_at = {}       # gid -> device time its read-out landed

    def grid_bytes(self, nx, ny):
        return nx * ny * 80

    def add(self, phi0, kind, vel, target):
        gid = self.next
        self.next += 1
        ny, nx = phi0.shape
        self.grids[gid] = [0, target, nx * ny, None]
        self.live_bytes += nx * ny * 80
        self.max_live_bytes = max(self.max_live_bytes, self.live_bytes)
        self.dev.push(self.s, nx * ny * 1e-9, "init")
        return gid

    def step(self, n):
        work = 0
        for g in self.grids.values():
            if g[3] is not None:
                continue
            adv = n if g[1] < 0 else max(0, min(n, g[1] - g[0]))
            g[0] += adv
            work += adv * g[2]
        self.dev.push(self.s, work * 1e-9, "step")
        self.max_queued_steps = max(self.max_queued_steps, self.dev.queued(self.s, "step"))

    def step_index(self, gid):
        return self.grids[gid][0]

    def retire(self, gid):
        self.grids[gid][3] = self.dev.mark(self.s)
        return self.grids[gid][3]

    def collect(self, gid, wait=False):
        self.dev.sync()
        fid = self.grids[gid][3]
        if fid not in self.dev.done:
            return None
        self.ready_at[gid] = self.dev.done[fid]
        self.remove(gid)
        return np.zeros(1)

    def fence(self):
        return self.dev.mark(self.s)

    def reached(self, fid):
        self.dev.sync()
        return fid in self.dev.done

    def phi(self, gid):
        raise AssertionError("the server must not wait for the device")

    def remove(self, gid):
        self.live_bytes -= self.grids[gid][2] * 80
        del self.grids[gid]


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


def small_trace(count=30, rate=400.0, seed=3):
    return S.poisson_trace(count, rate=rate, seed=seed, nmin=32, nmax=256, smin=50, smax=400)


def test_trace_statistics():
    tr = S.poisson_trace(4000, rate=200.0, seed=1)
    gaps = np.diff([0.0] + [r.arrival for r in tr])
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    n = np.array([r.n for r in tr])
    assert n.min() >= 64 and n.max() <= 2048
    assert abs(np.median(np.log(n)) - 0.5 * (np.log(64) + np.log(2048))) < 0.1
    assert 0.45 < np.mean([r.kind == "rotation" for r in tr]) < 0.55


def test_policy_budget_fifo_and_overlap():
    clock = FakeClock()
    fb = FakeBatch(clock)
    budget = 3 * 256 * 256 * 80
    srv = S.Server(fb, budget_bytes=budget, max_slots=8, slice_steps=16, clock=clock, sleep=clock.sleep)
    trace = small_trace()
    st = srv.run(trace)
    assert st["requests"] == len(trace)
    assert fb.max_live_bytes <= budget and st["peak_bytes"] <= budget
    res = {r.rid: r for r in srv.results}
    # first-come first-served admission
    adm = [res[r.rid].admitted for r in sorted(trace, key=lambda r: r.arrival)]
    assert all(a <= b + 1e-12 for a, b in zip(adm, adm[1:]))
    # continuous batching: requests join while others are running
    overlaps = sum(1 for a in res.values() for b in res.values()
                   if a.rid != b.rid and a.admitted < b.admitted < a.finished)
    assert overlaps > 0
    for r in trace:
        assert res[r.rid].latency >= 0 and res[r.rid].finished >= r.arrival
    assert st["p99_s"] >= st["p50_s"] > 0
    # never more than `depth` slices queued, and all offered work done
    assert fb.max_queued_steps <= 2
    assert srv.cell_updates == sum(r.cells * r.steps for r in trace)


def _lanes(clock, limits, dev=None):
    dev = dev or FakeDevice(clock)
    return [(FakeBatch(clock, dev), lim) for lim in limits], dev


def test_result_delivered_only_after_its_read_out_landed():
    clock = FakeClock()
    lanes, dev = _lanes(clock, [2e6, None])
    srv = S.Server(lanes, budget_bytes=3 * 256 * 256 * 80, max_slots=8, slice_steps=16, clock=clock,
                   sleep=clock.sleep)
    trace = small_trace(count=20)
    st = srv.run(trace)
    assert st["requests"] == 20 and st["failed"] == 0
    ready = [t for b, _ in lanes for t in b.ready_at.values()]
    assert len(ready) == 20
    # each result is collected at or after the device time its copy completed
    fin = sorted(r.finished for r in srv.results)
    assert all(f >= t - 1e-12 for f, t in zip(fin, sorted(ready)))


def test_lanes_keep_short_solves_off_the_resident_step_rate():
    """A resident 1024^2 grid and short requests: in one lockstep lane each small
    request advances at the whole batch's step rate; in a high-priority lane of
    its own it runs at its own."""
    trace = S.poisson_trace(40, rate=50.0, seed=5, nmin=32, nmax=128, smin=200, smax=2000)
    out = {}
    for name, limits in (("one", [None]), ("lanes", [1e8, None])):
        clock = FakeClock()
        lanes, dev = _lanes(clock, limits)
        srv = S.Server(lanes, budget_bytes=1 << 34, slice_steps=32, clock=clock, sleep=clock.sleep)
        srv.add_resident(np.zeros((1024, 1024)), "vortex", (1024.0, 0.05, 1e4))
        st = srv.run(trace)
        assert st["requests"] == 40 and st["failed"] == 0 and st["status"] == 0
        out[name] = st
    assert out["lanes"]["p50_s"] < 0.1 * out["one"]["p50_s"], (out["lanes"]["p50_s"], out["one"]["p50_s"])
    assert out["lanes"]["p99_s"] < 0.2 * out["one"]["p99_s"]
    # the resident grid keeps running in the low lane
    assert out["lanes"]["lanes"][-1]["resident_steps_per_s"] > 0


def test_requests_go_to_the_first_lane_they_fit():
    clock = FakeClock()
    lanes, dev = _lanes(clock, [64 * 64 * 100, 128 * 128 * 1000, None])
    srv = S.Server(lanes, budget_bytes=1 << 30, slice_steps=16, clock=clock, sleep=clock.sleep)
    reqs = [S.Request(0, 0.0, 64, 100, "vortex"), S.Request(1, 0.0, 64, 101, "vortex"),
            S.Request(2, 0.0, 128, 1000, "rotation"), S.Request(3, 0.0, 256, 400, "rotation")]
    assert [lanes.index(next(t for t in lanes if t[0] is srv._lane_for(r).backend)) for r in reqs] == [0, 1, 1, 2]
    st = srv.run(reqs)
    assert [ln["solved"] for ln in st["lanes"]] == [1, 2, 1]


def test_request_larger_than_budget_rejected():
    clock = FakeClock()
    srv = S.Server(FakeBatch(clock), budget_bytes=1000, clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        srv.run(small_trace(count=2))


class CodedError(RuntimeError):
    """Stand-in for the binding's error: carries a status code."""

    def __init__(self, code):
        super().__init__(f"status {code}")
        self.code = code


class RefusingBatch(FakeBatch):
    """FakeBatch whose add refuses a non-finite field (ENONFINITE) and reports
    ENOMEM on the add calls listed in `enomem_calls` (0-based)."""

    def __init__(self, clock, enomem_calls=()):
        super().__init__(clock)
        self.calls = 0
        self.enomem_calls = set(enomem_calls)

    def add(self, phi0, kind, vel, target):
        call = self.calls
        self.calls += 1
        if not np.isfinite(phi0).all():
            raise CodedError(5)
        if call in self.enomem_calls:
            raise CodedError(2)
        return super().add(phi0, kind, vel, target)


def _with_nan(trace, rid):
    out = []
    for r in trace:
        if r.rid == rid:
            phi0, _, _ = S.request_field(r)
            phi0 = phi0.copy()
            phi0[1, 2] = np.nan
            r = S.Request(r.rid, r.arrival, r.n, r.steps, r.kind, phi0)
        out.append(r)
    return out


def test_non_finite_request_fails_alone():
    clock = FakeClock()
    srv = S.Server(RefusingBatch(clock), budget_bytes=3 * 256 * 256 * 80, max_slots=8, slice_steps=16,
                   clock=clock, sleep=clock.sleep)
    trace = _with_nan(small_trace(count=12), rid=5)
    st = srv.run(trace)
    res = {r.rid: r for r in srv.results}
    assert st["requests"] == 12 and st["failed"] == 1
    assert res[5].error == 5 and res[5].phi is None
    assert all(res[r.rid].error == 0 and res[r.rid].finished >= r.arrival for r in trace if r.rid != 5)


def test_out_of_memory_is_retried_then_fails_only_when_alone():
    clock = FakeClock()
    fb = RefusingBatch(clock, enomem_calls=(2, 3))
    srv = S.Server(fb, budget_bytes=3 * 256 * 256 * 80, max_slots=8, slice_steps=16, clock=clock, sleep=clock.sleep)
    trace = small_trace(count=12, rate=1e7)   # all queued at once: two grids run when the third is refused
    st = srv.run(trace)
    assert fb.calls == 14                                  # the refused request was tried three times
    assert st["failed"] == 0 and st["requests"] == 12   # retried once running grids finished
    adm = [r.admitted for r in sorted(srv.results, key=lambda r: r.rid)]
    assert all(a <= b + 1e-12 for a, b in zip(adm, adm[1:]))   # still first come, first served
    clock = FakeClock()
    srv = S.Server(RefusingBatch(clock, enomem_calls=(0,)), budget_bytes=3 * 256 * 256 * 80, clock=clock,
                   sleep=clock.sleep)
    st = srv.run(small_trace(count=3))
    assert st["failed"] == 1 and srv.results[0].error == 2   # nothing running to wait for


def test_out_of_memory_beside_resident_grids_fails_and_ends():
    # a resident grid never finishes: ENOMEM with only residents on the device, or a
    # request that fits the budget only without them, must fail the request, not spin
    clock = FakeClock()
    fb = RefusingBatch(clock, enomem_calls=(1,))   # call 0 adds the resident grid
    srv = S.Server(fb, budget_bytes=3 * 256 * 256 * 80, slice_steps=16, clock=clock, sleep=clock.sleep)
    srv.add_resident(np.zeros((64, 64)), "vortex", (64.0, 0.05, 100.0))
    trace = small_trace(count=3)
    st = srv.run(trace, max_wall=1e3)
    assert st["requests"] == 3 and st["failed"] == 1
    first = min(trace, key=lambda r: r.arrival).rid
    assert {r.rid: r for r in srv.results}[first].error == 2
    clock = FakeClock()
    srv = S.Server(FakeBatch(clock), budget_bytes=300 * 300 * 80, slice_steps=16, clock=clock, sleep=clock.sleep)
    srv.add_resident(np.zeros((200, 200)), "vortex", (200.0, 0.05, 100.0))
    big = [S.Request(0, 0.0, 250, 20, "vortex"), S.Request(1, 0.0, 64, 20, "rotation")]
    st = srv.run(big, max_wall=1e3)
    res = {r.rid: r for r in srv.results}
    assert st["requests"] == 2 and res[0].error == 2 and res[1].error == 0
    assert clock.t < 1e3


def test_zero_step_request_is_served():
    clock = FakeClock()
    fb = FakeBatch(clock)
    srv = S.Server(fb, budget_bytes=1 << 30, slice_steps=16, clock=clock, sleep=clock.sleep)
    reqs = [S.Request(0, 0.0, 64, 0, "vortex"), S.Request(1, 0.0, 48, 0, "rotation"),
            S.Request(2, 0.0, 32, 40, "rotation")]
    for r in reqs:   # the velocity of a zero-step request is still a valid one
        phi0, kind, vel = S.request_field(r)
        assert np.isfinite(vel).all() and (kind != "vortex" or vel[2] > 0)
    st = srv.run(reqs)
    assert st["requests"] == 3 and st["failed"] == 0
    assert srv.cell_updates == 32 * 32 * 40


@pytest.mark.gpu
def test_served_non_finite_request_fails_alone():
    from paper_2007_07760_gb300 import native as N
    common = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")
    trace = _with_nan(S.poisson_trace(6, rate=2000.0, seed=9, nmin=32, nmax=64, smin=20, smax=60), rid=2)
    with N.Batch(**common) as b:
        srv = S.Server(b, budget_bytes=3 * b.grid_bytes(64, 64), slice_steps=8, keep_fields=True)
        st = srv.run(trace)
        assert st["status"] == 0 and b.status() == 0
    res = {r.rid: r for r in srv.results}
    assert st["failed"] == 1 and res[2].error == N.DUGKS_ENONFINITE
    for req in trace:
        if req.rid == 2:
            continue
        phi0, kind, vel = S.request_field(req)
        with N.Batch(**common) as solo:
            g = solo.add(phi0, kind, vel, req.steps)
            solo.step(req.steps)
            assert np.array_equal(solo.phi(g), res[req.rid].phi)


@pytest.mark.gpu
def test_served_results_equal_solo_runs():
    from paper_2007_07760_gb300 import native as N
    common = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")
    trace = S.poisson_trace(14, rate=2000.0, seed=7, nmin=32, nmax=96, smin=20, smax=120)
    with N.Batch(**common) as b:
        budget = 3 * b.grid_bytes(96, 96)
        srv = S.Server(b, budget_bytes=budget, slice_steps=8, keep_fields=True)
        st = srv.run(trace)
    assert st["requests"] == len(trace) and st["status"] == 0
    res = {r.rid: r for r in srv.results}
    for req in trace:
        assert np.isfinite(res[req.rid].phi).all()
        phi0, kind, vel = S.request_field(req)
        with N.Batch(**common) as solo:
            g = solo.add(phi0, kind, vel, req.steps)
            solo.step(req.steps + 5)
            assert solo.step_index(g) == req.steps
            assert np.array_equal(solo.phi(g), res[req.rid].phi)


@pytest.mark.gpu
def test_served_in_priority_lanes_equal_solo_runs():
    """Three lanes on streams of decreasing priority, one CTA per tile, a resident
    grid in the last: every result is its solo run's, bit for bit, and the
    server never waits for the device (retire / collect / fences only)."""
    import torch

    from paper_2007_07760_gb300 import native as N
    common = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")
    trace = S.poisson_trace(24, rate=3000.0, seed=11, nmin=32, nmax=128, smin=20, smax=160)
    trace.append(S.Request(24, 0.001, 48, 0, "rotation"))   # zero steps: the initial field comes back
    streams = [torch.cuda.Stream(priority=p) for p in (-2, -1, 0)]
    batches = [N.Batch(stream=s.cuda_stream, **common) for s in streams]
    try:
        for b in batches:
            b.set_ctas(-1)
        srv = S.Server([(batches[0], 64 * 64 * 60), (batches[1], None), (batches[2], None)],
                       budget_bytes=6 * batches[0].grid_bytes(128, 128), slice_steps=16, keep_fields=True)
        srv.add_resident(WL_drop(96), "vortex", (96.0, 0.05, 400.0))
        st = srv.run(trace)
        assert st["requests"] == len(trace) and st["failed"] == 0 and st["status"] == 0
        assert st["lanes"][0]["solved"] > 0 and st["lanes"][1]["solved"] > 0
    finally:
        for b in batches:
            b.close()
    res = {r.rid: r for r in srv.results}
    for req in trace:
        phi0, kind, vel = S.request_field(req)
        with N.Batch(**common) as solo:
            g = solo.add(phi0, kind, vel, req.steps)
            solo.step(req.steps + 5)
            assert np.array_equal(solo.phi(g), res[req.rid].phi), req.rid


def WL_drop(n):
    from paper_2007_07760_gb300 import workloads as WL
    return WL.drops(n, n, [(0.5 * n, 0.7 * n)], [0.2 * n], 4.0)
