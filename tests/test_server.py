"""Request server: admission, continuous batching and time-to-result.

The policy is tested on the CPU with a stand-in backend whose clock advances
with the work done; the GPU test checks that every served result equals the
same request solved alone."""
import numpy as np
import pytest

from paper_2007_07760_gb300 import server as S


class FakeBatch:
    """Batch interface without a device: steps cost cells * 1 ns of fake time."""

    def __init__(self, clock):
        self.clock = clock
        self.grids = {}
        self.next = 0
        self.live_bytes = 0
        self.max_live_bytes = 0

    def grid_bytes(self, nx, ny):
        return nx * ny * 80

    def add(self, phi0, kind, vel, target):
        gid = self.next
        self.next += 1
        ny, nx = phi0.shape
        self.grids[gid] = [0, target, nx * ny]
        self.live_bytes += nx * ny * 80
        self.max_live_bytes = max(self.max_live_bytes, self.live_bytes)
        return gid

    def step(self, n):
        work = 0
        for g in self.grids.values():
            adv = n if g[1] < 0 else max(0, min(n, g[1] - g[0]))
            g[0] += adv
            work += adv * g[2]
        self.clock.t += work * 1e-9

    def step_index(self, gid):
        return self.grids[gid][0]

    def phi(self, gid):
        return np.zeros(1)

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
