"""The batch's non-waiting calls: retire / collect, fences, adds and removals
while steps are in flight, and the one-CTA-per-tile launch. Each result must be
bitwise the result of the same grid stepped alone with the waiting calls."""
import time

import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

COMMON = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")


def _fields(seed, shapes):
    rng = np.random.default_rng(WL.SEED_BASE + seed)
    out = []
    for ny, nx in shapes:
        c = [(rng.uniform(0, nx), rng.uniform(0, ny))]
        out.append(WL.drops(nx, ny, c, [min(nx, ny) / 4], 4.0))
    return out


def _solo(phi0, kind, vel, steps, **kw):
    with N.Batch(**dict(COMMON, **kw)) as b:
        g = b.add(phi0, kind, vel, steps)
        b.step(steps + 3)
        assert b.step_index(g) == steps
        return b.phi(g)


def _collect(b, gid, limit_s=30.0):
    t0 = time.perf_counter()
    while True:
        phi = b.collect(gid)
        if phi is not None:
            return phi
        assert time.perf_counter() - t0 < limit_s, "read-out never landed"
        time.sleep(1e-3)


@pytest.mark.parametrize("precision", ["fp32", "fp16f", "fp64"])
def test_retire_collect_equals_solo(precision):
    a, c = _fields(1, [(72, 80), (40, 96)])
    vel = (0.03, -0.02)
    with N.Batch(**dict(COMMON, precision=precision)) as b:
        g1 = b.add(a, "uniform", vel)
        g2 = b.add(c, "rotation", (48.0, 20.0, 3e-3))
        b.step(21)
        t = b.retire(g1)
        assert b.step_index(g1) == 21
        b.step(9)                       # the retired grid is frozen, the other goes on
        assert b.step_index(g1) == 21 and b.step_index(g2) == 30
        p1 = _collect(b, g1)
        assert b.reached(t)
        p2 = b.phi(g2)
        assert b.status() == 0
    assert np.array_equal(p1, _solo(a, "uniform", vel, 21, precision=precision))
    assert np.array_equal(p2, _solo(c, "rotation", (48.0, 20.0, 3e-3), 30, precision=precision))


def test_adds_and_removals_while_steps_are_in_flight():
    """Grids join and leave between queued slices with no wait; each result is
    its solo run's, bit for bit."""
    shapes = [(64, 64), (96, 48), (40, 120), (128, 72), (56, 56), (64, 200)]
    fields = _fields(2, shapes)
    targets = [37, 80, 15, 64, 8, 50]
    vels = [("uniform", (0.02, 0.01)), ("vortex", (64.0, 0.05, 200.0)), ("rotation", (20.0, 60.0, 2e-3)),
            ("uniform", (-0.03, 0.02)), ("vortex", (56.0, 0.04, 50.0)), ("rotation", (32.0, 100.0, -1e-3))]
    got = {}
    with N.Batch(**COMMON) as b:
        b.set_ctas(-1)
        live = {}
        for i in range(3):
            live[b.add(fields[i], *vels[i], targets[i])] = i
        nxt = 3
        tickets = []
        pending = {}
        for _ in range(40):
            b.step(4)
            tickets.append(b.fence())
            for gid in [g for g, i in live.items() if b.step_index(g) >= targets[i]]:
                b.retire(gid)
                pending[gid] = live.pop(gid)
            for gid in list(pending):
                phi = b.collect(gid)
                if phi is not None:
                    got[pending.pop(gid)] = phi
            if nxt < len(fields) and len(live) < 3:
                live[b.add(fields[nxt], *vels[nxt], targets[nxt])] = nxt
                nxt += 1
        for gid in list(pending):
            got[pending.pop(gid)] = _collect(b, gid)
        assert b.status() == 0        # waits for the stream: every fence is passed
        assert all(b.reached(t) for t in tickets)
    assert sorted(got) == list(range(len(fields)))
    for i, phi in got.items():
        assert np.array_equal(phi, _solo(fields[i], *vels[i], targets[i])), i


@pytest.mark.parametrize("ctas", [-1, 7, 0])
def test_cta_count_does_not_change_results(ctas):
    a, c = _fields(3, [(100, 90), (33, 64)])
    with N.Batch(**COMMON) as ref, N.Batch(**COMMON) as b:
        b.set_ctas(ctas)
        r1, r2 = ref.add(a, "uniform", (0.02, 0.03)), ref.add(c, "vortex", (64.0, 0.05, 80.0))
        g1, g2 = b.add(a, "uniform", (0.02, 0.03)), b.add(c, "vortex", (64.0, 0.05, 80.0))
        ref.step(27)
        b.step(27)
        assert np.array_equal(ref.phi(r1), b.phi(g1)) and np.array_equal(ref.phi(r2), b.phi(g2))
        assert ref.mass(r1) == b.mass(g1)


def test_async_call_errors():
    (a,) = _fields(4, [(48, 48)])
    with N.Batch(**COMMON) as b:
        g = b.add(a, "uniform", (0.01, 0.0))
        b.step(3)
        out = np.empty((48, 48))
        with pytest.raises(N.DugksError) as e:   # not retiring
            N.dugks_batch_collect(b.b, g, out)
        assert e.value.code == N.DUGKS_EINVAL
        t = b.retire(g)
        with pytest.raises(N.DugksError) as e:   # twice
            b.retire(g)
        assert e.value.code == N.DUGKS_EINVAL
        with pytest.raises(N.DugksError) as e:   # a ticket never issued
            b.reached(t + 1000)
        assert e.value.code == N.DUGKS_EINVAL
        phi = b.collect(g, wait=True)
        assert phi is not None and phi.shape == (48, 48)
        with pytest.raises(N.DugksError) as e:   # the id is free now
            b.retire(g)
        assert e.value.code == N.DUGKS_EINVAL
        # a retiring grid can be dropped without collecting it, and the slot is reused
        g2 = b.add(a, "uniform", (0.01, 0.0), 5)
        b.step(5)
        b.retire(g2)
        b.remove(g2)
        g3 = b.add(a, "uniform", (0.01, 0.0), 3)
        b.step(8)
        assert b.step_index(g3) == 3
        b.retire(g3)
        assert np.array_equal(b.collect(g3, wait=True), _solo(a, "uniform", (0.01, 0.0), 3))
        assert b.status() == 0


def test_edge_cases_empty_batch_and_retire_before_any_step():
    (a,) = _fields(5, [(40, 56)])
    with N.Batch(**COMMON) as b:
        b.step(10)                      # no grids: nothing to do, no error
        t = b.fence()
        assert b.status() == 0 and b.reached(t)
        g = b.add(a, "vortex", (56.0, 0.05, 100.0), 30)
        b.retire(g)                     # at step 0: the initial field's phi
        got = _collect(b, g)
        b.step(5)                       # the batch is empty again
        assert b.status() == 0
    with N.Batch(**COMMON) as ref:
        r = ref.add(a, "vortex", (56.0, 0.05, 100.0), 30)
        assert np.array_equal(got, ref.phi(r))
