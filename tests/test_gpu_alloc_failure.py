"""Allocation failures, injected on the host: the library's allocation hook makes
the k-th device allocation report failure without asking the device, so no
device memory is exhausted. dugks_create must return DUGKS_ENOMEM at every one of
its allocations and give back everything it had taken (device free memory back
to where it was); dugks_batch_add must return DUGKS_ENOMEM at every one of its
allocations and leave the batch usable, its other grids stepping exactly as in a
batch that never saw a failure."""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
SLACK = 2 << 20   # allocation granularity


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.fixture(autouse=True)
def disarm():
    yield
    N.dugks_selftest_fail_allocs(0, 0)


@pytest.mark.parametrize("precision,stages", [("fp64", 2), ("fp32", 2), ("fp16f", 2), ("fp32", 3)])
def test_create_fails_cleanly_at_every_allocation(precision, stages):
    prob = WL.drop64(order=3, stages=stages, cfl=0.3 if stages == 3 else 0.8)   # three-stage: dt < 12 tau
    base = _free()
    k = 0
    while True:
        assert N.dugks_selftest_fail_allocs(k, 1) == N.DUGKS_OK
        try:
            s = N.Solver.from_problem(prob, precision=precision)
        except N.DugksError as e:
            assert e.code == N.DUGKS_ENOMEM, (k, e)
            assert abs(_free() - base) <= SLACK, f"allocation {k}: device memory not given back"
            k += 1
            assert k < 64
            continue
        N.dugks_selftest_fail_allocs(0, 0)
        break
    try:
        assert k >= 7   # the state planes, phi planes, scratch and status word each failed once
        s.step(5)
        assert s.status() == 0
    finally:
        s.close()
    assert abs(_free() - base) <= SLACK


def test_batch_add_fails_without_harming_the_batch():
    kw = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")
    rng = np.random.default_rng(WL.SEED_BASE + 21)
    first = WL.drops(80, 72, [(30.0, 40.0)], [12.0], 4.0)
    second = WL.drops(96, 64, [(50.0, 30.0)], [14.0], 4.0)
    vel = (0.02 * rng.uniform(-1, 1), 0.02 * rng.uniform(-1, 1))
    with N.Batch(**kw) as ref, N.Batch(**kw) as b:
        g_ref = ref.add(first, "uniform", vel)
        g1 = b.add(first, "uniform", vel)
        ref.step(4)
        b.step(4)
        base = _free()
        k = 0
        while True:
            N.dugks_selftest_fail_allocs(k, 1)
            try:
                g2 = b.add(second, "uniform", vel)
            except N.DugksError as e:
                assert e.code == N.DUGKS_ENOMEM, (k, e)
                assert b.status() == 0
                assert abs(_free() - base) <= SLACK, f"allocation {k}: device memory not given back"
                k += 1
                assert k < 64
                continue
            N.dugks_selftest_fail_allocs(0, 0)
            break
        assert k >= 5   # both state sets, three phi planes, the upload buffer
        ref.step(6)
        b.step(6)
        assert b.status() == 0
        assert np.array_equal(b.phi(g1), ref.phi(g_ref))
        assert b.step_index(g2) == 6
        assert np.isfinite(b.phi(g2)).all()
