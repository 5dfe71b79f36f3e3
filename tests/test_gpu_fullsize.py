"""Parity at the benchmark's full sizes, in its launch configurations.

* The 512-grid batch (sides log-uniform 64..512, 3.4e7 cells, FP32, the tuned
  default tile variant): every grid advances together; sampled grids (smallest,
  median, largest) are checked against the oracle run on that grid alone, and
  every grid's mass is conserved.
* The 4096 x 4096 single vortex in FP32 (the serving benchmark's resident grid),
  whole field against the oracle after a few steps.
* The 1024 x 1024 single vortex (the benchmark's main workload) in FP32, whole
  field against the oracle after 500 steps (the default tile, order-3 upwind),
  and for 40 steps with each other stencil order, the central flux and the
  three-stage scheme; the batch's sampled grids after 200 steps.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-5


def oracle_run(O, prob, steps):
    p = O.Params(prob.nx, prob.ny, W=prob.W, M=prob.M, cfl=prob.cfl, order=prob.order, flux=prob.flux,
                 stages=prob.stages, dtphiu=prob.dtphiu, vel_kind=prob.vel_kind, vel=prob.vel)
    return O.State(p, prob.phi0).run(steps)


@pytest.mark.parametrize("steps", [10, 200])
def test_batch512_sampled_grids_against_oracle(oracle, steps):
    probs = WL.random_batch(512)
    p0 = probs[0]
    with N.Batch(precision="fp32", W=p0.W, M=p0.M, cfl=p0.cfl, order=p0.order, flux=0, stages=2) as b:
        ids = [b.add(q.phi0, q.vel_kind, q.vel) for q in probs]
        m0 = [b.mass(i) for i in ids]
        b.step(steps)
        assert b.status() == 0
        for i, m in zip(ids, m0):
            assert abs(b.mass(i) - m) / m < 1e-5
        order = sorted(range(len(probs)), key=lambda j: probs[j].cells)
        for j in (order[0], order[len(order) // 2], order[-1]):
            ref = oracle_run(oracle, probs[j], steps).phi()
            assert np.abs(b.phi(ids[j]) - ref).max() < FP32_TOL, (j, probs[j].nx, probs[j].ny)


def test_vortex4096_fp32_against_oracle(oracle):
    prob = WL.vortex1024(n=4096)
    steps = 5
    with N.Solver.from_problem(prob, precision="fp32") as s:
        s.step(steps)
        assert s.status() == 0
        phi = s.phi()
    ref = oracle_run(oracle, prob, steps).phi()
    assert np.abs(phi - ref).max() < FP32_TOL


def test_vortex1024_fp32_500_steps(oracle):
    """The benchmark's main workload in its launch configuration (FP32, order-3
    upwind, two-stage, the default tile for the size) against the oracle after
    500 steps, with its mass."""
    prob = WL.vortex1024(n=1024)
    steps = 500
    with N.Solver.from_problem(prob, precision="fp32") as s:
        m0 = s.mass()
        s.step(steps)
        assert s.status() == 0
        phi, m = s.phi(), s.mass()
    ref = oracle_run(oracle, prob, steps)
    assert np.abs(phi - ref.phi()).max() < FP32_TOL
    assert abs(m - ref.mass()) / ref.mass() < 1e-7 and abs(m - m0) / m0 < 1e-7


@pytest.mark.parametrize("order,flux,stages", [(2, 0, 2), (4, 0, 2), (3, 1, 2), (3, 0, 3)])
def test_vortex1024_fp32_variants_60_steps(oracle, order, flux, stages):
    """1024 x 1024 vortex with the other stencil orders, the central flux and the
    three-stage scheme (at cfl 0.5: it needs dt < 12 tau), 40 steps."""
    prob = WL.vortex1024(n=1024, order=order, flux=flux, stages=stages, cfl=0.5 if stages == 3 else 0.8)
    steps = 40
    with N.Solver.from_problem(prob, precision="fp32") as s:
        s.step(steps)
        assert s.status() == 0
        phi = s.phi()
    ref = oracle_run(oracle, prob, steps).phi()
    assert np.abs(phi - ref).max() < FP32_TOL
