"""Parity at the benchmark's full sizes, in its launch configurations.

* The 512-grid batch (sides log-uniform 64..512, 3.4e7 cells, FP32, the tuned
  default tile variant): every grid advances together; sampled grids (smallest,
  median, largest) are checked against the oracle run on that grid alone, and
  every grid's mass is conserved.
* The 4096 x 4096 single vortex in FP32 (the serving benchmark's resident grid),
  whole field against the oracle after a few steps.
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


def test_batch512_sampled_grids_against_oracle(oracle):
    probs = WL.random_batch(512)
    p0 = probs[0]
    steps = 10
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
