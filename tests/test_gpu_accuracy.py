"""Accuracy of every precision against the FP64 oracle on the slotted-disk
rotation (256 x 256, order-3 upwind, two-stage, M = 0.002, cfl = 0.8), 2000
steps: max |dphi|, relative L2 difference and mass drift, each printed (run
pytest with -s to see the line) and bounded: FP64 1e-12 relative, FP32 5e-5
max |dphi| (the FP32 acceptance bound), FP16 storage 2e-3.
"""
import json

import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

STEPS = 2000


@pytest.fixture(scope="module")
def reference(oracle):
    prob = WL.slotted_disk256(order=3, flux=0)
    p = oracle.Params(prob.nx, prob.ny, W=prob.W, M=prob.M, cfl=prob.cfl, order=prob.order, flux=prob.flux,
                      stages=prob.stages, dtphiu=prob.dtphiu, vel_kind=prob.vel_kind, vel=prob.vel)
    st = oracle.State(p, prob.phi0)
    m0 = st.mass()
    st.run(STEPS)
    return prob, st.phi(), m0, st.mass()


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 5e-5), ("fp16f", 2e-3)])
def test_precision_against_oracle(reference, precision, bound):
    prob, ref, m0_ref, m_ref = reference
    with N.Solver.from_problem(prob, precision=precision) as s:
        m0 = s.mass()
        s.step(STEPS)
        phi = s.phi()
        m = s.mass()
        assert s.status() == 0
    d = phi - ref
    rep = {"precision": precision, "steps": STEPS, "max_abs_dphi": float(np.abs(d).max()),
           "rel_l2_dphi": float(np.sqrt((d ** 2).sum() / (ref ** 2).sum())),
           "mass_drift": float(abs(m - m0) / m0), "oracle_mass_drift": float(abs(m_ref - m0_ref) / m0_ref)}
    print("ACCURACY", json.dumps(rep))
    if precision == "fp64":
        assert rep["max_abs_dphi"] / np.abs(ref).max() < bound
    else:
        assert rep["max_abs_dphi"] < bound
    assert rep["mass_drift"] < (1e-12 if precision == "fp64" else 1e-5)
