"""Speed guards: the step kernels must stay within about twice their measured
times, so that a change that keeps the results but wrecks the code the compiler
makes (a loop no longer unrolled, parameters read through computed indices)
fails here rather than only in the benchmark.

Measured on GB300 (FP32, order 3 upwind, two-stage, single vortex): the 1024^2
step about 53 us for the default tile shape (8 warps x 3 rows) and 60 us for
16 warps x 1 row; one 1024^2 grid in a batch about 60 us per step. The bounds
are twice those, device-timed with CUDA events over 40 steps (state of 80 MB:
partly L2-resident, so the times are, if anything, lower than flushed ones)."""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

COMMON = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")


def _us_per_step(stream, step, K=40):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        step(K)
        b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / K * 1e3


@pytest.mark.parametrize("variant,bound_us", [(4, 110.0), (1, 125.0), (2, 110.0)])
def test_single_grid_step_time(variant, bound_us):
    prob = WL.vortex1024(n=1024)
    st = torch.cuda.Stream()
    with N.Solver.from_problem(prob, precision="fp32", stream=st.cuda_stream) as s:
        s.set_variant(variant)
        s.step(10)
        st.synchronize()
        us = _us_per_step(st, lambda K: N.dugks_step(s.ctx, K))
        assert s.status() == 0
    assert us < bound_us, f"variant {variant}: {us:.1f} us per 1024^2 step"


@pytest.mark.parametrize("ctas", [0, -1])
def test_batch_step_time(ctas):
    prob = WL.vortex1024(n=1024)
    st = torch.cuda.Stream()
    with N.Batch(stream=st.cuda_stream, **COMMON) as b:
        b.set_ctas(ctas)
        b.add(prob.phi0, prob.vel_kind, prob.vel)
        b.step(16)
        st.synchronize()
        us = _us_per_step(st, lambda K: b.step(K))
        assert b.status() == 0
    assert us < 130.0, f"batch (ctas {ctas}): {us:.1f} us per 1024^2 step"
    assert np.isfinite(us)
