"""The tile-variant autotuner on a single grid and on a batch.

It must pick a variant that is, by an independent timing with CUDA events on
the solver's own stream, no slower than the library's defaults by more than the
noise of one measurement, and answer the second time from its cache without
stepping.
"""
import os

import numpy as np
import pytest

from paper_2007_07760_gb300 import autotune
from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture
def cache_dir(tmp_path, monkeypatch):
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    return tmp_path


def event_ms(solver, stream, steps=40):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        N.dugks_step(solver.ctx, 5)
        a.record(stream)
        N.dugks_step(solver.ctx, steps)
        b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / steps


def test_single_grid_choice_and_cache(cache_dir):
    import torch
    prob = WL.vortex1024(n=1024)
    stream = torch.cuda.Stream()
    with N.Solver.from_problem(prob, precision="fp32", stream=stream.cuda_stream) as s:
        v = autotune.tune(s, "single", prob.cells)
        assert v in autotune.VARIANTS and N.dugks_get_variant(s.ctx) == v
        t_best = event_ms(s, stream)
        t_ref = {}
        for w in (2, 4):                       # the two defaults
            s.set_variant(w)
            t_ref[w] = event_ms(s, stream)
        assert t_best <= 1.08 * min(t_ref.values()), (v, t_best, t_ref)
        s.set_variant(v)
        before = s.step_index
        assert autotune.tune(s, "single", prob.cells) == v      # from the cache
        assert s.step_index == before and N.dugks_get_variant(s.ctx) == v
        assert s.status() == 0
    assert os.path.exists(os.path.join(cache_dir, "dugks_gb300", "tune.json"))


def test_batch_choice_is_valid(cache_dir):
    probs = WL.random_batch(count=24)
    with N.Batch(precision="fp32", W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2) as b:
        for q in probs:
            b.add(q.phi0, q.vel_kind, q.vel)
        v = autotune.tune(b, "batch", sum(q.cells for q in probs))
        assert v in autotune.VARIANTS
        assert b.status() == 0
        assert np.isfinite(b.mass(0))
