"""The allocation-free mass entry point against the context's own mass.

dugks_field_mass_noalloc serves callers that cannot call cudaMalloc where they
need a mass (under a framework whose caching allocator owns all device memory,
in loops that cannot take cudaMalloc's implicit synchronisation). It keeps its
per-tile partials in a static device array instead of allocated scratch. This
file is collected last so that a failure here comes after every other test has
run.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,dtype,rtol", [("fp64", 0, 1e-13), ("fp32", 1, 1e-6)])
def test_noalloc_mass_matches_context_mass_twice(precision, dtype, rtol):
    torch = pytest.importorskip("torch")
    prob = WL.drop64(order=3)
    stream = torch.cuda.Stream()
    tdtype = torch.float64 if dtype == 0 else torch.float32
    with N.Solver.from_problem(prob, precision=precision, stream=stream.cuda_stream) as s:
        field = torch.empty((prob.ny, prob.nx), dtype=tdtype, device="cuda")
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        for steps in (25, 40):          # two calls in a row on different fields
            s.step(steps)
            ref = s.mass()
            N.dugks_read_phi_device(s.ctx, field.data_ptr())
            code = N.dugks_field_mass_noalloc(field.data_ptr(), dtype, prob.nx, prob.ny, prob.nx,
                                              out.data_ptr(), stream.cuda_stream)
            assert code == N.DUGKS_OK
            stream.synchronize()
            got = float(out.item())
            assert abs(got - ref) / abs(ref) < rtol, (got, ref)
            out.fill_(float("nan"))
            torch.cuda.synchronize()


def test_noalloc_rejects_fields_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    field = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 4097 x 4096 needs 129 * 512 tiles > 65536: refused before any launch
    code = N.dugks_field_mass_noalloc(field.data_ptr(), 0, 4097, 4096, 4097, out.data_ptr(), None)
    assert code == N.DUGKS_EINVAL
    assert N.dugks_field_mass_noalloc(field.data_ptr(), 2, 4, 4, 4, out.data_ptr(), None) == N.DUGKS_EINVAL


def test_noalloc_serves_one_tile_column_at_the_tile_limit():
    # 32 x 524288 cells: one tile column of 65536 tile rows (the array's limit),
    # more tile rows than a grid's y dimension may hold
    torch = pytest.importorskip("torch")
    nx, ny = 32, 65536 * 8
    g = torch.Generator(device="cuda").manual_seed(2007077609)
    field = torch.rand((ny, nx), dtype=torch.float64, device="cuda", generator=g)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert N.dugks_field_mass_noalloc(field.data_ptr(), 0, nx, ny, nx, out.data_ptr(), None) == N.DUGKS_OK
        torch.cuda.synchronize()
        ref = float(field.sum().item())
        assert abs(float(out.item()) - ref) / ref < 1e-13
        field.mul_(0.5)
