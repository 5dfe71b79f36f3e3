"""DUGKS-T2S5 (order 5: the fifth-order reconstruction of Sec. III.A, read as the
degree-4 tensor-product Lagrange interpolant on the 5 x 5 cells centred at the
cell nearest to the back-traced point) on the GPU: the radius-2 TMA-staged
kernels with host-built Lagrange face stencils.

Against the oracle in FP64 (1e-12 relative), FP32 (5e-5) and FP16 storage on
ragged grids over the CFL numbers and velocity kinds; the refusals (central
flux, three-stage, the generic kernel, the face read-out); and the paper's
T2S5 rows of the diagonal-translation table (N = 128 at every CFL number,
N = 256 at 0.8) and of the interface-extension table (Pe = 256, CFL 0.8; at CFL
0.25 and 0.5 the ratios were 0.94) in FP64.
"""
import json
import os

import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL
from paper_tables import e_phi, extension_entries, paper_value

pytestmark = pytest.mark.gpu

KINDS = {"uniform": (0.03, -0.02), "rotation": (38.0, 35.0, 1.5e-3), "vortex": (77.0, 0.04, 30.0),
         "deformation": (77.0, 0.04, 30.0)}


def problem(nx, ny, cfl, kind, seed):
    rng = np.random.default_rng(WL.SEED_BASE + 110 + seed)
    cents = [tuple(rng.uniform(0, [nx, ny])) for _ in range(3)]
    phi0 = WL.drops(nx, ny, cents, [min(nx, ny) / 5, min(nx, ny) / 7, min(nx, ny) / 9], 4.0)
    return WL.Problem("t2s5", nx, ny, 4.0, 0.02, cfl, 5, 0, 2, kind, KINDS[kind], phi0, 60)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 5e-5), ("fp16f", 2e-5)])
@pytest.mark.parametrize("cfl", [0.8, 0.5, 0.25])
def test_t2s5_matches_oracle(oracle, precision, bound, cfl):
    kind = list(KINDS)[int(cfl * 20) % 4]
    prob = problem(77, 70, cfl, kind, seed=int(cfl * 20))
    p = oracle.Params(77, 70, W=4.0, M=0.02, cfl=cfl, order=5, flux=0, stages=2, vel_kind=kind, vel=prob.vel)
    ref = oracle.State(p, prob.phi0).run(60)
    with N.Solver.from_problem(prob, precision=precision) as s:
        s.step(60)
        assert s.status() == 0
        phi, m = s.phi(), s.mass()
    err = np.abs(phi - ref.phi()).max()
    assert (err / np.abs(ref.phi()).max() if precision == "fp64" else err) < bound, err
    if precision == "fp64":
        assert abs(m - ref.mass()) / ref.mass() < 1e-13


def test_t2s5_refusals():
    phi0 = WL.drops(32, 32, [(16, 16)], [6.0], 4.0)
    for kw in (dict(flux=1), dict(stages=3, cfl=0.5, M=0.02)):
        with pytest.raises(N.DugksError) as e:
            N.dugks_create(N.make_params(32, 32, order=5, **kw), phi0)
        assert e.value.code == N.DUGKS_EINVAL
    with N.Solver(32, 32, phi0, order=5, precision="fp64") as s:
        with pytest.raises(N.DugksError):
            s.set_variant(-1)
        z = np.zeros(9 * 32 * 32)
        assert N.lib().dugks_debug_faces(s.ctx, *[z.ctypes.data_as(N.ctypes.POINTER(N.ctypes.c_double))] * 4) \
            == N.DUGKS_EINVAL
        s.step(5)
        assert s.status() == 0


@pytest.mark.parametrize("n,cfl", [(128, 0.25), (128, 0.5), (128, 0.8), (256, 0.8)])
def test_t2s5_translation_table(n, cfl):
    prob = WL.translation(n, 5, 0, 2, cfl)
    with N.Solver.from_problem(prob, precision="fp64") as s:
        s.step(prob.steps)
        phi = s.phi()
    e = e_phi(phi, prob.phi0)
    ref = paper_value("T2S5", cfl, n)
    print("TABLE", json.dumps({"scheme": "T2S5", "cfl": cfl, "n": n, "E_phi": e, "ratio": e / ref}))
    assert abs(e / ref - 1) < 0.05, (e, ref)


@pytest.mark.parametrize("scheme,cfl,Pe,printed",
                         [e for e in extension_entries(("T2S5",)) if e[2] == 256 and e[1] == 0.8])
def test_t2s5_extension_table(scheme, cfl, Pe, printed):
    phi0, u, v, half = WL.extension(Pe, cfl)
    with N.Solver(256, 256, phi0, vel_kind="field", u=u, v=v, W=4.0, M=0.02, cfl=cfl, order=5, flux=0,
                  stages=2, precision="fp64") as s:
        s.step(half)
        N.dugks_set_velocity(s.ctx, N.DUGKS_VEL_FIELD, None, -u, -v)
        s.step(half)
        phi = s.phi()
    e = e_phi(phi, phi0)
    print("TABLE", json.dumps({"scheme": "T2S5-ext", "cfl": cfl, "Pe": Pe, "E_phi": e, "ratio": e / printed}))
    assert abs(e / printed - 1) < 0.15, (e, printed)
