"""Stage-by-stage parity of the face stage through dugks_debug_faces: bar f at the
east and north face midpoints (Eqs. (24)-(26)) and the original f there
(Eqs. (27)-(28)) of the GPU path against the oracle's stage functions applied to
the oracle's own state, after three steps (so d(phi u)/dt is active), for every
order and both reconstructions, on an 8 x 8 grid and on a 37 x 29 grid that
leaves ragged tiles in both directions. FP64 to 1e-12 of the largest value,
FP32 to 1e-5 and FP16 storage to 1e-4 absolute. The read-out leaves the
context's state, step index and later steps untouched."""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

STEPS = 3
BOUND = {"fp64": 1e-12, "fp32": 1e-5, "fp16f": 1e-4}


def _case(nx, ny):
    phi0 = WL.drops(nx, ny, [(0.45 * nx, 0.55 * ny)], [0.3 * min(nx, ny)], 3.0)
    return phi0, "rotation", (0.5 * nx, 0.5 * ny, 0.004)


def _oracle_faces(O, p, phi0):
    st = O.State(p, phi0)
    st.run(STEPS)
    X = st.f
    dt = p.cfl
    t = STEPS * dt
    h, a, b = O.coefficients(p)[:3]
    V, g = O.cell_quantities(p, O.phi_of(p, X), st.phi_prev, t, t - dt, dt, True)
    fbE, fbN = O.reconstruct(p, a * X + b * g, h)
    fE, fN = O.face_f(p, fbE, fbN, V, h, t + h)
    return fbE, fbN, fE, fN


@pytest.mark.parametrize("nx,ny", [(8, 8), (37, 29)])
@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16f"])
def test_faces_against_oracle(oracle, precision, order, flux, nx, ny):
    phi0, kind, vel = _case(nx, ny)
    p = oracle.Params(nx, ny, W=3.0, M=0.02, cfl=0.8, order=order, flux=flux, stages=2, vel_kind=kind, vel=vel)
    ref = _oracle_faces(oracle, p, phi0)
    with N.Solver(nx, ny, phi0, W=3.0, M=0.02, cfl=0.8, order=order, flux=flux, stages=2,
                  precision=precision, vel_kind=kind, vel=vel) as s:
        s.step(STEPS)
        got = s.debug_faces()
        assert s.status() == 0
    for name, gv, rv in zip(("bar f east", "bar f north", "f east", "f north"), got, ref):
        err = float(np.abs(gv - rv).max())
        scale = float(np.abs(rv).max()) if precision == "fp64" else 1.0
        assert err <= BOUND[precision] * scale, (name, precision, order, flux, nx, ny, err)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16f"])
def test_read_out_leaves_state_alone(precision):
    nx, ny = 37, 29
    phi0, kind, vel = _case(nx, ny)
    kw = dict(W=3.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision=precision, vel_kind=kind, vel=vel)
    with N.Solver(nx, ny, phi0, **kw) as a, N.Solver(nx, ny, phi0, **kw) as b:
        a.step(STEPS)
        b.step(STEPS)
        m = a.mass()
        before = a.phi()
        a.debug_faces()
        assert a.step_index == STEPS
        assert np.array_equal(a.phi(), before)
        assert a.mass() == m
        a.step(5)
        b.step(5)
        assert np.array_equal(a.phi(), b.phi())
        assert a.mass() == b.mass()


def test_read_out_rejects_three_stage_without_poisoning():
    nx, ny = 16, 16
    phi0, kind, vel = _case(nx, ny)
    with N.Solver(nx, ny, phi0, W=3.0, M=0.02, cfl=0.5, order=3, flux=0, stages=3, precision="fp64",
                  vel_kind=kind, vel=vel) as s:
        with pytest.raises(N.DugksError) as e:
            s.debug_faces()
        assert e.value.code == N.DUGKS_EINVAL
        s.step(2)   # still usable
        assert s.status() == 0
