"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance on phi: max_cells |phi_gpu - phi_oracle| / max_cells |phi_oracle|.
FP64: 1e-12 after the run (1000 steps for the 64x64 drop). FP32: 5e-5 max |dphi|.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 5e-5


def oracle_params(O, prob, **over):
    kw = dict(W=prob.W, M=prob.M, cfl=prob.cfl, order=prob.order, flux=prob.flux, stages=prob.stages,
              dtphiu=prob.dtphiu, vel_kind=prob.vel_kind, vel=prob.vel)
    kw.update(over)
    return O.Params(prob.nx, prob.ny, **kw)


def run_both(O, prob, steps, precision="fp64", field=None):
    if field is not None:
        u, v = field
        op = oracle_params(O, prob, vel_kind="field", u_field=u, v_field=v)
        gpu = N.Solver(prob.nx, prob.ny, prob.phi0, vel_kind="field", u=u, v=v, W=prob.W, M=prob.M,
                       cfl=prob.cfl, order=prob.order, flux=prob.flux, stages=prob.stages,
                       precision=precision, dtphiu=prob.dtphiu)
    else:
        op = oracle_params(O, prob)
        gpu = N.Solver.from_problem(prob, precision=precision)
    ref = O.State(op, prob.phi0).run(steps)
    with gpu:
        gpu.step(steps)
        phi = gpu.phi()
        mass = gpu.mass()
    return phi, ref.phi(), mass, ref.mass()


def rel_err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_drop64_fp64_1000_steps(oracle):
    """64x64 drop R = 16, W = 4, M = 0.01, u = (0.02, 0.02), order 2 upwind, 1000 steps."""
    prob = WL.drop64()
    phi, ref, m, mref = run_both(oracle, prob, 1000)
    assert rel_err(phi, ref) < FP64_TOL
    assert abs(m - mref) / mref < 1e-13


def small(nx, ny, order, flux, stages, cfl, vel_kind="uniform", vel=(0.03, -0.02), M=0.02, seed=0):
    rng = np.random.default_rng(WL.SEED_BASE + seed)
    cents = [tuple(rng.uniform(0, [nx, ny])) for _ in range(2)]
    phi0 = WL.drops(nx, ny, cents, [min(nx, ny) / 5, min(nx, ny) / 7], 4.0)
    return WL.Problem("small", nx, ny, 4.0, M, cfl, order, flux, stages, vel_kind, vel, phi0, 60)


VARIANTS = [(o, f, s, 0.8 if s == 2 else 0.5) for o in (2, 3, 4) for f in (0, 1) for s in (2, 3)]


@pytest.mark.parametrize("order,flux,stages,cfl", VARIANTS)
def test_variants_fp64_ragged(oracle, order, flux, stages, cfl):
    """Every order x flux x stage count on a ragged 45 x 27 grid (several tiles,
    partial last tile in both directions)."""
    prob = small(45, 27, order, flux, stages, cfl, seed=order * 10 + flux * 3 + stages)
    phi, ref, m, mref = run_both(oracle, prob, 60)
    assert rel_err(phi, ref) < FP64_TOL
    assert abs(m - mref) / mref < 1e-13


@pytest.mark.parametrize("kind,vel", [("rotation", (20.0, 14.0, 2e-3)), ("vortex", (40.0, 0.05, 30.0)),
                                      ("deformation", (40.0, 0.05, 30.0))])
@pytest.mark.parametrize("stages", [2, 3])
def test_velocity_kinds_fp64(oracle, kind, vel, stages):
    prob = small(40, 28, 3, 0, stages, 0.8 if stages == 2 else 0.5, vel_kind=kind, vel=vel, seed=7)
    phi, ref, _, _ = run_both(oracle, prob, 60)
    assert rel_err(phi, ref) < FP64_TOL


@pytest.mark.parametrize("precision,variant", [("fp64", 2), ("fp64", -1), ("fp32", 4), ("fp32", -1)])
@pytest.mark.parametrize("order,flux", [(3, 0), (2, 1), (4, 0)])
def test_deformation_flow_every_kernel(oracle, precision, variant, order, flux):
    """The smoothed deformation of Sec. III.D (time-dependent: reversed by cos(pi t/T))
    through the TMA-staged and the generic kernels, with the reversal inside the run."""
    prob = small(64, 48, order, flux, 2, 0.8, vel_kind="deformation", vel=(64.0, 0.05, 24.0), seed=13)
    ref = O_run(oracle, prob, 50)
    with N.Solver.from_problem(prob, precision=precision) as s:
        s.set_variant(variant)
        s.step(50)
        assert s.status() == 0
        phi = s.phi()
    err = np.abs(phi - ref).max()
    assert (err / np.abs(ref).max() if precision == "fp64" else err) < (FP64_TOL if precision == "fp64" else FP32_TOL)


def O_run(O, prob, steps):
    return O.State(oracle_params(O, prob), prob.phi0).run(steps).phi()


def test_velocity_field_fp64(oracle):
    prob = small(36, 20, 3, 0, 2, 0.8, seed=9)
    X, Y = WL.centres(36, 20)
    # a divergence-free cell field (discretely close enough for the test)
    u = 0.04 * np.sin(2 * np.pi * Y / 20)
    v = 0.03 * np.cos(2 * np.pi * X / 36)
    phi, ref, _, _ = run_both(oracle, prob, 40, field=(u, v))
    assert rel_err(phi, ref) < FP64_TOL


@pytest.mark.parametrize("n", [8, 9, 33])
def test_minimum_and_odd_sizes_fp64(oracle, n):
    prob = small(n, n + 3, 3, 0, 2, 0.8, seed=n)
    prob.phi0 = WL.drops(n, n + 3, [(n / 2, n / 2)], [n / 4], 4.0)
    phi, ref, _, _ = run_both(oracle, prob, 30)
    assert rel_err(phi, ref) < FP64_TOL


def test_drop64_fp32_1000_steps(oracle):
    prob = WL.drop64()
    phi, ref, m, mref = run_both(oracle, prob, 1000, precision="fp32")
    assert np.abs(phi - ref).max() < FP32_TOL
    assert abs(m - mref) / mref < 1e-6


@pytest.mark.parametrize("order,flux,stages,cfl", [(3, 0, 2, 0.8), (3, 1, 2, 0.8), (4, 0, 2, 0.8), (3, 0, 3, 0.5)])
def test_variants_fp32(oracle, order, flux, stages, cfl):
    prob = small(45, 27, order, flux, stages, cfl, seed=3)
    phi, ref, _, _ = run_both(oracle, prob, 200, precision="fp32")
    assert np.abs(phi - ref).max() < FP32_TOL


def test_fp16_storage_error_bounded(oracle):
    """FP16 deviation storage (f - w phi in half precision, phi an FP32 plane):
    error against the FP64 oracle after 1000 steps; measured 9.8e-6 on a GB300,
    bound twice that."""
    prob = WL.drop64(order=3)
    phi, ref, m, mref = run_both(oracle, prob, 1000, precision="fp16f")
    err = np.abs(phi - ref).max()
    assert err < 2e-5, err
    assert abs(m - mref) / mref < 1e-5


def test_slotted_disk_full_size_fp32_short_run(oracle):
    """The 256 x 256 slotted disk in the launch configuration of the benchmark,
    whole field against the oracle after 20 steps."""
    prob = WL.slotted_disk256(order=3, flux=0)
    phi, ref, _, _ = run_both(oracle, prob, 20, precision="fp32")
    assert np.abs(phi - ref).max() < FP32_TOL


def test_slotted_disk_full_size_fp64_central(oracle):
    prob = WL.slotted_disk256(order=3, flux=1)
    phi, ref, _, _ = run_both(oracle, prob, 20)
    assert rel_err(phi, ref) < FP64_TOL


def test_vortex1024_fp32_two_steps(oracle):
    prob = WL.vortex1024(order=3, flux=0)
    phi, ref, _, _ = run_both(oracle, prob, 2, precision="fp32")
    assert np.abs(phi - ref).max() < FP32_TOL


def test_mass_conserved_fp64_long():
    prob = small(64, 48, 3, 0, 2, 0.8, vel_kind="rotation", vel=(32, 24, 3e-3), seed=5)
    with N.Solver.from_problem(prob) as s:
        m0 = s.mass()
        s.step(2000)
        assert abs(s.mass() - m0) / m0 < 1e-13


def test_deterministic_and_checkpoint_resume():
    prob = small(40, 40, 3, 0, 2, 0.8, seed=11)
    with N.Solver.from_problem(prob, precision="fp32") as a:
        a.step(50)
        buf = np.empty(N.dugks_state_bytes(a.ctx), dtype=np.uint8)
        idx = N.dugks_save_state(a.ctx, buf)
        a.step(50)
        pa = a.phi()
    with N.Solver.from_problem(prob, precision="fp32") as b:
        N.dugks_load_state(b.ctx, buf, idx)
        assert b.step_index == 50
        b.step(50)
        pb = b.phi()
    with N.Solver.from_problem(prob, precision="fp32") as c:
        c.step(100)
        pc = c.phi()
    assert np.array_equal(pa, pb) and np.array_equal(pa, pc)


def test_invalid_parameters_rejected():
    phi0 = np.zeros((16, 16))
    bad = [dict(stages=3, cfl=0.8, M=0.02),          # dt >= 12 tau
           dict(order=6), dict(order=5, flux=1), dict(cfl=1.5), dict(W=-1.0),
           dict(precision="fp16f", stages=3, cfl=0.1, M=0.02)]
    for kw in bad:
        with pytest.raises(N.DugksError) as e:
            N.dugks_create(N.make_params(16, 16, **kw), phi0)
        assert e.value.code == N.DUGKS_EINVAL
    with pytest.raises(N.DugksError) as e:
        N.dugks_create(N.make_params(6, 16), np.zeros((16, 6)))
    assert e.value.code == N.DUGKS_EINVAL


def test_nonfinite_input_rejected():
    phi0 = np.zeros((16, 16))
    phi0[3, 4] = np.nan
    with pytest.raises(N.DugksError) as e:
        N.dugks_create(N.make_params(16, 16), phi0)
    assert e.value.code == N.DUGKS_ENONFINITE
