"""Tile variants of the TMA-staged two-stage kernel (warps x rows per thread).

Every variant of each precision against the FP64 oracle on a ragged grid that
spans several tiles in both directions with a partial last tile, all velocity
kinds; the FP32 variants against each other (same per-cell arithmetic; the
compiler may contract it differently per instantiation, so they agree to
rounding); the batch path with every variant against the single-grid path;
and the rejection of variant numbers outside the table.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

VARIANTS = list(range(6))
FP32_TOL = 5e-5


def problem(nx, ny, kind, seed):
    rng = np.random.default_rng(WL.SEED_BASE + 40 + seed)
    cents = [tuple(rng.uniform(0, [nx, ny])) for _ in range(3)]
    phi0 = WL.drops(nx, ny, cents, [min(nx, ny) / 5, min(nx, ny) / 7, min(nx, ny) / 9], 4.0)
    vel = {"uniform": (0.03, -0.02), "rotation": (nx / 2, ny / 2, 1.5e-3), "vortex": (float(nx), 0.04, 30.0)}[kind]
    return phi0, vel


def oracle_phi(O, nx, ny, phi0, order, flux, kind, vel, steps):
    p = O.Params(nx, ny, W=4.0, M=0.02, cfl=0.8, order=order, flux=flux, stages=2, vel_kind=kind, vel=vel)
    return O.State(p, phi0).run(steps).phi()


def solver_phi(nx, ny, phi0, order, flux, kind, vel, steps, precision, variant):
    with N.Solver(nx, ny, phi0, vel_kind=kind, vel=vel, W=4.0, M=0.02, cfl=0.8, order=order, flux=flux,
                  stages=2, precision=precision) as s:
        s.set_variant(variant)
        assert N.dugks_get_variant(s.ctx) == variant
        s.step(steps)
        assert s.status() == 0
        return s.phi()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("order,flux", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_fp32_variants_match_oracle(oracle, variant, order, flux):
    nx, ny = 77, 70      # 3 x 5 tiles of 31 x 15, 3 x 3 of 31 x 31: ragged in both directions
    kind = ["uniform", "rotation", "vortex"][(order + flux + variant) % 3]
    phi0, vel = problem(nx, ny, kind, seed=order * 2 + flux)
    ref = oracle_phi(oracle, nx, ny, phi0, order, flux, kind, vel, 60)
    phi = solver_phi(nx, ny, phi0, order, flux, kind, vel, 60, "fp32", variant)
    assert np.abs(phi - ref).max() < FP32_TOL


@pytest.mark.parametrize("variant", VARIANTS)
def test_fp64_variants_match_oracle(oracle, variant):
    nx, ny = 77, 70
    kind = ["uniform", "rotation", "vortex"][variant % 3]
    phi0, vel = problem(nx, ny, kind, seed=variant)
    ref = oracle_phi(oracle, nx, ny, phi0, 3, 0, kind, vel, 40)
    phi = solver_phi(nx, ny, phi0, 3, 0, kind, vel, 40, "fp64", variant)
    assert np.abs(phi - ref).max() / np.abs(ref).max() < 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
def test_fp16f_variants_error_bounded(oracle, variant):
    nx, ny = 77, 70
    phi0, vel = problem(nx, ny, "rotation", seed=11)
    ref = oracle_phi(oracle, nx, ny, phi0, 3, 0, "rotation", vel, 100)
    phi = solver_phi(nx, ny, phi0, 3, 0, "rotation", vel, 100, "fp16f", variant)
    assert np.abs(phi - ref).max() < 1.5e-5   # measured 6.6e-6 to 7.3e-6 over the variants


def test_fp32_variants_agree_to_rounding():
    """Same per-cell arithmetic in every tile shape, up to the contraction of
    multiply-adds chosen per instantiation."""
    nx, ny = 96, 64
    phi0, vel = problem(nx, ny, "vortex", seed=21)
    ref = solver_phi(nx, ny, phi0, 3, 0, "vortex", vel, 100, "fp32", 2)
    for v in VARIANTS:
        assert np.abs(solver_phi(nx, ny, phi0, 3, 0, "vortex", vel, 100, "fp32", v) - ref).max() < 2e-6, v


def test_invalid_variants_rejected():
    phi0, vel = problem(40, 30, "uniform", seed=1)
    with N.Solver(40, 30, phi0, vel=vel, order=3, precision="fp32") as s:
        for v in (6, 9, -2):
            with pytest.raises(N.DugksError):
                s.set_variant(v)
        assert N.dugks_get_variant(s.ctx) == 2
    with N.Batch(precision="fp32", W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2) as b:
        b.add(phi0, "uniform", vel)
        for v in (-1, 6):
            with pytest.raises(N.DugksError):
                b.set_variant(v)


@pytest.mark.parametrize("precision", ["fp32", "fp16f"])
def test_batch_variants_match_single_grid(precision):
    """Mixed batch with each variant: every grid equals its single-grid run with the
    same variant (same tile body; only the host- versus device-computed time
    factors of the vortex may round differently)."""
    grids = []
    for i, (nx, ny, kind) in enumerate([(45, 27, "uniform"), (64, 64, "rotation"), (33, 40, "vortex")]):
        phi0, vel = problem(nx, ny, kind, seed=30 + i)
        grids.append((phi0, kind, vel))
    for v in VARIANTS:
        with N.Batch(precision=precision, W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2) as b:
            b.set_variant(v)
            ids = [b.add(p0, k, vel) for p0, k, vel in grids]
            b.step(13)
            assert b.status() == 0
            for gid, (p0, k, vel) in zip(ids, grids):
                ny, nx = p0.shape
                solo = solver_phi(nx, ny, p0, 3, 0, k, vel, 13, precision, v)
                tol = 2e-6 if precision == "fp32" else 2e-5
                assert np.abs(b.phi(gid) - solo).max() < tol, (v, gid)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("order,flux", [(2, 0), (3, 0), (3, 1), (4, 0), (4, 1)])
def test_three_stage_fast_matches_oracle_and_generic(oracle, precision, order, flux):
    """The TMA-staged kernels of the three-stage scheme (two per step: tilde f at t'
    with the accumulator, then hat f) against the oracle and against the generic
    kernels, on a ragged grid with the single vortex."""
    nx, ny, steps = 77, 70, 40
    phi0, vel = problem(nx, ny, "vortex", seed=50 + order * 2 + flux)
    p = oracle.Params(nx, ny, W=4.0, M=0.02, cfl=0.5, order=order, flux=flux, stages=3, vel_kind="vortex", vel=vel)
    ref = oracle.State(p, phi0).run(steps).phi()
    out = {}
    for v in (2, -1):   # fast, generic
        with N.Solver(nx, ny, phi0, vel_kind="vortex", vel=vel, W=4.0, M=0.02, cfl=0.5, order=order, flux=flux,
                      stages=3, precision=precision) as s:
            s.set_variant(v)
            assert N.dugks_get_variant(s.ctx) == v
            s.step(steps)
            assert s.status() == 0
            out[v] = (s.phi(), s.mass())
    if precision == "fp64":
        for v in out:
            assert np.abs(out[v][0] - ref).max() / np.abs(ref).max() < 1e-12, v
        assert abs(out[2][1] - out[-1][1]) / out[-1][1] < 1e-13
    else:
        for v in out:
            assert np.abs(out[v][0] - ref).max() < FP32_TOL, v
        assert np.abs(out[2][0] - out[-1][0]).max() < 2e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16f"])
@pytest.mark.parametrize("flux", [0, 1])
def test_order4_fast_matches_oracle_and_generic(oracle, precision, flux):
    """Order 4 (radius-2 stencils: 5-cell state halo, 3-cell cell-quantity halo,
    5 x 6 face stencils) on the TMA-staged path against the oracle and the generic
    kernel, ragged grid, rotation."""
    nx, ny, steps = 77, 70, 60
    phi0, vel = problem(nx, ny, "rotation", seed=60 + flux)
    p = oracle.Params(nx, ny, W=4.0, M=0.02, cfl=0.8, order=4, flux=flux, stages=2, vel_kind="rotation", vel=vel)
    ref = oracle.State(p, phi0).run(steps).phi()
    out = {}
    for v in (2, -1):
        with N.Solver(nx, ny, phi0, vel_kind="rotation", vel=vel, W=4.0, M=0.02, cfl=0.8, order=4, flux=flux,
                      stages=2, precision=precision) as s:
            s.set_variant(v)
            assert N.dugks_get_variant(s.ctx) == v
            s.step(steps)
            assert s.status() == 0
            out[v] = s.phi()
    tol = {"fp64": 1e-12, "fp32": FP32_TOL, "fp16f": 1.5e-5}[precision]   # FP16: measured 4.5e-6 to 7.1e-6
    for v in out:
        err = np.abs(out[v] - ref).max()
        assert (err / np.abs(ref).max() if precision == "fp64" else err) < tol, (v, err)


SMALL_GRIDS = [(8, 11), (9, 12), (31, 31), (33, 36), (62, 93), (63, 32), (100, 47)]


@pytest.mark.parametrize("nx,ny", SMALL_GRIDS)
@pytest.mark.parametrize("order,flux", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_fp32_odd_grids_every_velocity_kind(oracle, nx, ny, order, flux):
    """The two default tiles (8 x 2 and 8 x 3) on grids smaller than a tile, one
    tile wide, multiples of 31 and one past them, with every velocity kind (the
    cell field included): against the oracle (FP32 bound) and against each other
    (rounding only)."""
    kinds = ["uniform", "rotation", "vortex", "field"]
    kind = kinds[(nx + ny + order + flux) % 4]
    rng = np.random.default_rng(WL.SEED_BASE + 70 + nx + ny)
    phi0 = WL.drops(nx, ny, [tuple(rng.uniform(0, [nx, ny]))], [min(nx, ny) / 3], 4.0)
    steps = 50
    if kind == "field":
        x = np.arange(nx) + 0.5
        y = np.arange(ny) + 0.5
        u = 0.03 * np.sin(2 * np.pi * y / ny)[:, None] * np.ones((1, nx))
        v = 0.02 * np.cos(2 * np.pi * x / nx)[None, :] * np.ones((ny, 1))
        p = oracle.Params(nx, ny, W=4.0, M=0.02, cfl=0.8, order=order, flux=flux, stages=2, vel_kind="field",
                          u_field=u, v_field=v)
        ref = oracle.State(p, phi0).run(steps).phi()
        out = {}
        for var in (2, 4):
            with N.Solver(nx, ny, phi0, vel_kind="field", u=u, v=v, W=4.0, M=0.02, cfl=0.8, order=order,
                          flux=flux, stages=2, precision="fp32") as s:
                s.set_variant(var)
                s.step(steps)
                assert s.status() == 0
                out[var] = s.phi()
    else:
        vel = {"uniform": (0.03, -0.02), "rotation": (nx / 2, ny / 2, 1.5e-3),
               "vortex": (float(nx), 0.04, 30.0)}[kind]
        ref = oracle_phi(oracle, nx, ny, phi0, order, flux, kind, vel, steps)
        out = {var: solver_phi(nx, ny, phi0, order, flux, kind, vel, steps, "fp32", var) for var in (2, 4)}
    for var in out:
        assert np.abs(out[var] - ref).max() < FP32_TOL, var
    assert np.abs(out[2] - out[4]).max() < 2e-6
