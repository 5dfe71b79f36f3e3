"""Pins of the oracle's prescribed velocity fields and of the time levels at which
the step evaluates them (Sec. II.A: u prescribed and divergence free; Eq. (14b):
the d(phi u)/dt source; Eqs. (24)-(28): faces at t_n + h; Sec. II.B.2: the
three-stage faces at t_n + dt/6 and t_n + 3 dt/4 and the cell stage at t').

* Every analytic field (rotation, single vortex, the smoothed deformation of
  Sec. III.D) is checked against a stream function psi, written here
  independently of the oracle's formulas: u = -d psi / dy, v = d psi / dx, taken
  by central differences of psi. That fixes sign, axis, amplitude and the
  cos(pi t / T) reversal, and makes the fields divergence free by construction;
  the discrete divergence of the oracle's own field is checked too.
* The rigid rotation turns a blob anticlockwise about its centre: after a
  quarter turn its centroid sits where the exact rotation puts it.
* Time levels: under a uniform flow reversed by cos(pi t / T), a Fourier mode
  returns exactly to its start at t = T (the displacement is
  U T / pi sin(pi t / T)), and the spatial phase errors of the scheme cancel
  between the outward and return legs. What remains is the time error of the
  stepping, second order when the faces see u at t_n + h, the cell stage at t
  and the backward difference of phi u spans t_old = t_n - dt. Evaluating the
  faces at t_n, dropping t_old, or misplacing either three-stage level leaves a
  net shift of 3.5e-4 to 3.7e-2 cells instead of below 4e-5.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import workloads as WL


def _psi_vortex(L, U, T):
    # u = -U sin^2(pi x/L) sin(2 pi y/L) c(t), v = U sin^2(pi y/L) sin(2 pi x/L) c(t)
    # derive from psi = (U L / pi) sin^2(pi x/L) sin^2(pi y/L) cos(pi t/T)
    return lambda x, y, t: U * L / np.pi * np.sin(np.pi * x / L) ** 2 * np.sin(np.pi * y / L) ** 2 * np.cos(
        np.pi * t / T)


def _psi_rotation(cx, cy, om):
    # anticlockwise rigid rotation at angular speed om: psi = om r^2 / 2
    return lambda x, y, t: 0.5 * om * ((x - cx) ** 2 + (y - cy) ** 2)


def _psi_deformation(L, U, T):
    # u = -U sin(4 pi x/L) sin(4 pi y/L) c(t), v = -U cos(4 pi x/L) cos(4 pi y/L) c(t)
    # derive from psi = -(U L / 4 pi) sin(4 pi x/L) cos(4 pi y/L) cos(pi t/T)
    a = 4 * np.pi / L
    return lambda x, y, t: -U / a * np.sin(a * x) * np.cos(a * y) * np.cos(np.pi * t / T)


def _from_psi(psi, x, y, t, e=1e-4):
    return np.array([-(psi(x, y + e, t) - psi(x, y - e, t)) / (2 * e),
                     (psi(x + e, y, t) - psi(x - e, y, t)) / (2 * e)])


@pytest.mark.parametrize("kind,vel,psi", [
    ("vortex", (128.0, 0.05, 819.2), _psi_vortex(128.0, 0.05, 819.2)),
    ("vortex", (1.0, 1.3, 8.0), _psi_vortex(1.0, 1.3, 8.0)),
    ("rotation", (128.0, 128.0, 2 * np.pi / 13107.2), _psi_rotation(128.0, 128.0, 2 * np.pi / 13107.2)),
    ("rotation", (3.0, -2.0, -0.7), _psi_rotation(3.0, -2.0, -0.7)),
    ("deformation", (512.0, 0.04, 12800.0), _psi_deformation(512.0, 0.04, 12800.0)),
    ("deformation", (64.0, 1.0, 3.0), _psi_deformation(64.0, 1.0, 3.0)),
])
def test_velocity_is_the_curl_of_its_stream_function(oracle, kind, vel, psi):
    p = oracle.Params(16, 16, vel_kind=kind, vel=vel)
    rng = np.random.default_rng(2007077611)
    scale = vel[0] if kind in ("vortex", "deformation") else 100.0
    T = vel[2] if kind in ("vortex", "deformation") else 1.0
    for _ in range(200):
        x, y = rng.uniform(-0.5, 1.5, 2) * scale
        t = rng.uniform(0, 2.5) * T
        got = oracle.velocity(p, x, y, t)
        ref = _from_psi(psi, x, y, t)
        mag = np.abs(_from_psi(psi, x, y, 0.0)).max() + 1e-300
        assert np.abs(got - ref).max() <= 1e-6 * mag + 1e-12, (x, y, t, got, ref)


def test_vortex_reverses_and_vanishes_at_half_period(oracle):
    L, U, T = 64.0, 0.05, 100.0
    p = oracle.Params(16, 16, vel_kind="vortex", vel=(L, U, T))
    # at (L/4, L/2): sin^2(pi/4) sin(pi) = 0 and sin^2(pi/2) sin(pi/2) = 1
    np.testing.assert_allclose(oracle.velocity(p, L / 4, L / 2, 0.0), [0.0, U], atol=1e-15)
    rng = np.random.default_rng(7)
    for x, y in rng.uniform(0, L, (20, 2)):
        u0 = oracle.velocity(p, x, y, 0.0)
        assert np.abs(oracle.velocity(p, x, y, T / 2)).max() < 1e-15
        np.testing.assert_allclose(oracle.velocity(p, x, y, T), -u0, atol=1e-16)
        np.testing.assert_allclose(oracle.velocity(p, x, y, 2 * T), u0, atol=1e-16)


@pytest.mark.parametrize("kind,vel", [("vortex", (64.0, 0.05, 50.0)), ("rotation", (20.0, 30.0, 0.01)),
                                      ("deformation", (256.0, 0.05, 50.0))])
def test_discrete_divergence_vanishes(oracle, kind, vel):
    p = oracle.Params(16, 16, vel_kind=kind, vel=vel)
    rng = np.random.default_rng(11)
    for e in (0.5, 0.25):
        worst = 0.0
        for x, y in rng.uniform(0, 64, (50, 2)):
            du = oracle.velocity(p, x + e, y, 3.0)[0] - oracle.velocity(p, x - e, y, 3.0)[0]
            dv = oracle.velocity(p, x, y + e, 3.0)[1] - oracle.velocity(p, x, y - e, 3.0)[1]
            worst = max(worst, abs(du + dv) / (2 * e))
        # exactly zero for the rotation; second-order truncation (~ U k^3 e^2) for the others
        k = np.pi / 64 if kind == "vortex" else 4 * np.pi / 256
        assert worst < (1e-15 if kind == "rotation" else 4 * 0.05 * k ** 3 * e * e + 1e-16)


def test_cell_field_face_value_is_the_mean_of_its_cells(oracle):
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal((2, 9, 10))
    p = oracle.Params(10, 9, vel_kind="field", u_field=u, v_field=v)
    for i, j in [(0, 0), (3, 4), (9, 8), (5, 0)]:
        east = oracle.velocity(p, i + 1.0, j + 0.5, 0.0)
        north = oracle.velocity(p, i + 0.5, j + 1.0, 0.0)
        ie, jn = (i + 1) % 10, (j + 1) % 9
        np.testing.assert_allclose(east, [(u[j, i] + u[j, ie]) / 2, (v[j, i] + v[j, ie]) / 2], rtol=1e-15)
        np.testing.assert_allclose(north, [(u[j, i] + u[jn, i]) / 2, (v[j, i] + v[jn, i]) / 2], rtol=1e-15)
        np.testing.assert_allclose(oracle.velocity(p, i + 0.5, j + 0.5, 0.0), [u[j, i], v[j, i]], rtol=1e-15)


def test_rotation_turns_a_blob_anticlockwise(oracle):
    """A blob at (44, 32) on a 64^2 grid rotated about (32, 32) for a quarter turn
    ends at (32, 44): the centroid moves there within a tenth of a cell."""
    n, steps, cfl = 64, 400, 0.8
    om = 0.5 * np.pi / (steps * cfl)
    phi0 = WL.drops(n, n, [(44.0, 32.0)], [6.0], 4.0)
    p = oracle.Params(n, n, M=0.002, cfl=cfl, order=3, flux=0, vel_kind="rotation", vel=(32.0, 32.0, om))
    ph = oracle.State(p, phi0).run(steps).phi()
    x = np.arange(n) + 0.5
    cx = (ph * x[None, :]).sum() / ph.sum()
    cy = (ph * x[:, None]).sum() / ph.sum()
    assert abs(cx - 32.0) < 0.1 and abs(cy - 44.0) < 0.1, (cx, cy)


def _net_shift_after_reversal(oracle, N, stages, cfl, order, flux, U=0.08, M=0.05):
    x = np.arange(N) + 0.5
    phi0 = np.tile(0.5 + 0.1 * np.sin(2 * np.pi * x / N), (8, 1))
    steps = 4 * N
    T = steps * cfl    # u = U cos(pi t / T): out and back, the mode ends where it started
    # theta -> 0 as W -> infinity: linear advection-diffusion
    p = oracle.Params(N, 8, W=1e12, M=M, cfl=cfl, order=order, flux=flux, stages=stages, dtphiu=1,
                      vel_kind="reversing", vel=(U, 0.0, T))
    ph = oracle.State(p, phi0).run(steps).phi()[0] - 0.5
    basis = np.exp(-2j * np.pi * x / N)
    c1, c0 = np.sum(ph * basis), np.sum((phi0[0] - 0.5) * basis)
    return -np.angle(c1 / c0) / (2 * np.pi / N)


@pytest.mark.parametrize("stages,cfl", [(2, 0.8), (2, 0.4), (3, 0.25), (3, 0.5)])
@pytest.mark.parametrize("order,flux", [(2, 0), (3, 0), (2, 1), (4, 0)])
def test_time_levels_return_a_reversed_mode_to_its_start(oracle, stages, cfl, order, flux):
    s32 = _net_shift_after_reversal(oracle, 32, stages, cfl, order, flux)
    s64 = _net_shift_after_reversal(oracle, 64, stages, cfl, order, flux)
    assert abs(s64) < 1e-4, s64
    assert abs(s32) / abs(s64) > 3.3, (s32, s64)   # second order in time (dt = cfl, N-proportional run)
