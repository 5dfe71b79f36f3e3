"""Pins of the oracle's full time step against facts the mathematics fixes.

* cell relations of both schemes checked against their definitions
  (Eqs. (18), (19), (23), (29), (31)-(34));
* moments: the source and collision terms carry no mass (Sec. II.B.1);
* periodic mass conservation (fluxes telescope);
* a uniform field is a fixed point; a planar tanh slab at rest is an
  equilibrium of the conservative Allen-Cahn equation (Sec. II.A);
* closed form: with theta = 0 the equation is linear advection-diffusion and a
  Fourier mode decays at exp(-M k^2 t) and drifts at u (pins tau = 3 M, the flux
  sign and the d(phi u)/dt source term);
* symmetry and shift equivariance;
* the three-stage limit dt < 12 tau reproduces the missing table entries
  (Sec. III.A: no three-stage results at C = 0.8 with M = 0.02).
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import workloads as WL

EX = np.array([0, 1, 1, 0, -1, -1, -1, 0, 1])
EY = np.array([0, 0, 1, 1, 1, 0, -1, -1, -1])


@pytest.mark.parametrize("cfl,M", [(0.8, 0.01), (0.5, 0.02), (0.25, 0.002)])
def test_two_stage_relation_from_definitions(oracle, cfl, M):
    """bar f^+ = f + (h/2)(Omega + S) with h = dt/2, from tilde f = f - (dt/2)(Omega + S)."""
    p = oracle.Params(8, 8, M=M, cfl=cfl, stages=2)
    c = oracle.coefficients(p)
    rng = np.random.default_rng(1)
    f, g = rng.standard_normal(50), rng.standard_normal(50)
    tau, dt = 3 * M, cfl
    os_ = -(f - g) / tau                      # Omega + S = -(f - f^eq - tau S)/tau
    ft = f - dt / 2 * os_
    assert c[0] == pytest.approx(dt / 2)
    np.testing.assert_allclose(c[1] * ft + c[2] * g, f + c[0] / 2 * os_, rtol=1e-13, atol=1e-13)
    # and tilde f^+ = (4/3) bar f^+ - (1/3) tilde f equals f + (dt/2)(Omega + S)
    np.testing.assert_allclose(4 / 3 * (c[1] * ft + c[2] * g) - ft / 3, f + dt / 2 * os_, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("cfl,M", [(0.5, 0.02), (0.25, 0.01), (0.1, 0.002)])
def test_three_stage_relations_from_definitions(oracle, cfl, M):
    p = oracle.Params(8, 8, M=M, cfl=cfl, stages=3)
    c = oracle.coefficients(p)
    rng = np.random.default_rng(2)
    f, g = rng.standard_normal(50), rng.standard_normal(50)
    tau, dt = 3 * M, cfl
    os_ = -(f - g) / tau
    fhat = f - dt / 4 * os_                   # Eq. (19)
    A = c[1] * fhat + c[2] * g                # Eq. (31)
    assert c[0] == pytest.approx(dt / 6) and c[3] == pytest.approx(5 * dt / 12)
    np.testing.assert_allclose(A, f + dt / 12 * os_, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(0.75 * A + 0.25 * fhat, f, rtol=1e-12, atol=1e-12)          # Eq. (32)
    np.testing.assert_allclose(1.25 * A - 0.25 * fhat, f + dt / 6 * os_, rtol=1e-12, atol=1e-12)  # Eq. (33)
    ft = f - dt / 6 * os_                     # Eq. (18a) at t'
    np.testing.assert_allclose(c[4] * ft + c[5] * g, f + 5 * dt / 24 * os_, rtol=1e-12, atol=1e-12)  # Eq. (34)
    np.testing.assert_allclose(c[6] * (ft - g), os_, rtol=1e-12, atol=1e-12)                # Eq. (29)


def test_three_stage_quadrature_weights_exact_to_degree_two():
    """Eq. (16): flux weights 3/7, 4/7 at the nodes 1/6, 3/4 (Eq. (20)) and the
    collision weights 3/4, 1/4 at 1/3, 1 integrate 1, t, t^2 over [0, 1] exactly."""
    for nodes, w in ((np.array([1 / 6, 3 / 4]), np.array([3 / 7, 4 / 7])),
                     (np.array([1 / 3, 1.0]), np.array([3 / 4, 1 / 4]))):
        for d in range(3):
            assert np.dot(w, nodes ** d) == pytest.approx(1.0 / (d + 1), abs=1e-15)


def test_moments_of_source_and_equilibrium(oracle):
    n = 16
    phi = WL.drops(n, n, [(8, 8)], [4], 4.0)
    p = oracle.Params(n, n, vel_kind="uniform", vel=(0.03, -0.01))
    V, g = oracle.cell_quantities(p, phi, phi * 0.99, 1.0, 0.2, 0.8, True)
    np.testing.assert_allclose(g.sum(axis=0), phi, atol=1e-15)          # sum f^eq = phi, sum S = 0
    w = np.array([4 / 9] + [1 / 9, 1 / 36] * 4)
    S = w[:, None, None] * (EX[:, None, None] * V[0] + EY[:, None, None] * V[1])
    np.testing.assert_allclose(S.sum(axis=0), 0.0, atol=1e-17)


@pytest.mark.parametrize("order,flux,stages,cfl", [
    (2, 0, 2, 0.8), (3, 0, 2, 0.8), (3, 1, 2, 0.5), (4, 0, 2, 0.8), (3, 0, 3, 0.5), (4, 1, 3, 0.25)])
def test_mass_conserved(oracle, order, flux, stages, cfl):
    n = 32
    phi0 = WL.drops(n, n, [(10.3, 17.1)], [7.0], 4.0)
    p = oracle.Params(n, n, M=0.02, cfl=cfl, order=order, flux=flux, stages=stages,
                      vel_kind="rotation", vel=(16, 16, 2e-3))
    s = oracle.State(p, phi0)
    m0 = s.mass()
    s.run(150)
    assert abs(s.mass() - m0) / m0 < 1e-13


@pytest.mark.parametrize("stages", [2, 3])
def test_uniform_field_is_fixed_point(oracle, stages):
    n = 12
    phi0 = np.full((n, n), 0.3)
    p = oracle.Params(n, n, M=0.02, cfl=0.5, order=3, stages=stages, vel_kind="uniform", vel=(0.04, 0.02))
    s = oracle.State(p, phi0)
    f0 = s.f.copy()
    s.run(40)
    assert np.abs(s.f - f0).max() < 1e-15
    assert np.abs(s.phi() - 0.3).max() < 1e-15
    w = np.array([4 / 9] + [1 / 9, 1 / 36] * 4)
    feq = w * 0.3 * (1 + 3 * (EX * 0.04 + EY * 0.02))
    np.testing.assert_allclose(s.f[:, 0, 0], feq, atol=1e-16)


@pytest.mark.parametrize("order,flux,stages,cfl", [(2, 0, 2, 0.8), (3, 0, 2, 0.8), (2, 1, 2, 0.8),
                                                  (4, 0, 2, 0.8), (3, 0, 3, 0.5)])
def test_planar_slab_is_stationary(oracle, order, flux, stages, cfl):
    """The tanh profile solves phi' = theta, so at u = 0 the slab stays put; the
    drift falls at second order in 1/W (the face-source error, Sec. III.A)."""
    drift = []
    for W in (4.0, 8.0):
        n = int(16 * W)
        phi0 = WL.planar_slab(n, W)[:8].copy()
        p = oracle.Params(n, 8, W=W, M=0.02, cfl=cfl, order=order, flux=flux, stages=stages)
        s = oracle.State(p, phi0)
        s.run(int(5 * W * W / cfl))
        drift.append(np.abs(s.phi() - phi0).max())
    assert drift[0] < 0.025
    assert drift[0] / drift[1] > 2.8


def _fourier_mode(oracle, N, U, M, cfl, order, flux, stages, steps, dtphiu):
    x = np.arange(N) + 0.5
    a = 0.1
    phi0 = np.tile(0.5 + a * np.sin(2 * np.pi * x / N), (8, 1))
    # theta = 4 phi (1 - phi) / W vanishes as W -> infinity: linear advection-diffusion
    p = oracle.Params(N, 8, W=1e12, M=M, cfl=cfl, order=order, flux=flux, stages=stages,
                      dtphiu=dtphiu, vel_kind="uniform", vel=(U, 0.0))
    s = oracle.State(p, phi0).run(steps)
    ph = s.phi()[0] - 0.5
    basis = np.exp(-2j * np.pi * x / N)
    c1, c0 = np.sum(ph * basis), np.sum((phi0[0] - 0.5) * basis)
    t, k = steps * cfl, 2 * np.pi / N
    rate = -np.log(abs(c1) / abs(c0)) / t
    shift = -np.angle(c1 / c0) / k
    return rate / (M * k * k) - 1.0, shift / (U * t) - 1.0


@pytest.mark.parametrize("order,flux,stages,cfl", [(2, 0, 2, 0.8), (3, 0, 2, 0.8), (2, 1, 2, 0.8),
                                                  (4, 0, 2, 0.8), (3, 0, 3, 0.25)])
def test_advection_diffusion_closed_form(oracle, order, flux, stages, cfl):
    """Decay rate M k^2 and drift speed U converge at second order (pins tau = 3M)."""
    errs = []
    for N in (16, 32):
        steps = int(N * N / 16 / cfl)
        errs.append(_fourier_mode(oracle, N, 0.05, 0.05, cfl, order, flux, stages, steps, 1))
    (d16, s16), (d32, s32) = errs
    assert abs(d32) < 7e-3 and abs(s32) < 5e-3
    assert abs(d16) / abs(d32) > 2.3
    assert abs(s16) / max(abs(s32), 1e-12) > 2.3 or abs(s32) < 1e-4


def test_dtphiu_source_removes_velocity_dependent_diffusion(oracle):
    """Without the d(phi u)/dt part of Eq. (14b) the recovered diffusivity is
    M - tau u^2 = M (1 - 3 u^2); with it, the error falls at second order."""
    U = 0.05
    d_no, _ = _fourier_mode(oracle, 64, U, 0.05, 0.8, 2, 0, 2, 320, 0)
    d_yes, _ = _fourier_mode(oracle, 64, U, 0.05, 0.8, 2, 0, 2, 320, 1)
    assert d_no == pytest.approx(-3 * U * U, rel=0.1)
    assert abs(d_yes) < 0.15 * abs(d_no)


def test_centred_drop_keeps_square_symmetry(oracle):
    n = 24
    phi0 = WL.drops(n, n, [(12, 12)], [6.0], 4.0)
    p = oracle.Params(n, n, M=0.02, cfl=0.8, order=3, flux=0, stages=2)
    s = oracle.State(p, phi0).run(60)
    ph = s.phi()
    assert np.abs(ph - ph.T).max() < 1e-14
    assert np.abs(ph - ph[:, ::-1]).max() < 1e-14
    assert np.abs(ph - ph[::-1, :]).max() < 1e-14


def test_integer_shift_equivariance(oracle):
    n = 20
    phi0 = WL.drops(n, n, [(7.3, 9.1)], [5.0], 4.0)
    p = oracle.Params(n, n, M=0.02, cfl=0.8, order=3, vel_kind="uniform", vel=(0.03, 0.01))
    a = oracle.State(p, phi0).run(30).phi()
    b = oracle.State(p, np.roll(phi0, (3, 5), axis=(0, 1))).run(30).phi()
    assert np.abs(np.roll(a, (3, 5), axis=(0, 1)) - b).max() < 1e-15


def test_three_stage_time_step_limit_matches_paper(oracle):
    """With tau = 3 M the limit dt < 12 tau removes exactly the C = 0.8, M = 0.02
    three-stage runs and keeps C = 0.5 (Sec. III.A)."""
    assert not oracle.check(oracle.Params(16, 16, M=0.02, cfl=0.8, stages=3))
    assert oracle.check(oracle.Params(16, 16, M=0.02, cfl=0.5, stages=3))
    assert oracle.check(oracle.Params(16, 16, M=0.02, cfl=0.8, stages=2))
