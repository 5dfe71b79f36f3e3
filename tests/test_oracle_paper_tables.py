"""Oracle pin on the paper's printed numbers: the diagonal translation of Sec. III.A
(N = 128, two-stage, order-3 upwind, CFL 0.8: 8000 steps) reproduces the printed
E_phi within 2% (the paper leaves the initial distribution, d(phi u)/dt and the
stencil coefficients unstated; this build's readings give 0.6%)."""
import pytest

from paper_tables import e_phi, paper_value, problem

pytestmark = pytest.mark.slow


def test_translation_t2s3_cfl08_n128(oracle):
    prob = problem("T2S3", 0.8, 128)
    p = oracle.Params(prob.nx, prob.ny, W=prob.W, M=prob.M, cfl=prob.cfl, order=prob.order, flux=prob.flux,
                      stages=prob.stages, dtphiu=prob.dtphiu, vel_kind=prob.vel_kind, vel=prob.vel)
    phi = oracle.State(p, prob.phi0).run(prob.steps).phi()
    ref = paper_value("T2S3", 0.8, 128)
    assert abs(e_phi(phi, prob.phi0) / ref - 1) < 0.02
