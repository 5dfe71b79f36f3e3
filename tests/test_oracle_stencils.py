"""Pins of the oracle's finite-difference stencils against facts of calculus.

The paper cites isotropic finite differences (Kumar 2004) without coefficients
(Sec. II.B.1, Sec. II.B.2); the oracle derives them from lattice moments. These
tests fix them by exactness on polynomials, the predicted isotropic leading
error, and the measured convergence order on smooth periodic data.
"""
import math

import numpy as np
import pytest

# which -> (m, n): derivative d^m/dx^m d^n/dy^n
DERIV = {0: (1, 0), 1: (0, 1), 2: (2, 0), 3: (1, 1), 4: (0, 2), 5: (3, 0), 6: (2, 1), 7: (1, 2), 8: (0, 3)}


def apply_at_origin(c, a, b):
    """Stencil c[dy+2, dx+2] applied to the monomial x^a y^b, evaluated at (0, 0)."""
    s = 0.0
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            s += c[dy + 2, dx + 2] * float(dx) ** a * float(dy) ** b
    return s


def exact_at_origin(m, n, a, b):
    return float(math.factorial(m) * math.factorial(n)) if (a, b) == (m, n) else 0.0


def lap_derivative_at_origin(m, n, a, b, power):
    """(d^m_x d^n_y) lap^power (x^a y^b) at the origin."""
    total = 0.0
    for i in range(power + 1):
        coef = math.comb(power, i)
        total += coef * exact_at_origin(m + 2 * i, n + 2 * (power - i), a, b)
    return total


EXACT_DEGREE = {  # (order, which) -> highest polynomial degree differentiated exactly
    **{(o, w): 2 for o in (2, 3) for w in (0, 1)},
    **{(o, w): 3 for o in (2, 3) for w in (2, 3, 4)},
    **{(4, w): 4 for w in (0, 1)},
    **{(4, w): 5 for w in (2, 3, 4)},
    **{(4, w): 4 for w in (5, 6, 7, 8)},
}


@pytest.mark.parametrize("order,which", sorted(EXACT_DEGREE))
def test_polynomial_exactness(oracle, order, which):
    c = oracle.stencil(order, which)
    m, n = DERIV[which]
    deg = EXACT_DEGREE[(order, which)]
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            assert apply_at_origin(c, a, b) == pytest.approx(exact_at_origin(m, n, a, b), abs=1e-12), (a, b)
    # one degree higher the stencil must not be exact (it is not of higher order)
    errs = [abs(apply_at_origin(c, a, deg + 1 - a) - exact_at_origin(m, n, a, deg + 1 - a))
            for a in range(deg + 2)]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("which", [0, 1])
def test_nine_point_gradient_leading_error_isotropic(oracle, which):
    """Leading error of the lattice-moment gradient is (1/6) d_a lap F."""
    c = oracle.stencil(2, which)
    m, n = DERIV[which]
    for a in range(4):
        b = 3 - a
        err = apply_at_origin(c, a, b) - exact_at_origin(m, n, a, b)
        assert err == pytest.approx(lap_derivative_at_origin(m, n, a, b, 1) / 6.0, abs=1e-12)


@pytest.mark.parametrize("which", [0, 1])
def test_fourth_order_gradient_leading_error_isotropic(oracle, which):
    """Fifth-order error of the order-4 gradient is alpha d_a lap^2 F, one alpha."""
    c = oracle.stencil(4, which)
    m, n = DERIV[which]
    ratios = []
    for a in range(6):
        b = 5 - a
        err = apply_at_origin(c, a, b) - exact_at_origin(m, n, a, b)
        ref = lap_derivative_at_origin(m, n, a, b, 2)
        if ref == 0.0:
            assert abs(err) < 1e-12
        else:
            ratios.append(err / ref)
    assert len(ratios) == 3 and max(ratios) - min(ratios) < 1e-12 and abs(ratios[0]) > 1e-6


def test_order4_gradient_coefficients_rational(oracle):
    """The moment system has the rational solution 13/30, 2/15, -1/60, -1/60, -1/30."""
    c = oracle.stencil(4, 0)
    expect = {(1, 0): 13 / 30, (1, 1): 2 / 15, (1, 2): -1 / 60, (2, 0): -1 / 60, (2, 1): -1 / 30, (2, 2): 0.0}
    for (ax, ay), v in expect.items():
        for sy in (-1, 1):
            assert c[sy * ay + 2, ax + 2] == pytest.approx(v, abs=1e-14)
            assert c[sy * ay + 2, -ax + 2] == pytest.approx(-v, abs=1e-14)


def _wave(N, kx, ky):
    x = np.arange(N) + 0.5
    X, Y = np.meshgrid(x, x)
    th = 2 * np.pi * (kx * X + ky * Y) / N
    return th, 2 * np.pi / N


@pytest.mark.parametrize("order,which,expect", [
    (2, 0, 2), (2, 2, 2), (2, 3, 2), (4, 0, 4), (4, 1, 4), (4, 2, 4), (4, 3, 4), (4, 5, 2), (4, 6, 2)])
def test_measured_order(oracle, order, which, expect):
    m, n = DERIV[which]
    errs = []
    for N in (32, 64):
        th, k = _wave(N, 1, 2)
        F = np.sin(th)
        # d^m_x d^n_y sin(theta) with theta = k (x + 2 y)
        amp = (k * 1) ** m * (k * 2) ** n
        exact = amp * np.sin(th + (m + n) * np.pi / 2)
        errs.append(np.abs(oracle.derivative(order, which, F) - exact).max() / np.abs(exact).max())
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - expect) < 0.15, (errs, rate)


def test_isotropy_of_nine_point_gradient(oracle):
    """Equal |k| gives equal gradient error for the isotropic stencil; the
    5-point central difference (anisotropic) does not (the paper's diamond)."""
    N = 128
    rel = {}
    rel5 = {}
    for kv in ((5, 0), (3, 4)):
        th, k = _wave(N, *kv)
        F = np.sin(th)
        gx, gy = oracle.derivative(2, 0, F), oracle.derivative(2, 1, F)
        ex, ey = k * kv[0] * np.cos(th), k * kv[1] * np.cos(th)
        rel[kv] = np.abs(np.hypot(gx, gy) - np.hypot(ex, ey)).max()
        g5x = (np.roll(F, -1, 1) - np.roll(F, 1, 1)) / 2
        g5y = (np.roll(F, -1, 0) - np.roll(F, 1, 0)) / 2
        rel5[kv] = np.abs(np.hypot(g5x, g5y) - np.hypot(ex, ey)).max()
    assert rel[(5, 0)] / rel[(3, 4)] == pytest.approx(1.0, abs=0.01)
    assert abs(rel5[(5, 0)] / rel5[(3, 4)] - 1.0) > 0.3
