"""Pins of the oracle's face reconstruction (Eqs. (24)-(26), Sec. II.B.2), and of the
fifth-order reconstruction of DUGKS-T2S5 (Sec. III.A) against numpy's polynomial fit.

An independent per-face routine finds the cell centre nearest to the
back-traced point x_b - xi h by explicit geometric search (ties averaged), and
expands a Taylor series there with derivatives written out as neighbour sums.
"""
import numpy as np
import pytest

EX = [0, 1, 1, 0, -1, -1, -1, 0, 1]
EY = [0, 0, 1, 1, 1, 0, -1, -1, -1]


def _sh(F, dx, dy):
    """F evaluated at (i + dx, j + dy) on the periodic grid."""
    return np.roll(np.roll(F, -dy, axis=0), -dx, axis=1)


def nine_point_derivs(F):
    """Lattice-moment gradient and Hessian written out as neighbour sums."""
    E, W, N, S = _sh(F, 1, 0), _sh(F, -1, 0), _sh(F, 0, 1), _sh(F, 0, -1)
    NE, NW, SE, SW = _sh(F, 1, 1), _sh(F, -1, 1), _sh(F, 1, -1), _sh(F, -1, -1)
    gx = (E - W) / 3 + (NE + SE - NW - SW) / 12
    gy = (N - S) / 3 + (NE + NW - SE - SW) / 12
    corners = NE + NW + SE + SW
    hxx = 2 / 3 * (E + W) - 1 / 3 * (N + S) + corners / 6 - 4 / 3 * F
    hyy = 2 / 3 * (N + S) - 1 / 3 * (E + W) + corners / 6 - 4 / 3 * F
    hxy = (NE - NW - SE + SW) / 4
    return dict(gx=gx, gy=gy, hxx=hxx, hxy=hxy, hyy=hyy)


def derivs(oracle, F, order):
    if order in (2, 3):
        return nine_point_derivs(F)
    names = ["gx", "gy", "hxx", "hxy", "hyy", "txxx", "txxy", "txyy", "tyyy"]
    return {n: oracle.derivative(4, w, F) for w, n in enumerate(names)}


def taylor(D, F, i, j, dx, dy, order):
    v = F[j, i] + dx * D["gx"][j, i] + dy * D["gy"][j, i]
    if order >= 3:
        v += 0.5 * dx * dx * D["hxx"][j, i] + dx * dy * D["hxy"][j, i] + 0.5 * dy * dy * D["hyy"][j, i]
    if order >= 4:
        v += (dx ** 3 * D["txxx"][j, i] + 3 * dx * dx * dy * D["txxy"][j, i]
              + 3 * dx * dy * dy * D["txyy"][j, i] + dy ** 3 * D["tyyy"][j, i]) / 6
    return v


def brute_faces(oracle, fbp, h, order, flux):
    _, ny, nx = fbp.shape
    outE = np.zeros_like(fbp)
    outN = np.zeros_like(fbp)
    for k in range(9):
        F = fbp[k]
        D = derivs(oracle, F, order)
        for j in range(ny):
            for i in range(nx):
                for face, (xb, yb), out in ((0, (i + 1.0, j + 0.5), outE), (1, (i + 0.5, j + 1.0), outN)):
                    if flux == 0:
                        qx, qy = xb - EX[k] * h, yb - EY[k] * h
                        cands = []
                        for ci in range(i - 1, i + 3):
                            for cj in range(j - 1, j + 3):
                                d = np.hypot(qx - (ci + 0.5), qy - (cj + 0.5))
                                cands.append((d, ci, cj))
                        dmin = min(c[0] for c in cands)
                        near = [c for c in cands if c[0] <= dmin + 1e-12]
                        vals = [taylor(D, F, ci % nx, cj % ny, qx - (ci + 0.5), qy - (cj + 0.5), order)
                                for _, ci, cj in near]
                        out[k, j, i] = sum(vals) / len(vals)
                    else:
                        if face == 0:
                            L, R = F[j, i], F[j, (i + 1) % nx]
                            gn = R - L
                            gt = 0.5 * (D["gy"][j, i] + D["gy"][j, (i + 1) % nx])
                            gxb, gyb = gn, gt
                        else:
                            L, R = F[j, i], F[(j + 1) % ny, i]
                            gn = R - L
                            gt = 0.5 * (D["gx"][j, i] + D["gx"][(j + 1) % ny, i])
                            gxb, gyb = gt, gn
                        out[k, j, i] = 0.5 * (L + R) - h * (EX[k] * gxb + EY[k] * gyb)
    return outE, outN


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("h", [0.4, 0.25, 1 / 12, 1 / 3])
def test_faces_match_brute_force(oracle, order, flux, h):
    rng = np.random.default_rng(11 + order + 10 * flux)
    p = oracle.Params(8, 8, order=order, flux=flux)
    fbp = rng.standard_normal((9, 8, 8))
    E, N = oracle.reconstruct(p, fbp, h)
    bE, bN = brute_faces(oracle, fbp, h, order, flux)
    assert np.abs(E - bE).max() < 1e-13
    assert np.abs(N - bN).max() < 1e-13


@pytest.mark.parametrize("order", [2, 3, 4])
def test_upwind_reproduces_polynomial_exactly(oracle, order):
    """Upwind reconstruction of a degree-(order-1) polynomial returns the
    polynomial's value at the back-traced point (away from the periodic seam)."""
    n = 20
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    rng = np.random.default_rng(5)
    deg = order - 1
    coef = rng.standard_normal((deg + 1, deg + 1))

    def poly(px, py):
        return sum(coef[a, b] * (px - 10) ** a * (py - 10) ** b
                   for a in range(deg + 1) for b in range(deg + 1 - a))

    fbp = np.stack([poly(X, Y)] * 9)
    h = 0.35
    p = oracle.Params(n, n, order=order, flux=0)
    E, N = oracle.reconstruct(p, fbp, h)
    for k in range(9):
        for j in range(5, 15):
            for i in range(5, 15):
                assert E[k, j, i] == pytest.approx(poly(i + 1.0 - EX[k] * h, j + 0.5 - EY[k] * h), abs=1e-9)
                assert N[k, j, i] == pytest.approx(poly(i + 0.5 - EX[k] * h, j + 1.0 - EY[k] * h), abs=1e-9)


def test_face_value_order_on_smooth_data(oracle):
    """Upwind face values converge at (at least) the stencil order p on a smooth
    periodic field: the local error of an order-(p-1) Taylor expansion is O(dx^p)."""
    errs = {2: [], 3: [], 4: []}
    for n in (32, 64):
        x = np.arange(n) + 0.5
        X, Y = np.meshgrid(x, x)
        k = 2 * np.pi / n
        fbp = np.stack([np.sin(k * (X + 2 * Y))] * 9)
        h = 0.3
        for order in (2, 3, 4):
            p = oracle.Params(n, n, order=order, flux=0)
            E, _ = oracle.reconstruct(p, fbp, h)
            ex = np.stack([np.sin(k * ((X + 0.5 - EX[q] * h) + 2 * (Y - EY[q] * h))) for q in range(9)])
            errs[order].append(np.abs(E - ex).max())
    for order in (2, 3):
        rate = np.log2(errs[order][0] / errs[order][1])
        assert abs(rate - order) < 0.2, (order, rate)
    # order 4: at least fourth order (its fifth-order terms still dominate here)
    assert np.log2(errs[4][0] / errs[4][1]) > 3.8
    assert errs[4][1] < errs[3][1] < errs[2][1]


# ---- order 5: DUGKS-T2S5 (Sec. III.A: fifth-order, not isotropic; no stencil printed) ----
def _interp_polyfit(F, m, n, qx, qy):
    """Degree-4 interpolant through the 5 x 5 cells around cell (m, n), evaluated at
    q: numpy's polynomial fit row by row, then across the rows (an independent
    construction of the same tensor-product interpolant)."""
    ny, nx = F.shape
    xs = np.arange(m - 2, m + 3) + 0.5
    ys = np.arange(n - 2, n + 3) + 0.5
    rows = []
    for y in range(n - 2, n + 3):
        vals = [F[y % ny, x % nx] for x in range(m - 2, m + 3)]
        rows.append(np.polyval(np.polyfit(xs - qx, vals, 4), 0.0))
    return np.polyval(np.polyfit(ys - qy, rows, 4), 0.0)


def _brute5(fbp, h):
    _, ny, nx = fbp.shape
    outE, outN = np.zeros_like(fbp), np.zeros_like(fbp)
    for k in range(9):
        F = fbp[k]
        for j in range(ny):
            for i in range(nx):
                for (xb, yb), out, face in (((i + 1.0, j + 0.5), outE, 0), ((i + 0.5, j + 1.0), outN, 1)):
                    qx, qy = xb - EX[k] * h, yb - EY[k] * h
                    # the cell centres nearest to q along the face normal (both on a tie);
                    # along the face q stays in the face's row or column
                    if face == 0:
                        d = [abs(qx - (c + 0.5)) for c in (i, i + 1)]
                        cells = [(c, j) for c, dc in zip((i, i + 1), d) if dc <= min(d) + 1e-12]
                    else:
                        d = [abs(qy - (c + 0.5)) for c in (j, j + 1)]
                        cells = [(i, c) for c, dc in zip((j, j + 1), d) if dc <= min(d) + 1e-12]
                    out[k, j, i] = np.mean([_interp_polyfit(F, m, n, qx, qy) for m, n in cells])
    return outE, outN


@pytest.mark.parametrize("h", [0.4, 0.25, 0.5, 1 / 12])
def test_order5_faces_match_brute_force(oracle, h):
    rng = np.random.default_rng(51)
    p = oracle.Params(10, 9, order=5, flux=0)
    fbp = rng.standard_normal((9, 9, 10))
    E, N = oracle.reconstruct(p, fbp, h)
    bE, bN = _brute5(fbp, h)
    assert np.abs(E - bE).max() < 1e-11
    assert np.abs(N - bN).max() < 1e-11


def test_order5_reproduces_degree_four_in_each_variable(oracle):
    n = 24
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    rng = np.random.default_rng(52)
    coef = rng.standard_normal((5, 5)) * 0.1

    def poly(px, py):
        return sum(coef[a, b] * ((px - 12) / 4) ** a * ((py - 12) / 4) ** b for a in range(5) for b in range(5))

    fbp = np.stack([poly(X, Y)] * 9)
    h = 0.3
    E, N = oracle.reconstruct(oracle.Params(n, n, order=5, flux=0), fbp, h)
    for k in range(9):
        for j in range(6, 18):
            for i in range(6, 18):
                assert E[k, j, i] == pytest.approx(poly(i + 1.0 - EX[k] * h, j + 0.5 - EY[k] * h), abs=1e-10)
                assert N[k, j, i] == pytest.approx(poly(i + 0.5 - EX[k] * h, j + 1.0 - EY[k] * h), abs=1e-10)


def test_order5_face_values_converge_at_fifth_order(oracle):
    errs = []
    for n in (32, 64):
        x = np.arange(n) + 0.5
        X, Y = np.meshgrid(x, x)
        k = 2 * np.pi / n
        fbp = np.stack([np.sin(k * (X + 2 * Y))] * 9)
        h = 0.3
        E, _ = oracle.reconstruct(oracle.Params(n, n, order=5, flux=0), fbp, h)
        ex = np.stack([np.sin(k * ((X + 0.5 - EX[q] * h) + 2 * (Y - EY[q] * h))) for q in range(9)])
        errs.append(np.abs(E - ex).max())
    assert abs(np.log2(errs[0] / errs[1]) - 5) < 0.3, errs


def test_order5_only_upwind_two_stage(oracle):
    assert oracle.check(oracle.Params(16, 16, order=5, flux=0, stages=2))
    assert not oracle.check(oracle.Params(16, 16, order=5, flux=1, stages=2))
    assert not oracle.check(oracle.Params(16, 16, order=5, flux=0, stages=3, cfl=0.5, M=0.02))
