/*
 * dugks_oracle.c -- plain, slow, FP64 CPU oracle of the DUGKS time step for the
 * conservative Allen-Cahn equation (Yang, Zhong & Zhuo, "Performance evaluation
 * of high-order reconstruction for discrete unified gas-kinetic scheme in
 * tracking fluid interfaces").
 *
 * TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code with the CUDA library.
 *
 * Every stage is a whole-grid pass over plain arrays in the order the method
 * states it; there is no tiling, fusion or reordering. Readings of points the
 * paper leaves open are marked "Reading:".
 *
 * Notation (Sec. II.B): D2Q9 with xi_k = sqrt(3 RT) e_k = e_k since RT = 1/3,
 * weights 4/9, 1/9, 1/36; tau = M / RT (Reading: the paper never writes the
 * link; it is the Chapman-Enskog relation and matches the missing three-stage
 * entries where dt >= 12 tau); dt = C (Eq. (39) with unit cells).
 *
 * Parity pins: stencils by polynomial exactness and measured order; face values
 * by an independent brute-force routine; the step by mass conservation, uniform
 * invariance, the stationary tanh slab, and the closed-form decay and drift of a
 * Fourier mode under advection-diffusion (theta = 0); the velocity fields by
 * their stream functions, and the time levels at which the step evaluates them
 * by a mode that a reversing flow must return to its start (test-only velocity
 * kind 4).
 */
#include "dugks_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
/* Velocity order of Sec. II.B.2: (0,0),(1,0),(1,1),(0,1),(-1,1),(-1,0),(-1,-1),(0,-1),(1,-1). */
static const int EX[Q] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static const int EY[Q] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
static const double WQ[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0,
                             1.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0};
static const double RT = 1.0 / 3.0;
static const double PI = 3.14159265358979323846;

static int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static size_t idx(const orc_params *p, int i, int j) {
    return (size_t)wrapi(j, p->ny) * (size_t)p->nx + (size_t)wrapi(i, p->nx);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Isotropic finite-difference stencils (Sec. II.B.1 cites Kumar 2004 for them  */
/* without coefficients). Each is derived here from lattice moments.           */
/* ------------------------------------------------------------------------ */

#define S5(dx, dy) (((dy) + 2) * 5 + ((dx) + 2))

/* Adds scale * (1/cs^2) sum_k w_k e_ka F(x + s e_k) / s : the D2Q9 moment
 * gradient at spacing s (cs^2 = RT). Leading error (s^2/6) d_a lap F, isotropic. */
static void add_lattice_gradient(int axis, int s, double scale, double c[25]) {
    for (int k = 0; k < Q; k++) {
        int e = axis == 0 ? EX[k] : EY[k];
        c[S5(s * EX[k], s * EY[k])] += scale * WQ[k] * e / RT / s;
    }
}

/* Adds scale * (1/cs^4) sum_k w_k (e_ka e_kb - cs^2 delta_ab) F(x + s e_k) / s^2. */
static void add_lattice_hessian(int a, int b, int s, double scale, double c[25]) {
    for (int k = 0; k < Q; k++) {
        int ea = a == 0 ? EX[k] : EY[k];
        int eb = b == 0 ? EX[k] : EY[k];
        double m = ea * eb - (a == b ? RT : 0.0);
        c[S5(s * EX[k], s * EY[k])] += scale * WQ[k] * m / (RT * RT) / (double)(s * s);
    }
}

/* Dense solve with partial pivoting; A is n x n row-major, b overwritten by x. */
static int solve_dense(int n, double *A, double *b) {
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (fabs(A[piv * n + c]) < 1e-300) return -1;
        if (piv != c) {
            for (int k = 0; k < n; k++) {
                double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
            }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* Fourth-order d/dx on the 5x5 block without its corners: antisymmetric in x,
 * symmetric in y, weights a(ax, ay) at (+-ax, +-ay). Conditions on the moments
 * m(px, py) = sum c x^px y^py: m(1,0) = 1; m(3,0) = m(1,2) = 0 (no third-order
 * error); the fifth-order error is isotropic, i.e. proportional to d_x lap^2,
 * which needs m(5,0) = 5 m(3,2) = 5 m(1,4). */
static void iso4_gradient_x(double c[25]) {
    static const int PX[5][2] = {{1, 0}, {1, 1}, {1, 2}, {2, 0}, {2, 1}};
    double A[25], b[5] = {1, 0, 0, 0, 0};
    for (int u = 0; u < 5; u++) {
        double m10 = 0, m30 = 0, m12 = 0, m50 = 0, m32 = 0, m14 = 0;
        for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2) {
                if (PX[u][1] == 0 && sy == 1) continue;   /* (ax, 0) counted once */
                double x = sx * PX[u][0], y = sy * PX[u][1], w = sx;
                m10 += w * x; m30 += w * x * x * x; m12 += w * x * y * y;
                m50 += w * pow(x, 5); m32 += w * x * x * x * y * y; m14 += w * x * pow(y, 4);
            }
        A[0 * 5 + u] = m10; A[1 * 5 + u] = m30; A[2 * 5 + u] = m12;
        A[3 * 5 + u] = m50 - 5 * m32; A[4 * 5 + u] = m50 - 5 * m14;
    }
    solve_dense(5, A, b);
    for (int u = 0; u < 5; u++)
        for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2) {
                if (PX[u][1] == 0 && sy == 1) continue;
                c[S5(sx * PX[u][0], sy * PX[u][1])] += sx * b[u];
            }
}

static void transpose25(const double in[25], double out[25]) {
    for (int dy = -2; dy <= 2; dy++)
        for (int dx = -2; dx <= 2; dx++) out[S5(dy, dx)] = in[S5(dx, dy)];
}

int orc_stencil(int order, int which, double c[25]) {
    memset(c, 0, 25 * sizeof(double));
    if (order == 2 || order == 3) {
        switch (which) {
        case 0: add_lattice_gradient(0, 1, 1.0, c); return 0;
        case 1: add_lattice_gradient(1, 1, 1.0, c); return 0;
        case 2: add_lattice_hessian(0, 0, 1, 1.0, c); return 0;
        case 3: add_lattice_hessian(0, 1, 1, 1.0, c); return 0;
        case 4: add_lattice_hessian(1, 1, 1, 1.0, c); return 0;
        default: return -1;
        }
    }
    if (order != 4) return -1;
    double t[25];
    memset(t, 0, sizeof t);
    switch (which) {
    case 0: iso4_gradient_x(c); return 0;
    case 1: iso4_gradient_x(t); transpose25(t, c); return 0;
    case 2: case 3: case 4: {
        /* Reading: Richardson extrapolation (4 H_1 - H_2) / 3 of the lattice
         * Hessians at spacings 1 and 2; fourth order. */
        int a = which == 4 ? 1 : 0, b = which == 2 ? 0 : 1;
        add_lattice_hessian(a, b, 1, 4.0 / 3.0, c);
        add_lattice_hessian(a, b, 2, -1.0 / 3.0, c);
        return 0;
    }
    case 5: case 8: {
        /* Reading: second-order third derivative along one axis,
         * (F(2) - 2 F(1) + 2 F(-1) - F(-2)) / 2. */
        static const double d3[5] = {-0.5, 1.0, 0.0, -1.0, 0.5};
        for (int m = -2; m <= 2; m++) {
            if (which == 5) c[S5(m, 0)] = d3[m + 2];
            else c[S5(0, m)] = d3[m + 2];
        }
        return 0;
    }
    case 6: case 7: {
        /* Mixed third derivatives as products of the 3-point second difference
         * and the central first difference (second order). */
        static const double d2[3] = {1.0, -2.0, 1.0}, d1[3] = {-0.5, 0.0, 0.5};
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) {
                if (which == 6) c[S5(a, b)] = d2[a + 1] * d1[b + 1];   /* d_xx d_y */
                else c[S5(a, b)] = d1[a + 1] * d2[b + 1];              /* d_x d_yy */
            }
        return 0;
    }
    default: return -1;
    }
}

int orc_derivative(int order, int which, const double *F, int nx, int ny, double *out) {
    double c[25];
    if (orc_stencil(order, which, c)) return -1;
    orc_params p;
    memset(&p, 0, sizeof p);
    p.nx = nx; p.ny = ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double s = 0.0;
            for (int dy = -2; dy <= 2; dy++)
                for (int dx = -2; dx <= 2; dx++)
                    if (c[S5(dx, dy)] != 0.0) s += c[S5(dx, dy)] * F[idx(&p, i + dx, j + dy)];
            out[(size_t)j * nx + i] = s;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Velocity fields (prescribed, divergence free, Sec. II.A).                  */
/* ------------------------------------------------------------------------ */

void orc_velocity(const orc_params *p, double x, double y, double t, double uv[2]) {
    switch (p->vel_kind) {
    case 0:
        uv[0] = p->vel[0]; uv[1] = p->vel[1];
        return;
    case 1: /* rigid rotation about (cx, cy) at angular speed omega (Sec. III.B) */
        uv[0] = -p->vel[2] * (y - p->vel[1]);
        uv[1] = p->vel[2] * (x - p->vel[0]);
        return;
    case 2: { /* single vortex on a periodic box of side L, reversed by cos(pi t / T) */
        double L = p->vel[0], U = p->vel[1], T = p->vel[2];
        double sx = sin(PI * x / L), sy = sin(PI * y / L), c = cos(PI * t / T);
        uv[0] = -U * sx * sx * sin(2.0 * PI * y / L) * c;
        uv[1] = U * sy * sy * sin(2.0 * PI * x / L) * c;
        return;
    }
    case 3: { /* cell-centre field: x, y are centres or face midpoints */
        int i0 = (int)floor(x - 0.5), j0 = (int)floor(y - 0.5);
        double fx = x - 0.5 - i0, fy = y - 0.5 - j0;   /* 0 or 1/2 on the grid points used */
        double u00 = p->u_field[idx(p, i0, j0)], v00 = p->v_field[idx(p, i0, j0)];
        double u10 = p->u_field[idx(p, i0 + 1, j0)], v10 = p->v_field[idx(p, i0 + 1, j0)];
        double u01 = p->u_field[idx(p, i0, j0 + 1)], v01 = p->v_field[idx(p, i0, j0 + 1)];
        double u11 = p->u_field[idx(p, i0 + 1, j0 + 1)], v11 = p->v_field[idx(p, i0 + 1, j0 + 1)];
        uv[0] = (1 - fx) * (1 - fy) * u00 + fx * (1 - fy) * u10 + (1 - fx) * fy * u01 + fx * fy * u11;
        uv[1] = (1 - fx) * (1 - fy) * v00 + fx * (1 - fy) * v10 + (1 - fx) * fy * v01 + fx * fy * v11;
        return;
    }
    case 5: { /* smoothed deformation (Sec. III.D): 4 x 4 cells of vortices on a box of side L,
               * u = -U sin(4 pi x/L) sin(4 pi y/L) cos(pi t/T), v = -U cos(4 pi x/L) cos(4 pi y/L) cos(pi t/T) */
        double L = p->vel[0], U = p->vel[1], T = p->vel[2], c = cos(PI * t / T);
        uv[0] = -U * sin(4.0 * PI * x / L) * sin(4.0 * PI * y / L) * c;
        uv[1] = -U * cos(4.0 * PI * x / L) * cos(4.0 * PI * y / L) * c;
        return;
    }
    case 4: { /* uniform flow reversed by the vortex's factor cos(pi t / T): test-only kind
               * whose exact displacement (ux, uy) T / pi sin(pi t / T) pins the time levels */
        double c = cos(PI * t / p->vel[2]);
        uv[0] = p->vel[0] * c; uv[1] = p->vel[1] * c;
        return;
    }
    default:
        uv[0] = uv[1] = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Cell quantities: theta, n, D, S, f^eq (Sec. II.A, Eqs. (2), (4), (14)).    */
/* ------------------------------------------------------------------------ */

void orc_cell_quantities(const orc_params *p, const double *phi, const double *phi_old,
                         double t, double t_old, double dtD, int use_D, double *V, double *g) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    const double tau = p->M / RT;
    double *gx = malloc(N * sizeof(double)), *gy = malloc(N * sizeof(double));
    /* Reading: the gradient of phi for n is the isotropic one of the order; DUGKS-T2S5,
     * whose reconstruction is not an isotropic stencil, takes the fourth-order one */
    const int gorder = p->order == 5 ? 4 : p->order;
    orc_derivative(gorder, 0, phi, nx, ny, gx);
    orc_derivative(gorder, 1, phi, nx, ny, gy);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)j * nx + i;
            double x = i + 0.5, y = j + 0.5, ph = phi[c];
            /* Eq. (2): n = grad phi / |grad phi|. Reading: n = 0 where |grad phi|^2 <= 1e-24. */
            double g2 = gx[c] * gx[c] + gy[c] * gy[c];
            double nxv = 0.0, nyv = 0.0;
            if (g2 > 1e-24) {
                double inv = 1.0 / sqrt(g2);
                nxv = gx[c] * inv; nyv = gy[c] * inv;
            }
            /* Eq. (4) */
            double theta = -4.0 * (ph - p->phiA) * (ph - p->phiB) / (p->W * (p->phiA - p->phiB));
            double u[2];
            orc_velocity(p, x, y, t, u);
            /* Reading: d(phi u)/dt by a backward difference between two time levels. */
            double Dx = 0.0, Dy = 0.0;
            if (use_D) {
                double uo[2];
                orc_velocity(p, x, y, t_old, uo);
                Dx = (ph * u[0] - phi_old[c] * uo[0]) / dtD;
                Dy = (ph * u[1] - phi_old[c] * uo[1]) / dtD;
            }
            /* Eq. (14b): S_k = w_k theta xi_k.n + w_k xi_k.D / RT = w_k xi_k.V */
            double Vx = theta * nxv + Dx / RT, Vy = theta * nyv + Dy / RT;
            V[c] = Vx;
            V[N + c] = Vy;
            for (int k = 0; k < Q; k++) {
                double feq = WQ[k] * ph * (1.0 + (EX[k] * u[0] + EY[k] * u[1]) / RT); /* Eq. (14a) */
                double S = WQ[k] * (EX[k] * Vx + EY[k] * Vy);
                g[k * N + c] = feq + tau * S;
            }
        }
    free(gx);
    free(gy);
}

void orc_phi(const orc_params *p, const double *X, double *phi) {
    const size_t N = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < N; c++) {
        double s = 0.0;
        for (int k = 0; k < Q; k++) s += X[k * N + c];   /* Eq. (30): unweighted sum */
        phi[c] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Face reconstruction at the back-traced point x_b - xi h (Eqs. (24)-(26)).   */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *F, *gx, *gy, *hxx, *hxy, *hyy, *txxx, *txxy, *txyy, *tyyy;
} deriv_set;

/* Taylor expansion of one direction's bar f^+ about cell c, evaluated at c + d:
 * value + d.grad + (1/2) d d : H (order >= 3) + (1/6) d d d : T (order 4).
 * Reading: Eq. (26) prints "d^2 : grad^2" without the 1/2 of a Taylor series. */
static double taylor(const orc_params *p, const deriv_set *D, size_t c, double dx, double dy) {
    double v = D->F[c] + dx * D->gx[c] + dy * D->gy[c];
    if (p->order >= 3)
        v += 0.5 * (dx * dx * D->hxx[c] + 2.0 * dx * dy * D->hxy[c] + dy * dy * D->hyy[c]);
    if (p->order >= 4)
        v += (dx * dx * dx * D->txxx[c] + 3.0 * dx * dx * dy * D->txxy[c] +
              3.0 * dx * dy * dy * D->txyy[c] + dy * dy * dy * D->tyyy[c]) / 6.0;
    return v;
}

/* Weight of node a (a = -2..2, unit spacing, centre 0) of the degree-4 Lagrange
 * interpolant at offset s from the centre node. */
static double lagrange5(int a, double s) {
    double w = 1.0;
    for (int b = -2; b <= 2; b++)
        if (b != a) w *= (s - b) / (double)(a - b);
    return w;
}

/* bar f^+ at q from the 5 x 5 cells centred at the cell (m, n): the tensor-product
 * degree-4 interpolant (error O(dx^5), not isotropic). */
static double interp5(const orc_params *p, const double *F, int m, int n, double qx, double qy) {
    const double sx = qx - (m + 0.5), sy = qy - (n + 0.5);
    double v = 0.0;
    for (int b = -2; b <= 2; b++) {
        double row = 0.0;
        for (int a = -2; a <= 2; a++) row += lagrange5(a, sx) * F[idx(p, m + a, n + b)];
        v += lagrange5(b, sy) * row;
    }
    return v;
}

/* DUGKS-T2S5 (Sec. III.A: fifth-order reconstruction, a stencil "not isotropic",
 * no stencil printed). Reading: bar f^+ at the back-traced point q = x_b - xi h
 * is the tensor-product degree-4 Lagrange interpolant on the 5 x 5 cells centred
 * at the cell nearest to q (upwind-biased); on a face (xi normal to it zero) the
 * two nearest cells tie and the two interpolants are averaged, as for Eq. (26);
 * along the face q stays in the face's row. */
static void reconstruct5(const orc_params *p, const double *fbp, double h, double *fbarE, double *fbarN) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    for (int k = 0; k < Q; k++) {
        const double *F = fbp + k * N;
        const int ex = EX[k], ey = EY[k];
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = (size_t)j * nx + i;
                double qx = i + 1.0 - ex * h, qy = j + 0.5 - ey * h;   /* east face */
                double vE = ex > 0 ? interp5(p, F, i, j, qx, qy)
                          : ex < 0 ? interp5(p, F, i + 1, j, qx, qy)
                                   : 0.5 * (interp5(p, F, i, j, qx, qy) + interp5(p, F, i + 1, j, qx, qy));
                qx = i + 0.5 - ex * h; qy = j + 1.0 - ey * h;          /* north face */
                double vN = ey > 0 ? interp5(p, F, i, j, qx, qy)
                          : ey < 0 ? interp5(p, F, i, j + 1, qx, qy)
                                   : 0.5 * (interp5(p, F, i, j, qx, qy) + interp5(p, F, i, j + 1, qx, qy));
                fbarE[k * N + c] = vE;
                fbarN[k * N + c] = vN;
            }
    }
}

void orc_reconstruct(const orc_params *p, const double *fbp, double h, double *fbarE, double *fbarN) {
    if (p->order == 5) {
        reconstruct5(p, fbp, h, fbarE, fbarN);
        return;
    }
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    double *buf = malloc(9 * N * sizeof(double));
    deriv_set D;
    D.gx = buf; D.gy = buf + N; D.hxx = buf + 2 * N; D.hxy = buf + 3 * N; D.hyy = buf + 4 * N;
    D.txxx = buf + 5 * N; D.txxy = buf + 6 * N; D.txyy = buf + 7 * N; D.tyyy = buf + 8 * N;
    double *planes[9] = {D.gx, D.gy, D.hxx, D.hxy, D.hyy, D.txxx, D.txxy, D.txyy, D.tyyy};
    int nd = p->order == 2 ? 2 : (p->order == 3 ? 5 : 9);
    for (int k = 0; k < Q; k++) {
        D.F = (double *)fbp + k * N;
        for (int w = 0; w < nd; w++) orc_derivative(p->order, w, D.F, nx, ny, planes[w]);
        const double ex = EX[k], ey = EY[k];
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t c = (size_t)j * nx + i;
                size_t cE = idx(p, i + 1, j), cN = idx(p, i, j + 1);
                double vE, vN;
                if (p->flux == 0) {
                    /* Upwind: expand about the cell centre nearest to q = x_b - xi h.
                     * East face x_b = (i+1, j+1/2): q_x = i + 1 - xi_x h lies in cell i
                     * when xi_x > 0 and in cell i+1 when xi_x < 0 (h <= 1/2); for
                     * xi_x = 0 it is on the face. Reading: that tie averages the two
                     * expansions. Along the face, q stays in row j. */
                    if (ex > 0) vE = taylor(p, &D, c, 0.5 - h, -ey * h);
                    else if (ex < 0) vE = taylor(p, &D, cE, h - 0.5, -ey * h);
                    else vE = 0.5 * (taylor(p, &D, c, 0.5, -ey * h) + taylor(p, &D, cE, -0.5, -ey * h));
                    if (ey > 0) vN = taylor(p, &D, c, -ex * h, 0.5 - h);
                    else if (ey < 0) vN = taylor(p, &D, cN, -ex * h, h - 0.5);
                    else vN = 0.5 * (taylor(p, &D, c, -ex * h, 0.5) + taylor(p, &D, cN, -ex * h, -0.5));
                } else {
                    /* Central, Eq. (25): face value = mean of the two cells; face
                     * gradient: normal part (F_R - F_L) / dx, tangential part the mean
                     * of the two cells' tangential derivatives (Reading). */
                    double FbE = 0.5 * (D.F[c] + D.F[cE]);
                    double gxE = D.F[cE] - D.F[c], gyE = 0.5 * (D.gy[c] + D.gy[cE]);
                    vE = FbE - h * (ex * gxE + ey * gyE);
                    double FbN = 0.5 * (D.F[c] + D.F[cN]);
                    double gxN = 0.5 * (D.gx[c] + D.gx[cN]), gyN = D.F[cN] - D.F[c];
                    vN = FbN - h * (ex * gxN + ey * gyN);
                }
                /* Eq. (24): bar f(x_b, t + h) = bar f^+(x_b - xi h, t) */
                fbarE[k * N + c] = vE;
                fbarN[k * N + c] = vN;
            }
    }
    free(buf);
}

/* Eqs. (27)-(28) at the faces; the face source is the mean of the two
 * neighbouring cells' source at the base time (as stated in Sec. III.A). */
void orc_face_f(const orc_params *p, const double *fbarE, const double *fbarN, const double *V,
                double h, double t_face, double *fE, double *fN) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    const double tau = p->M / RT;
    const double den = 2.0 * tau + h;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)j * nx + i;
            for (int face = 0; face < 2; face++) {
                const double *fb = face == 0 ? fbarE : fbarN;
                double *out = face == 0 ? fE : fN;
                size_t cn = face == 0 ? idx(p, i + 1, j) : idx(p, i, j + 1);
                double xb = face == 0 ? i + 1.0 : i + 0.5, yb = face == 0 ? j + 0.5 : j + 1.0;
                /* Eq. (28). Reading: the sum is unweighted (the weights are
                 * already inside f^eq; only the unweighted sum is conserved). */
                double phib = 0.0;
                for (int k = 0; k < Q; k++) phib += fb[k * N + c];
                double u[2];
                orc_velocity(p, xb, yb, t_face, u);
                double Vx = 0.5 * (V[c] + V[cn]), Vy = 0.5 * (V[N + c] + V[N + cn]);
                for (int k = 0; k < Q; k++) {
                    double feq = WQ[k] * phib * (1.0 + (EX[k] * u[0] + EY[k] * u[1]) / RT);
                    double S = WQ[k] * (EX[k] * Vx + EY[k] * Vy);
                    out[k * N + c] = (2.0 * tau * fb[k * N + c] + h * feq + tau * h * S) / den;
                }
            }
        }
}

void orc_flux(const orc_params *p, const double *fE, const double *fN, double *L) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)j * nx + i, cW = idx(p, i - 1, j), cS = idx(p, i, j - 1);
            for (int k = 0; k < Q; k++)
                /* Eq. (21) on a unit cell with the inward normal of the paper */
                L[k * N + c] = -(EX[k] * (fE[k * N + c] - fE[k * N + cW]) +
                                 EY[k] * (fN[k * N + c] - fN[k * N + cS]));
        }
}

/* ------------------------------------------------------------------------ */
/* Time steps.                                                                */
/* ------------------------------------------------------------------------ */

int orc_check(const orc_params *p) {
    if (p->nx < 8 || p->ny < 8) return -1;
    if (!(p->W > 0) || !(p->M > 0) || !(p->cfl > 0) || p->cfl > 1.0) return -1;
    if (p->order < 2 || p->order > 5 || (p->flux != 0 && p->flux != 1)) return -1;
    /* order 5: DUGKS-T2S5 (Sec. III.A), the two-stage scheme with upwind faces */
    if (p->order == 5 && (p->flux != 0 || p->stages != 2)) return -1;
    if (p->stages < 1 || p->stages > 3) return -1;   /* 1: streaming-collision DVM (Sec. II.B.1) */
    if (p->stages == 1 && p->order > 4) return -1;
    if (p->phiA == p->phiB) return -1;
    if (p->vel_kind < 0 || p->vel_kind > 5) return -1;
    if (p->vel_kind == 5 && (p->vel[0] <= 0 || p->vel[2] <= 0)) return -1;
    if (p->vel_kind == 3 && (!p->u_field || !p->v_field)) return -1;
    if (p->vel_kind == 2 && (p->vel[0] <= 0 || p->vel[2] <= 0)) return -1;
    if (p->vel_kind == 4 && !(p->vel[2] > 0)) return -1;
    /* Three-stage DUGKS needs dt < 12 tau (Sec. III.A). */
    if (p->stages == 3 && !(p->cfl < 12.0 * p->M / RT)) return -1;
    return 0;
}

/* flux part of one stage: faces from bar f^+ over time h, velocity at t_face */
static void stage_flux(const orc_params *p, const double *fbp, const double *V, double h,
                       double t_face, double *L, double *w1, double *w2, double *w3, double *w4) {
    orc_reconstruct(p, fbp, h, w1, w2);
    orc_face_f(p, w1, w2, V, h, t_face, w3, w4);
    orc_flux(p, w3, w4, L);
}

/* Cell-relation coefficients of one step.
 * Two-stage: c[0] = h = dt/2, bar f^+ = c[1] tilde f + c[2] g.
 * Three-stage: c[0] = h1 = dt/6, A = c[1] hat f + c[2] g (Eq. (31));
 *              c[3] = h2 = 5 dt/12, B = c[4] tilde f' + c[5] g' (Eq. (34));
 *              c[6]: Omega + S at t' = c[6] (tilde f' - g') (Eq. (29)). */
int orc_coefficients(const orc_params *p, double c[8]) {
    const double dt = p->cfl, tau = p->M / RT;
    memset(c, 0, 8 * sizeof(double));
    if (p->stages == 2) {
        /* Original DUGKS: tilde f = f - (dt/2)(Omega + S) and
         * bar f^+ = f + (h/2)(Omega + S) with Omega + S = -(f - g)/tau give,
         * eliminating f (as Eqs. (31)-(34) do for three stages),
         * bar f^+ = (2 tau - h)/(2 tau + dt) tilde f + (dt + h)/(2 tau + dt) g. */
        const double h = 0.5 * dt;
        c[0] = h;
        c[1] = (2.0 * tau - h) / (2.0 * tau + dt);
        c[2] = (dt + h) / (2.0 * tau + dt);
        return 0;
    }
    c[0] = dt / 6.0;
    c[1] = (12.0 * tau - dt) / (12.0 * tau + 3.0 * dt);
    c[2] = 4.0 * dt / (12.0 * tau + 3.0 * dt);
    c[3] = 5.0 * dt / 12.0;
    c[4] = (24.0 * tau - 5.0 * dt) / (24.0 * tau + 4.0 * dt);
    c[5] = 9.0 * dt / (24.0 * tau + 4.0 * dt);
    /* Reading: Eq. (29) prints -6 dt / (6 tau + dt); with tilde f = f - (dt/6)(Omega+S)
     * and Omega + S = -(f - g)/tau the factor is -6 / (6 tau + dt). */
    c[6] = -6.0 / (6.0 * tau + dt);
    return 0;
}

static int step_once(const orc_params *p, double *X, double *phi_prev, long n) {
    const size_t N = (size_t)p->nx * p->ny;
    const double dt = p->cfl, t = n * dt;
    const int useD = p->dtphiu && n > 0;   /* Reading: D = 0 at the first step */
    double *phi = malloc(N * sizeof(double)), *V = malloc(2 * N * sizeof(double));
    double *g = malloc(9 * N * sizeof(double)), *fbp = malloc(9 * N * sizeof(double));
    double *L = malloc(9 * N * sizeof(double));
    double *w1 = malloc(9 * N * sizeof(double)), *w2 = malloc(9 * N * sizeof(double));
    double *w3 = malloc(9 * N * sizeof(double)), *w4 = malloc(9 * N * sizeof(double));

    orc_phi(p, X, phi);
    orc_cell_quantities(p, phi, phi_prev, t, t - dt, dt, useD, V, g);

    if (p->stages == 2) {
        /* Original DUGKS (state tilde f); tilde f^+ = (4/3) bar f^+ - (1/3) tilde f
         * follows from the same definitions. */
        double cf[8];
        orc_coefficients(p, cf);
        const double h = cf[0], a = cf[1], b = cf[2];
        for (size_t q = 0; q < 9 * N; q++) fbp[q] = a * X[q] + b * g[q];
        stage_flux(p, fbp, V, h, t + h, L, w1, w2, w3, w4);
        for (size_t q = 0; q < 9 * N; q++)
            X[q] = (4.0 / 3.0) * fbp[q] - (1.0 / 3.0) * X[q] + dt * L[q];
    } else {
        /* Three-stage third-order DUGKS, steps (i)-(iv) of Sec. II.B.2. State hat f. */
        double *A = fbp, *ft1 = malloc(9 * N * sizeof(double)), *Lss = malloc(9 * N * sizeof(double));
        double *phi1 = malloc(N * sizeof(double));
        /* (i) Eq. (31): bar f^{+, dt/6}(t_n); flux at t* = t_n + dt/6 */
        double cf[8];
        orc_coefficients(p, cf);
        const double h1 = cf[0], a1 = cf[1], b1 = cf[2];
        for (size_t q = 0; q < 9 * N; q++) A[q] = a1 * X[q] + b1 * g[q];
        stage_flux(p, A, V, h1, t + h1, L, w1, w2, w3, w4);
        /* (ii) Eq. (33) tilde f^+ = (5/4) A - (1/4) hat f; Eq. (15): tilde f(t') */
        for (size_t q = 0; q < 9 * N; q++)
            ft1[q] = (1.25 * A[q] - 0.25 * X[q]) + (dt / 3.0) * L[q];
        /* cell quantities at t' = t_n + dt/3 (Eq. (30b)); D between t_n and t' */
        orc_phi(p, ft1, phi1);
        double *V1 = malloc(2 * N * sizeof(double)), *g1 = malloc(9 * N * sizeof(double));
        orc_cell_quantities(p, phi1, phi, t + dt / 3.0, t, dt / 3.0, p->dtphiu, V1, g1);
        /* (iii) Eq. (34): bar f^{+, 5dt/12}(t'); flux at t** = t_n + 3 dt / 4 */
        const double h2 = cf[3], a2 = cf[4], b2 = cf[5];
        double *B = malloc(9 * N * sizeof(double));
        for (size_t q = 0; q < 9 * N; q++) B[q] = a2 * ft1[q] + b2 * g1[q];
        stage_flux(p, B, V1, h2, t + 0.75 * dt, Lss, w1, w2, w3, w4);
        /* (iv) Eq. (32) f(t_n) = (3/4) A + (1/4) hat f; Eq. (29) Omega + S at t';
         * Eq. (16) for hat f^{n+1}. */
        const double cos_ = cf[6];
        for (size_t q = 0; q < 9 * N; q++) {
            double fn = 0.75 * A[q] + 0.25 * X[q];
            double os = cos_ * (ft1[q] - g1[q]);
            X[q] = fn + 0.75 * dt * os + (dt / 7.0) * (3.0 * L[q] + 4.0 * Lss[q]);
        }
        free(ft1); free(Lss); free(phi1); free(V1); free(g1); free(B);
    }
    memcpy(phi_prev, phi, N * sizeof(double));
    free(phi); free(V); free(g); free(fbp); free(L); free(w1); free(w2); free(w3); free(w4);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Streaming-collision DVM (Sec. II.B.1, Eqs. (8)-(14)). State: tilde f^+ of   */
/* Eq. (9) at the cell centres; phi_prev = phi at t.                          */
/* ------------------------------------------------------------------------ */

/* Eq. (11b) and Eqs. (13)-(14): phi(t + dt) from the streamed tilde f', the cell
 * quantities at t + dt (d(phi u)/dt by the backward difference from t, as for
 * DUGKS), and the collision
 * tilde f^+ = tilde f' + 2 dt/(2 tau + dt) (f^eq + tau S - tilde f'). */
static void dvm_collide(const orc_params *p, double *X, const double *Fs, double *phi_prev, double t, double dt) {
    const size_t N = (size_t)p->nx * p->ny;
    const double tau = p->M / RT;
    double *phi = malloc(N * sizeof(double)), *V = malloc(2 * N * sizeof(double));
    double *g = malloc(9 * N * sizeof(double));
    orc_phi(p, Fs, phi);   /* Eq. (13). Reading: the unweighted sum, as for Eq. (28) */
    orc_cell_quantities(p, phi, phi_prev, t + dt, t, dt, p->dtphiu, V, g);
    const double beta = 2.0 * dt / (2.0 * tau + dt);
    for (size_t q = 0; q < 9 * N; q++) X[q] = Fs[q] + beta * (g[q] - Fs[q]);
    memcpy(phi_prev, phi, N * sizeof(double));
    free(phi); free(V); free(g);
}

/* One DVM step: Eq. (11a) streaming, tilde f'_k(x_c) = tilde f^+_k(x_c - xi_k dt),
 * the value at the back-traced point taken from the Taylor expansion of Eq. (12)
 * about the centre x_n of the cell that contains it. Reading: Eq. (12) prints
 * "(.)^2 : grad^2" without the 1/2 of a Taylor series (as Eq. (26)); the cell
 * holding x_c - xi_k dt is the neighbour x_c - xi_k for dt >= 1/2 (the paper's
 * "starting cell just adjacent to the targeting cell"; at dt = 1/2 the point is on
 * the cell edge and the neighbour is taken) and x_c itself below. Then Eq. (11b). */
static void dvm_step(const orc_params *p, double *X, double *phi_prev, long n) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    const double dt = p->cfl, t = n * dt;
    const int s = dt >= 0.5 ? 1 : 0;
    double *Fs = malloc(9 * N * sizeof(double)), *buf = malloc(9 * N * sizeof(double));
    deriv_set D;
    D.gx = buf; D.gy = buf + N; D.hxx = buf + 2 * N; D.hxy = buf + 3 * N; D.hyy = buf + 4 * N;
    D.txxx = buf + 5 * N; D.txxy = buf + 6 * N; D.txyy = buf + 7 * N; D.tyyy = buf + 8 * N;
    double *planes[9] = {D.gx, D.gy, D.hxx, D.hxy, D.hyy, D.txxx, D.txxy, D.txyy, D.tyyy};
    const int nd = p->order == 2 ? 2 : (p->order == 3 ? 5 : 9);
    for (int k = 0; k < Q; k++) {
        D.F = X + k * N;
        for (int w = 0; w < nd; w++) orc_derivative(p->order, w, D.F, nx, ny, planes[w]);
        /* displacement from x_n = x_c - s xi_k to x_c - xi_k dt */
        const double dx = EX[k] * (s - dt), dy = EY[k] * (s - dt);
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                Fs[k * N + (size_t)j * nx + i] = taylor(p, &D, idx(p, i - s * EX[k], j - s * EY[k]), dx, dy);
    }
    dvm_collide(p, X, Fs, phi_prev, t, dt);
    free(Fs);
    free(buf);
}

/* The lattice Boltzmann step (dt = 1): plain streaming from the neighbour
 * x_c - xi_k, then the same collision. Written independently of the Taylor
 * streaming above so that "the DVM at C = 1 is the LBM" (Sec. III.A) is a check
 * between two codes. */
static void lbm_step(const orc_params *p, double *X, double *phi_prev, long n) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    double *Fs = malloc(9 * N * sizeof(double));
    for (int k = 0; k < Q; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                Fs[k * N + (size_t)j * nx + i] = X[k * N + idx(p, i - EX[k], j - EY[k])];
    dvm_collide(p, X, Fs, phi_prev, (double)n, 1.0);
    free(Fs);
}

int orc_run_lbm(const orc_params *p, double *state, double *phi_prev, long step0, long nsteps) {
    if (orc_check(p) || p->stages != 1 || p->cfl != 1.0) return -1;
    for (long s = 0; s < nsteps; s++) lbm_step(p, state, phi_prev, step0 + s);
    return 0;
}

int orc_init(const orc_params *p, const double *phi0, double *state, double *phi_prev) {
    if (orc_check(p)) return -1;
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    const double dt = p->cfl;
    double *V = malloc(2 * N * sizeof(double)), *g = malloc(9 * N * sizeof(double));
    /* Reading: start from f = f^eq (Omega = 0) with D = 0. */
    orc_cell_quantities(p, phi0, phi0, 0.0, 0.0, dt, 0, V, g);
    /* tilde f or hat f, Eq. (19); the DVM's tilde f^+ = f + (dt/2)(Omega + S), Eq. (9) */
    const double frac = p->stages == 2 ? 0.5 : p->stages == 3 ? 0.25 : -0.5;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = (size_t)j * nx + i;
            double u[2];
            orc_velocity(p, i + 0.5, j + 0.5, 0.0, u);
            for (int k = 0; k < Q; k++) {
                double feq = WQ[k] * phi0[c] * (1.0 + (EX[k] * u[0] + EY[k] * u[1]) / RT);
                double S = WQ[k] * (EX[k] * V[c] + EY[k] * V[N + c]);
                state[k * N + c] = feq - frac * dt * S;
            }
        }
    memcpy(phi_prev, phi0, N * sizeof(double));
    free(V);
    free(g);
    return 0;
}

int orc_run(const orc_params *p, double *state, double *phi_prev, long step0, long nsteps) {
    if (orc_check(p)) return -1;
    for (long s = 0; s < nsteps; s++) {
        if (p->stages == 1) dvm_step(p, state, phi_prev, step0 + s);
        else step_once(p, state, phi_prev, step0 + s);
    }
    return 0;
}

double orc_mass(const orc_params *p, const double *state) {
    const size_t N = (size_t)p->nx * p->ny;
    double m = 0.0;
    for (size_t c = 0; c < N; c++)
        for (int k = 0; k < Q; k++) m += state[k * N + c];
    return m;
}
