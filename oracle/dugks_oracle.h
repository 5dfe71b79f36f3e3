/*
 * dugks_oracle.h -- plain FP64 CPU oracle of the DUGKS time step for the
 * conservative Allen-Cahn equation (Yang, Zhong & Zhuo, "Performance evaluation
 * of high-order reconstruction for discrete unified gas-kinetic scheme in
 * tracking fluid interfaces").
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. It shares no code, header, table
 * or constant with the CUDA library; the product path never calls it.
 *
 * Grid: nx * ny cells of unit size, periodic in both directions, cell (i, j) has
 * its centre at (i + 1/2, j + 1/2); planes are stored row-major, x fastest.
 * A "9-plane" array holds direction k at offset k * nx * ny.
 */
#ifndef DUGKS_ORACLE_H
#define DUGKS_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;
    double W;        /* interface width, Sec. II.A */
    double M;        /* mobility; relaxation time tau = M / RT = 3 M */
    double cfl;      /* CFL number C; dt = C dx / sqrt(3 RT) = C, Eq. (39) */
    int order;       /* 2, 3 or 4; 5 = DUGKS-T2S5 (fifth-order upwind reconstruction,
                        two-stage, upwind only) */
    int flux;        /* 0 = upwind Eq. (26), 1 = central Eq. (25) */
    int stages;      /* 2 = original DUGKS, 3 = three-stage third-order DUGKS,
                        1 = streaming-collision DVM (Sec. II.B.1; flux unused) */
    int dtphiu;      /* 1 = keep the d(phi u)/dt part of the source Eq. (14b) */
    double phiA, phiB;
    int vel_kind;    /* 0 uniform, 1 rigid rotation, 2 single vortex, 3 cell field,
                        4 reversing uniform (test-only: pins the time levels),
                        5 smoothed deformation (Sec. III.D) */
    double vel[4];   /* uniform (ux, uy); rotation (cx, cy, omega); vortex (L, U, T);
                        reversing uniform (ux, uy, T): (ux, uy) cos(pi t / T);
                        deformation (L, U, T) */
    const double *u_field, *v_field;   /* vel_kind 3: cell-centre components */
} orc_params;

/* 5x5 coefficient table of a derivative stencil, index (dy + 2) * 5 + (dx + 2).
 * which: 0 d/dx, 1 d/dy, 2 d2/dx2, 3 d2/dxdy, 4 d2/dy2,
 *        5 d3/dx3, 6 d3/dx2dy, 7 d3/dxdy2, 8 d3/dy3.
 * Returns 0, or -1 for an unsupported (order, which). */
int orc_stencil(int order, int which, double coef[25]);

/* out = stencil(order, which) applied to the periodic plane F. */
int orc_derivative(int order, int which, const double *F, int nx, int ny, double *out);

void orc_velocity(const orc_params *p, double x, double y, double t, double uv[2]);

/* Cell quantities at one time level from the order parameter phi:
 * V = theta n + D / RT (so that S_k = w_k xi_k . V), g_k = f^eq_k + tau S_k.
 * D = (phi u(t) - phi_old u(t_old)) / dtD when use_D, else 0. */
void orc_cell_quantities(const orc_params *p, const double *phi, const double *phi_old,
                         double t, double t_old, double dtD, int use_D,
                         double *V /* 2 planes */, double *g /* 9 planes */);

/* bar f at the east (x = i+1) and north (y = j+1) face midpoints of every cell,
 * from the cell values of bar f^+ (Eqs. (24)-(26)), reconstruction over time h. */
void orc_reconstruct(const orc_params *p, const double *fbp, double h,
                     double *fbarE, double *fbarN);

/* Original distribution at the faces, Eqs. (27)-(28); velocity at t_face. */
void orc_face_f(const orc_params *p, const double *fbarE, const double *fbarN,
                const double *V, double h, double t_face, double *fE, double *fN);

/* Meso-flux Eq. (21) of every cell, L_k = -[xi_x (f_E - f_W) + xi_y (f_N - f_S)]. */
void orc_flux(const orc_params *p, const double *fE, const double *fN, double *L);

/* phi = sum_k X_k. */
void orc_phi(const orc_params *p, const double *X, double *phi);

/* Initial state from phi0: f = f^eq, state = f^eq - (dt/2) S (two-stage),
 * f^eq - (dt/4) S (three-stage) or f^eq + (dt/2) S (DVM); phi_prev = phi0.
 * Returns 0 or -1 (bad params). */
int orc_init(const orc_params *p, const double *phi0, double *state, double *phi_prev);

/* Advance nsteps full time steps starting at step index step0. Returns 0 or -1. */
int orc_run(const orc_params *p, double *state, double *phi_prev, long step0, long nsteps);

/* The lattice Boltzmann method (stages = 1, cfl = 1): plain streaming from the
 * neighbour cell, then the DVM's collision. Returns 0 or -1. */
int orc_run_lbm(const orc_params *p, double *state, double *phi_prev, long step0, long nsteps);

/* Sum of phi over all cells. */
double orc_mass(const orc_params *p, const double *state);

/* Cell-relation coefficients of one step (see the definition for the layout). */
int orc_coefficients(const orc_params *p, double c[8]);

/* Validate parameters the way the paper restricts them (dt < 12 tau for three-stage). */
int orc_check(const orc_params *p);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
