// dugks_dvm.cuh -- the streaming-collision discrete velocity method (DVM) of
// Sec. II.B.1 on the GPU, and at C = 1 the lattice Boltzmann method.
//
// State: tilde f^+_k = f_k + (dt/2)(Omega_k + S_k) at the cell centres (Eq. (9)),
// 9 planes in the ghost-bordered layout, and phi of the state as a plane. One
// fused kernel per step, one CTA per 32 x 8 tile:
//   pass 1  streaming, Eq. (11a): tilde f'_k(x_c) = tilde f^+_k(x_c - xi_k dt), the
//           value at the back-traced point from the Taylor expansion of Eq. (12)
//           (value + d.grad + d d : H / 2 (+ d d d : T / 6 at order 4), the
//           isotropic stencils of the DUGKS path) about the centre x_n = x_c - s xi_k
//           of the cell that holds it (s = 1 for dt >= 1/2, else 0), so
//           d = xi_k (s - dt); phi(t + dt) = sum_k tilde f'_k (Eq. (13)) on the tile
//           plus the ring the gradient of phi needs. At dt = 1 the back-traced
//           point is the neighbour's centre: plain streaming, the LBM.
//   pass 2  cell quantities at t + dt from the new phi (Eqs. (2), (4), (14): n,
//           theta, d(phi u)/dt by the backward difference from t, f^eq, S) and the
//           collision of Eq. (11b): tilde f^+ = tilde f' + 2 dt/(2 tau + dt)
//           (f^eq + tau S - tilde f') for the moving directions, the rest direction
//           closing the moment phi(t + dt) (equal to Eq. (11b) up to rounding); the
//           new state, phi and an FP64 mass partial per tile are written.
// The state tile (halo 2R + 1: the phi ring, the shift, the Taylor stencil; R + 1
// for the LBM) is read with plain coalesced loads; the ghost border makes it one
// rectangle.
#pragma once

#include "dugks_kernels.cuh"

namespace dugks {

// Per-run constants of the DVM step.
template <typename T>
struct DvmExtra {
    T d;      // displacement of the back-traced point from x_n per unit lattice velocity: s - dt
    T beta;   // collision factor 2 dt / (2 tau + dt)
    int s;    // shift of the expansion cell: x_n = x_c - s xi_k
};

template <typename T, int ORDER, bool LBM>
struct DvmTile {
    static constexpr int TX = 32, TY = 8, NT = TX * TY;
    static constexpr int R = ORDER == 4 ? 2 : 1;          // stencil radius
    static constexpr int HS = LBM ? R + 1 : 2 * R + 1;    // state halo
    static constexpr int SW = TX + 2 * HS, SH = TY + 2 * HS;
    static constexpr int PW = TX + 2 * R, PH = TY + 2 * R;   // phi(t + dt) region
    static constexpr int RING = PW * PH - TX * TY;
    static constexpr size_t oP = sizeof(T) * 9 * SW * SH;
    static constexpr size_t oRed = (oP + sizeof(T) * PW * PH + 15) / 16 * 16;
    static constexpr size_t smem_bytes = oRed + sizeof(double) * 32;
    static_assert(HS <= GHOST, "the halo fits the ghost border");
    static_assert(RING <= NT, "one ring cell per thread");
};

template <typename T, int ORDER, bool LBM>
__global__ void __launch_bounds__(256) dvm_step_kernel(const StepParams<T> p, const DvmExtra<T> dv) {
    using DT = DvmTile<T, ORDER, LBM>;
    constexpr int TX = DT::TX, TY = DT::TY, HS = DT::HS, SW = DT::SW, SH = DT::SH, R = DT::R;
    constexpr int PW = DT::PW, PH = DT::PH;
    extern __shared__ __align__(16) unsigned char smem[];
    T *sF = reinterpret_cast<T *>(smem);
    T *sP = reinterpret_cast<T *>(smem + DT::oP);
    double *sred = reinterpret_cast<double *>(smem + DT::oRed);
    const int tid = threadIdx.x, x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = p.nx, ny = p.ny;

    // the state tile with its halo (cells beyond the ghost border, needed by no
    // cell of the grid, are clamped to it)
    const T *X = static_cast<const T *>(p.X);
    for (int i = tid; i < 9 * SW * SH; i += DT::NT) {
        const int k = i / (SW * SH), r = i - k * (SW * SH), yy = r / SW, xx = r - yy * SW;
        const int gx = min(x0 + xx - HS, nx + GHOST - 1), gy = min(y0 + yy - HS, ny + GHOST - 1);
        sF[i] = X[k * p.plane + gidx(p, gx, gy)];
    }
    __syncthreads();

    // pass 1: streaming of cell (x, y) of the tile frame (Eqs. (11a), (12)), phi(t + dt)
    auto stream = [&](int x, int y, T (&fs)[9]) -> T {
        T phi = T(0);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const T *F = sF + k * SW * SH;
            if constexpr (LBM) {
                fs[k] = F[(y - ey(k) + HS) * SW + (x - ex(k) + HS)];
            } else {
                const int xn = x - dv.s * ex(k), yn = y - dv.s * ey(k);
                fs[k] = taylor<T, ORDER>(F + (yn + HS) * SW + (xn + HS), SW, dv.d * T(ex(k)), dv.d * T(ey(k)));
            }
            phi += fs[k];   // Eq. (13), the unweighted sum
        }
        return phi;
    };
    const int tx = tid & 31, ty = tid >> 5;
    T fs[9];
    sP[(ty + R) * PW + (tx + R)] = stream(tx, ty, fs);
    if (tid < DT::RING) {   // the ring of the phi region: rows above and below, then the side columns
        int rx, ry;
        if (tid < 2 * R * PW) {
            const int band = tid / PW;
            ry = band < R ? band - R : TY + band - R;
            rx = tid - band * PW - R;
        } else {
            const int e = tid - 2 * R * PW, col = e / TY;
            rx = col < R ? col - R : TX + col - R;
            ry = e - col * TY;
        }
        T tmp[9];
        sP[(ry + R) * PW + (rx + R)] = stream(rx, ry, tmp);
    }
    __syncthreads();

    // pass 2: cell quantities at t + dt and the collision (Eqs. (2), (4), (14), (11b))
    const int gx = x0 + tx, gy = y0 + ty;
    double msum = 0.0;
    if (gx < nx && gy < ny) {
        const T *P = sP + (ty + R) * PW + (tx + R);
        const T ph = P[0];
        T gxp, gyp;
        grad_p<T, ORDER>(P, PW, gxp, gyp);
        const T g2 = gxp * gxp + gyp * gyp;
        T nxv = T(0), nyv = T(0);
        if (g2 > T(1e-24)) {
            const T inv = T(1) / sqrt(g2);
            nxv = gxp * inv;
            nyv = gyp * inv;
        }
        const T theta = p.theta_c * (ph - p.phiA) * (ph - p.phiB);
        T u, v;
        vel_cell(p, gx, gy, p.t, u, v);   // at t + dt
        T Dx = T(0), Dy = T(0);
        const size_t g = gidx(p, gx, gy);
        if (p.useD) {   // d(phi u)/dt between t and t + dt
            T uo, vo;
            vel_cell(p, gx, gy, p.t_old, uo, vo);
            const T po = p.phi_old[g];
            Dx = (ph * u - po * uo) * p.inv_dtD;
            Dy = (ph * v - po * vo) * p.inv_dtD;
        }
        const T Vx = theta * nxv + T(3) * Dx, Vy = theta * nyv + T(3) * Dy;
        T *O = static_cast<T *>(p.out1);
        // the rest component closes the sum (sum_k f^eq_k = phi, sum_k S_k = 0): the state
        // keeps the moment phi(t + dt) up to one rounding, as the DUGKS kernels do
        T rest = ph;
#pragma unroll
        for (int k = 1; k < 9; k++) {
            const T xu = T(ex(k)) * u + T(ey(k)) * v, xv = T(ex(k)) * Vx + T(ey(k)) * Vy;
            const T gk = wq<T>(k) * (ph * (T(1) + T(3) * xu) + p.tau * xv);   // f^eq + tau S
            const T o = fs[k] + dv.beta * (gk - fs[k]);
            rest -= o;
            put_cell(p, O + k * p.plane, gx, gy, o);
        }
        put_cell(p, O, gx, gy, rest);
        p.phi_out[g] = ph;
        msum = (double)ph;
    }
    const double s = block_sum(msum, sred);
    if (tid == 0 && p.mass_partial) p.mass_partial[blockIdx.y * p.tiles_x + blockIdx.x] = s;
}

}  // namespace dugks
