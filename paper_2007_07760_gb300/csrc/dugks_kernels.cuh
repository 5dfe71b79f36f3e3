// dugks_kernels.cuh -- device code of the DUGKS time step (sm_103a).
//
// Method: Yang, Zhong & Zhuo, "Performance evaluation of high-order
// reconstruction for discrete unified gas-kinetic scheme in tracking fluid
// interfaces" (equation numbers are the paper's). Unit cells, D2Q9 with
// xi_k = e_k (RT = 1/3), tau = 3 M, periodic boundaries.
//
// One CTA owns a TX x TY tile of cells. A step (or one stage of the
// three-stage scheme) is a single fused kernel:
//   S0  stage the state X (9 SoA planes) of the tile plus a halo of H cells
//       into shared memory; phi = sum_k X_k                 (Eq. (30))
//   S1  on the tile plus 1 + R cells: grad phi (isotropic, order p), n, theta,
//       d(phi u)/dt, source vector V, g_k = f^eq_k + tau S_k and
//       bar f^+_k = a X_k + b g_k                           (Eqs. (2), (4), (14))
//   S2  every east / north face of the tile plus one ring: bar f_k at the
//       back-traced point x_b - xi_k h (upwind Taylor expansion from the
//       nearest cell, or central), phi_b = sum_k bar f_k, f^eq_b, S_b and the
//       original f_b                                        (Eqs. (24)-(28))
//   S3  every cell of the tile: meso-flux L_k (Eq. (21)) and the output
//       combination out = alpha X + beta g + gamma L (+ accumulator), plus the
//       cell's phi and an FP64 per-tile mass partial.
// R is the stencil radius (1 for p <= 3, 2 for p = 4) and H = 1 + 2R.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dugks {

// ---- D2Q9 lattice (Sec. II.B.2) ---------------------------------------------
__host__ __device__ __forceinline__ constexpr int ex(int k) {
    return k == 0 ? 0 : (k == 1 || k == 2 || k == 8) ? 1 : (k == 3 || k == 7) ? 0 : -1;
}
__host__ __device__ __forceinline__ constexpr int ey(int k) {
    return k == 0 ? 0 : (k == 2 || k == 3 || k == 4) ? 1 : (k == 1 || k == 5) ? 0 : -1;
}
template <typename T>
__host__ __device__ __forceinline__ constexpr T wq(int k) {
    return k == 0 ? T(4) / T(9) : (k & 1) ? T(1) / T(9) : T(1) / T(36);
}

enum Kind { KIND_T2 = 0, KIND_T3A = 1, KIND_T3B = 2 };
enum Vel { VEL_UNIFORM = 0, VEL_ROTATION = 1, VEL_VORTEX = 2, VEL_FIELD = 3, VEL_DEFORM = 4 };

// Storage of the distribution and of phi:
//  * Store<double, double>: full FP64 values; phi of a state is sum_k X_k
//  * Store<float, float>: full FP32 values plus phi as an FP32 plane of its own,
//    updated by phi + sum of the face fluxes with unbiased stochastic rounding;
//    sum_k X_k equals that phi up to rounding
//  * Store<float, __half>: half-precision scaled deviations
//    q_k = (f_k - w_k phi) * s / w_k, phi likewise its own plane (two-stage only)
// phi_plane: phi is read from and written to its planes rather than summed;
// t2 / t3: the schemes that storage serves.
template <typename T, typename ST>
struct Store;
template <>
struct Store<double, double> {
    static constexpr bool deviation = false, phi_plane = false, t2 = true, t3 = true;
};
template <>
struct Store<float, float> {
    static constexpr bool deviation = false, phi_plane = true, t2 = true, t3 = true;
};
template <>
struct Store<float, __half> {
    static constexpr bool deviation = true, phi_plane = true, t2 = true, t3 = false;
};

// Storage layout of every plane: (ny + 2 GHOST) rows of `pitch` elements; cell
// (x, y), 0 <= x < nx, 0 <= y < ny, sits at row y + GHOST, column x + GHOST.
// The GHOST-wide border holds periodic copies, written by whichever kernel
// writes the cell, so a tile plus its halo is always one rectangular box.
constexpr int GHOST = 5;

template <typename T>
struct StepParams {
    int nx, ny, pitch;          // pitch: elements between rows
    size_t plane;               // elements between planes = (ny + 2 GHOST) * pitch
    int *status;                // sticky device flags (bit 0 non-finite, bit 1 wait timeout)
    int tiles_x;                // CTAs along x (mass partial index = by * tiles_x + bx)
    int tile_w, tile_h;         // cells per CTA tile (mass partial kernel)
    const void *X;              // 9 planes in (storage type)
    const void *acc;            // KIND_T3B: accumulator planes (type T)
    const T *phi_cur;           // phi plane: phi of X (authoritative)
    const T *phi_old;           // phi at the older time level of d(phi u)/dt
    T *phi_out;                 // phi plane: phi of out1; otherwise (T2/T3A) phi of X
    T *phi_out2;                // phi plane, T3A: phi of out2 (the accumulator)
    const T *phi_acc;           // phi plane, T3B: phi of the accumulator
    void *out1;                 // 9 planes (storage type for T2/T3B, T for T3A)
    T *out2;                    // KIND_T3A: accumulator planes
    double *mass_partial;       // per-CTA sum of phi of out1 (T2, T3B), may be null
    const T *ufield, *vfield;   // VEL_FIELD cell-centre components
    T a, b;                     // bar f^+ = a X + b g
    T h;                        // reconstruction time of the faces
    T c1, c2, c3;               // f_b = c1 bar f + c2 f^eq_b + c3 S_b   (Eq. (27))
    T al1, be1, ga1;            // out1 = al1 X + be1 g + ga1 L (+ acc)
    T al2, be2, ga2;            // out2 = al2 X + be2 g + ga2 L
    T tau, theta_c, phiA, phiB; // theta = theta_c (phi - phiA)(phi - phiB)   (Eq. (4))
    T inv_dtD;                  // 1 / (time between phi_old and X)
    int useD;
    int vel_kind;
    T vp0, vp1, vp2;            // velocity parameters
    T t, t_old, t_face;         // time of X, of phi_old, of the faces
    T qscale, qinv;             // deviation storage scale s and 1 / s
    uint32_t seed;              // step index: the counter of the stochastic rounding
    double *dbg;                // generic kernel, debug: face values out (null normally)
};

template <typename T>
__device__ __forceinline__ size_t gidx(const StepParams<T> &p, int x, int y) {
    return (size_t)(y + GHOST) * p.pitch + (size_t)(x + GHOST);
}

// Writes v at cell (x, y) and at each of its periodic images inside the ghost border.
template <typename T, typename V>
__device__ __forceinline__ void put_cell(const StepParams<T> &p, V *plane, int x, int y, V v) {
    plane[gidx(p, x, y)] = v;
    const bool xl = x < GHOST, xh = x >= p.nx - GHOST, yl = y < GHOST, yh = y >= p.ny - GHOST;
    if (!(xl | xh | yl | yh)) return;
#pragma unroll
    for (int ay = -1; ay <= 1; ay++) {
        const int yy = y + ay * p.ny;
        if (yy < -GHOST || yy >= p.ny + GHOST) continue;
#pragma unroll
        for (int ax = -1; ax <= 1; ax++) {
            const int xx = x + ax * p.nx;
            if ((ax == 0 && ay == 0) || xx < -GHOST || xx >= p.nx + GHOST) continue;
            plane[gidx(p, xx, yy)] = v;
        }
    }
}

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic
// stream serialization may be scheduled before the kernel ahead of it in the
// stream has finished, once every CTA of that kernel has signalled (pdl_trigger)
// or exited; it must then wait (pdl_wait) for that kernel to complete, with its
// memory visible, before reading its results. Both are no-ops for a kernel
// launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ int wrapc(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// ---- prescribed velocity (Sec. II.A; Sec. III) ------------------------------
template <typename T>
__device__ __forceinline__ T sinpi_(T x);
template <>
__device__ __forceinline__ double sinpi_(double x) { return sinpi(x); }
template <>
__device__ __forceinline__ float sinpi_(float x) { return sinpif(x); }
template <typename T>
__device__ __forceinline__ T cospi_(T x);
template <>
__device__ __forceinline__ double cospi_(double x) { return cospi(x); }
template <>
__device__ __forceinline__ float cospi_(float x) { return cospif(x); }

// smoothed deformation of Sec. III.D without its reversal factor: 4 x 4 cells of
// vortices on a box of side L, u = -U sin(4 pi x/L) sin(4 pi y/L),
// v = -U cos(4 pi x/L) cos(4 pi y/L)
template <typename T>
__device__ __forceinline__ void deform_spatial(const StepParams<T> &p, T x, T y, T &u, T &v) {
    const T L = p.vp0, U = p.vp1;
    const T sx = sinpi_(T(4) * x / L), sy = sinpi_(T(4) * y / L);
    const T cx = cospi_(T(4) * x / L), cy = cospi_(T(4) * y / L);
    u = -U * sx * sy;
    v = -U * cx * cy;
}

template <typename T>
__device__ __forceinline__ void vel_analytic(const StepParams<T> &p, T x, T y, T t, T &u, T &v) {
    if (p.vel_kind == VEL_UNIFORM) {
        u = p.vp0;
        v = p.vp1;
    } else if (p.vel_kind == VEL_ROTATION) {
        u = -p.vp2 * (y - p.vp1);
        v = p.vp2 * (x - p.vp0);
    } else if (p.vel_kind == VEL_DEFORM) {   // reversed by cos(pi t / T)
        deform_spatial(p, x, y, u, v);
        const T c = cospi_(t / p.vp2);
        u *= c;
        v *= c;
    } else {  // single vortex, period box L, amplitude U, reversal period T
        const T L = p.vp0, U = p.vp1;
        const T sx = sinpi_(x / L), sy = sinpi_(y / L), c = cospi_(t / p.vp2);
        u = -U * sx * sx * sinpi_(T(2) * y / L) * c;
        v = U * sy * sy * sinpi_(T(2) * x / L) * c;
    }
}

// velocity at the centre of cell (gx, gy) (wrapped indices)
template <typename T>
__device__ __forceinline__ void vel_cell(const StepParams<T> &p, int gx, int gy, T t, T &u, T &v) {
    if (p.vel_kind == VEL_FIELD) {
        const size_t c = gidx(p, gx, gy);
        u = p.ufield[c];
        v = p.vfield[c];
    } else {
        vel_analytic(p, T(gx) + T(0.5), T(gy) + T(0.5), t, u, v);
    }
}

// velocity at the east (dir 0: x = gx + 1) or north (dir 1: y = gy + 1) face midpoint
template <typename T>
__device__ __forceinline__ void vel_face(const StepParams<T> &p, int gx, int gy, int dir, T t, T &u, T &v) {
    if (p.vel_kind == VEL_FIELD) {
        int nxg = gx, nyg = gy;
        if (dir == 0) nxg = gx + 1 == p.nx ? 0 : gx + 1;
        else nyg = gy + 1 == p.ny ? 0 : gy + 1;
        const size_t c0 = gidx(p, gx, gy), c1 = gidx(p, nxg, nyg);
        u = T(0.5) * (p.ufield[c0] + p.ufield[c1]);
        v = T(0.5) * (p.vfield[c0] + p.vfield[c1]);
    } else if (dir == 0) {
        vel_analytic(p, T(gx) + T(1), T(gy) + T(0.5), t, u, v);
    } else {
        vel_analytic(p, T(gx) + T(0.5), T(gy) + T(1), t, u, v);
    }
}

// ---- isotropic finite differences (Sec. II.B.1, II.B.2) ----------------------
// F points at the centre value of a shared-memory plane with row stride ld.
#define FA(dx, dy) F[(dy) * ld + (dx)]

// Lattice-moment gradient (1/cs^2) sum_k w_k e_k F(x + e_k): leading error
// (1/6) grad lap F, isotropic.
template <typename T>
__device__ __forceinline__ void grad9(const T *F, int ld, T &gx, T &gy) {
    const T ne = FA(1, 1), nw = FA(-1, 1), se = FA(1, -1), sw = FA(-1, -1);
    gx = (FA(1, 0) - FA(-1, 0)) * T(1.0 / 3.0) + ((ne - nw) + (se - sw)) * T(1.0 / 12.0);
    gy = (FA(0, 1) - FA(0, -1)) * T(1.0 / 3.0) + ((ne - se) + (nw - sw)) * T(1.0 / 12.0);
}

// Lattice-moment Hessian (1/cs^4) sum_k w_k (e_a e_b - cs^2 delta_ab) F(x + s e_k) / s^2.
template <typename T, int S>
__device__ __forceinline__ void hess9(const T *F, int ld, T &hxx, T &hxy, T &hyy) {
    const T c = FA(0, 0);
    const T ew = FA(S, 0) + FA(-S, 0), ns = FA(0, S) + FA(0, -S);
    const T ne = FA(S, S), nw = FA(-S, S), se = FA(S, -S), sw = FA(-S, -S);
    const T cor = (ne + nw) + (se + sw);
    constexpr T inv = T(1) / T(S * S);
    hxx = (T(2.0 / 3.0) * ew - T(1.0 / 3.0) * ns + T(1.0 / 6.0) * cor - T(4.0 / 3.0) * c) * inv;
    hyy = (T(2.0 / 3.0) * ns - T(1.0 / 3.0) * ew + T(1.0 / 6.0) * cor - T(4.0 / 3.0) * c) * inv;
    hxy = ((ne - nw) - (se - sw)) * T(0.25) * inv;
}

// Fourth-order gradient on the 5x5 block without corners, with isotropic
// fifth-order error: weights 13/30, 2/15, -1/60 (at (1, +-2)), -1/60 (at (2, 0)),
// -1/30 (at (2, +-1)), antisymmetric along the derivative.
template <typename T>
__device__ __forceinline__ void grad21(const T *F, int ld, T &gx, T &gy) {
    gx = T(13.0 / 30.0) * (FA(1, 0) - FA(-1, 0)) +
         T(2.0 / 15.0) * ((FA(1, 1) - FA(-1, 1)) + (FA(1, -1) - FA(-1, -1))) -
         T(1.0 / 60.0) * ((FA(1, 2) - FA(-1, 2)) + (FA(1, -2) - FA(-1, -2))) -
         T(1.0 / 60.0) * (FA(2, 0) - FA(-2, 0)) -
         T(1.0 / 30.0) * ((FA(2, 1) - FA(-2, 1)) + (FA(2, -1) - FA(-2, -1)));
    gy = T(13.0 / 30.0) * (FA(0, 1) - FA(0, -1)) +
         T(2.0 / 15.0) * ((FA(1, 1) - FA(1, -1)) + (FA(-1, 1) - FA(-1, -1))) -
         T(1.0 / 60.0) * ((FA(2, 1) - FA(2, -1)) + (FA(-2, 1) - FA(-2, -1))) -
         T(1.0 / 60.0) * (FA(0, 2) - FA(0, -2)) -
         T(1.0 / 30.0) * ((FA(1, 2) - FA(1, -2)) + (FA(-1, 2) - FA(-1, -2)));
}

template <typename T, int ORDER>
__device__ __forceinline__ void grad_p(const T *F, int ld, T &gx, T &gy) {
    if constexpr (ORDER == 4) grad21(F, ld, gx, gy);
    else grad9(F, ld, gx, gy);
}

// Taylor expansion about the cell at F evaluated at displacement (dx, dy):
// value + d.grad (+ 1/2 d d : H for p >= 3) (+ 1/6 d d d : T for p = 4).
template <typename T, int ORDER>
__device__ __forceinline__ T taylor(const T *F, int ld, T dx, T dy) {
    T gx, gy;
    grad_p<T, ORDER>(F, ld, gx, gy);
    T v = FA(0, 0) + dx * gx + dy * gy;
    if constexpr (ORDER >= 3) {
        T hxx, hxy, hyy;
        if constexpr (ORDER == 4) {
            // (4 H_1 - H_2) / 3: fourth order
            T axx, axy, ayy, bxx, bxy, byy;
            hess9<T, 1>(F, ld, axx, axy, ayy);
            hess9<T, 2>(F, ld, bxx, bxy, byy);
            hxx = T(4.0 / 3.0) * axx - T(1.0 / 3.0) * bxx;
            hxy = T(4.0 / 3.0) * axy - T(1.0 / 3.0) * bxy;
            hyy = T(4.0 / 3.0) * ayy - T(1.0 / 3.0) * byy;
        } else {
            hess9<T, 1>(F, ld, hxx, hxy, hyy);
        }
        v += T(0.5) * (dx * dx * hxx + T(2) * dx * dy * hxy + dy * dy * hyy);
    }
    if constexpr (ORDER == 4) {
        // second-order third derivatives (products of central differences)
        const T txxx = T(0.5) * (FA(2, 0) - FA(-2, 0)) - (FA(1, 0) - FA(-1, 0));
        const T tyyy = T(0.5) * (FA(0, 2) - FA(0, -2)) - (FA(0, 1) - FA(0, -1));
        const T txxy = T(0.5) * ((FA(1, 1) - FA(1, -1)) + (FA(-1, 1) - FA(-1, -1))) - (FA(0, 1) - FA(0, -1));
        const T txyy = T(0.5) * ((FA(1, 1) - FA(-1, 1)) + (FA(1, -1) - FA(-1, -1))) - (FA(1, 0) - FA(-1, 0));
        v += (dx * dx * dx * txxx + T(3) * dx * dx * dy * txxy + T(3) * dx * dy * dy * txyy +
              dy * dy * dy * tyyy) * T(1.0 / 6.0);
    }
    return v;
}
#undef FA

// ---- block reduction in FP64 (fixed order: deterministic) -------------------
__device__ __forceinline__ double block_sum(double v, double *sred) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; w++) s += sred[w];
    }
    __syncthreads();
    return s;  // valid in thread 0
}

// 32-bit integer hash (xor-shift / multiply rounds), used as a counter-based
// source of uniform bits: hash(cell, step) needs no state. Shifts and
// multipliers are the published "lowbias32" constants found by C. Wellons'
// hash-prospector search ("Prospecting for Hash Functions", 2018).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// a + b rounded stochastically to float: the exact sum s + e is found with the
// error-free two-sum (Knuth), then the neighbour of s on the side of e is taken
// with probability |e| / |neighbour - s|, so the rounding is unbiased in
// expectation and small increments are not lost to round-to-nearest
__device__ __forceinline__ float add_sr(float a, float b, uint32_t bits) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    if (e == 0.0f || s == 0.0f) return s;
    const int away = (e > 0.0f) == (s > 0.0f) ? 1 : -1;   // step away from or toward zero
    const float n = __int_as_float(__float_as_int(s) + away);
    const float u = (float)(bits >> 8) * 0x1p-24f;
    return u * fabsf(__fsub_rn(n, s)) < fabsf(e) ? n : s;
}

// the uniform bits of cell (gx, gy) at the step p.seed
template <typename T>
__device__ __forceinline__ uint32_t sr_bits(const StepParams<T> &p, int gx, int gy) {
    return mix32(((uint32_t)gy * (uint32_t)p.nx + (uint32_t)gx) ^ mix32(p.seed));
}

template <typename ST>
__device__ __forceinline__ float to_f(ST v);
template <>
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// ---- the fused step kernel ----------------------------------------------------
template <typename T, typename ST, int ORDER, int FLUX, int KIND, int TX, int TY>
struct Tile {
    static constexpr int R = ORDER == 4 ? 2 : 1;
    static constexpr int H = 1 + 2 * R;
    static constexpr int WH = TX + 2 * H, HH = TY + 2 * H;          // state region
    static constexpr int WC = TX + 2 + 2 * R, HC = TY + 2 + 2 * R;  // cell-quantity region
    static constexpr int WF = TX + 1, HF = TY + 1;                  // face owners
    static constexpr int NH = WH * HH, NC = WC * HC, NF = WF * HF;
    static constexpr size_t red_offset = (sizeof(T) * (size_t)(9 * NH + NH + 9 * NC + 4 * NC + 18 * NF) + 15) / 16 * 16;
    static constexpr size_t smem_bytes = red_offset + 64 * sizeof(double);
};

template <typename T, typename ST, int ORDER, int FLUX, int KIND, int TX, int TY>
__global__ void __launch_bounds__(256) step_kernel(const StepParams<T> p) {
    using TL = Tile<T, ST, ORDER, FLUX, KIND, TX, TY>;
    constexpr int R = TL::R, H = TL::H, WH = TL::WH, WC = TL::WC, WF = TL::WF;
    constexpr int NH = TL::NH, NC = TL::NC, NF = TL::NF;
    constexpr bool DEV = Store<T, ST>::deviation, PHIP = Store<T, ST>::phi_plane;
    static_assert(KIND == KIND_T2 ? Store<T, ST>::t2 : Store<T, ST>::t3, "scheme not served by this storage");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sX = reinterpret_cast<T *>(smem_raw);  // [9][NH]
    T *sPhi = sX + 9 * NH;                    // [NH]
    T *sFbp = sPhi + NH;                      // [9][NC]
    T *sV = sFbp + 9 * NC;                    // [2][NC]
    T *sP = sV + 2 * NC;                      // [2][NC]
    T *sFb = sP + 2 * NC;                     // [9][2][NF]
    double *sred = reinterpret_cast<double *>(smem_raw + TL::red_offset);

    const int nx = p.nx, ny = p.ny;
    const size_t plane = p.plane;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x, nt = blockDim.x;

    // S0: state + halo -> shared memory; phi of X
    for (int idx = tid; idx < NH; idx += nt) {
        const int ly = idx / WH, lx = idx - ly * WH;
        int gx = x0 - H + lx, gy = y0 - H + ly;
        gx = wrapc(gx, nx);
        gy = wrapc(gy, ny);
        const size_t g = gidx(p, gx, gy);
        if constexpr (DEV) {
            const __half *Xq = static_cast<const __half *>(p.X);
            const T ph = p.phi_cur[g];
#pragma unroll
            for (int k = 0; k < 9; k++) sX[k * NH + idx] = wq<T>(k) * (ph + to_f(Xq[k * plane + g]) * p.qinv);
            sPhi[idx] = ph;
        } else {
            const T *Xf = static_cast<const T *>(p.X);
            T ph = T(0);
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const T v = Xf[k * plane + g];
                sX[k * NH + idx] = v;
                ph += v;
            }
            sPhi[idx] = PHIP ? p.phi_cur[g] : ph;
        }
    }
    __syncthreads();

    // S1: cell quantities and bar f^+ on the tile plus 1 + R cells
    for (int idx = tid; idx < NC; idx += nt) {
        const int ly = idx / WC, lx = idx - ly * WC;
        const int rx = lx - (1 + R), ry = ly - (1 + R);       // relative to the tile origin
        const int hidx = (ry + H) * WH + (rx + H);
        int gx = x0 + rx, gy = y0 + ry;
        gx = wrapc(gx, nx);
        gy = wrapc(gy, ny);
        const T ph = sPhi[hidx];
        T gxp, gyp;
        grad_p<T, ORDER>(sPhi + hidx, WH, gxp, gyp);
        const T g2 = gxp * gxp + gyp * gyp;
        T nxv = T(0), nyv = T(0);
        if (g2 > T(1e-24)) {  // n = grad phi / |grad phi| (Eq. (2)); n = 0 where it vanishes
            const T inv = T(1) / sqrt(g2);
            nxv = gxp * inv;
            nyv = gyp * inv;
        }
        const T theta = p.theta_c * (ph - p.phiA) * (ph - p.phiB);  // Eq. (4)
        T u, v;
        vel_cell(p, gx, gy, p.t, u, v);
        T Dx = T(0), Dy = T(0);
        if (p.useD) {  // d(phi u)/dt, backward difference
            T uo, vo;
            vel_cell(p, gx, gy, p.t_old, uo, vo);
            const T po = p.phi_old[gidx(p, gx, gy)];
            Dx = (ph * u - po * uo) * p.inv_dtD;
            Dy = (ph * v - po * vo) * p.inv_dtD;
        }
        // S_k = w_k xi_k . V with V = theta n + D / RT           (Eq. (14b))
        const T Vx = theta * nxv + T(3) * Dx, Vy = theta * nyv + T(3) * Dy;
        // g_k = f^eq_k + tau S_k = w_k (phi + xi_k . P),  P = phi u / RT + tau V
        const T Px = T(3) * ph * u + p.tau * Vx, Py = T(3) * ph * v + p.tau * Vy;
        sV[idx] = Vx;
        sV[NC + idx] = Vy;
        sP[idx] = Px;
        sP[NC + idx] = Py;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const T gk = wq<T>(k) * (ph + (T(ex(k)) * Px + T(ey(k)) * Py));
            // a + b = 1: written as an increment so FP32 keeps the non-equilibrium part
            const T xk = sX[k * NH + hidx];
            sFbp[k * NC + idx] = xk + p.b * (gk - xk);
        }
    }
    __syncthreads();

    // S2: faces. Owner cell (fx, fy) in [-1, TX) x [-1, TY) computes its east and
    // north faces.
    for (int idx = tid; idx < NF; idx += nt) {
        const int fy = idx / WF - 1, fx = idx - (fy + 1) * WF - 1;
        const int ci = (fy + 1 + R) * WC + (fx + 1 + R);  // owner in the cell-quantity region
        const int cE = ci + 1, cN = ci + WC;
        T fe[9], fn[9];
        T phE = T(0), phN = T(0);
        const T h = p.h;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const T *F = sFbp + k * NC;
            const T exk = T(ex(k)), eyk = T(ey(k));
            T vE, vN;
            if constexpr (FLUX == 0) {
                // Upwind (Eq. (26)): expand about the cell centre nearest to
                // x_b - xi h; a tie (xi normal to the face = 0) averages both sides.
                if (ex(k) > 0) vE = taylor<T, ORDER>(F + ci, WC, T(0.5) - h, -eyk * h);
                else if (ex(k) < 0) vE = taylor<T, ORDER>(F + cE, WC, h - T(0.5), -eyk * h);
                else vE = T(0.5) * (taylor<T, ORDER>(F + ci, WC, T(0.5), -eyk * h) +
                                    taylor<T, ORDER>(F + cE, WC, T(-0.5), -eyk * h));
                if (ey(k) > 0) vN = taylor<T, ORDER>(F + ci, WC, -exk * h, T(0.5) - h);
                else if (ey(k) < 0) vN = taylor<T, ORDER>(F + cN, WC, -exk * h, h - T(0.5));
                else vN = T(0.5) * (taylor<T, ORDER>(F + ci, WC, -exk * h, T(0.5)) +
                                    taylor<T, ORDER>(F + cN, WC, -exk * h, T(-0.5)));
            } else {
                // Central (Eq. (25)): face mean, normal difference, mean tangential derivative.
                T gxc, gyc, gxe, gye, gxn, gyn;
                grad_p<T, ORDER>(F + ci, WC, gxc, gyc);
                grad_p<T, ORDER>(F + cE, WC, gxe, gye);
                grad_p<T, ORDER>(F + cN, WC, gxn, gyn);
                const T Fc = F[ci], Fe = F[cE], Fn = F[cN];
                vE = T(0.5) * (Fc + Fe) - h * (exk * (Fe - Fc) + eyk * (T(0.5) * (gyc + gye)));
                vN = T(0.5) * (Fc + Fn) - h * (exk * (T(0.5) * (gxc + gxn)) + eyk * (Fn - Fc));
            }
            fe[k] = vE;
            fn[k] = vN;
            phE += vE;
            phN += vN;
        }
        int gx = x0 + fx, gy = y0 + fy;
        gx = wrapc(gx, nx);
        gy = wrapc(gy, ny);
        T uE, vE_, uN, vN_;
        vel_face(p, gx, gy, 0, p.t_face, uE, vE_);
        vel_face(p, gx, gy, 1, p.t_face, uN, vN_);
        // face source: mean of the two cells at the base time
        const T VxE = T(0.5) * (sV[ci] + sV[cE]), VyE = T(0.5) * (sV[NC + ci] + sV[NC + cE]);
        const T VxN = T(0.5) * (sV[ci] + sV[cN]), VyN = T(0.5) * (sV[NC + ci] + sV[NC + cN]);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const T exk = T(ex(k)), eyk = T(ey(k)), w = wq<T>(k);
            const T feqE = w * phE * (T(1) + T(3) * (exk * uE + eyk * vE_));
            const T feqN = w * phN * (T(1) + T(3) * (exk * uN + eyk * vN_));
            const T SE = w * (exk * VxE + eyk * VyE), SN = w * (exk * VxN + eyk * VyN);
            // c1 + c2 = 1: f_b = bar f + c2 (f^eq_b - bar f) + c3 S_b
            sFb[(2 * k) * NF + idx] = fe[k] + p.c2 * (feqE - fe[k]) + p.c3 * SE;
            sFb[(2 * k + 1) * NF + idx] = fn[k] + p.c2 * (feqN - fn[k]) + p.c3 * SN;
        }
        // debug read-out: bar f and f at the east and north faces of the tile's own
        // cells, four arrays of 9 x ny x nx doubles (each face has one owner)
        if (p.dbg != nullptr && fx >= 0 && fy >= 0 && x0 + fx < nx && y0 + fy < ny) {
            const size_t n = (size_t)nx * ny, c = (size_t)gy * nx + gx;
#pragma unroll
            for (int k = 0; k < 9; k++) {
                p.dbg[(0 * 9 + k) * n + c] = (double)fe[k];
                p.dbg[(1 * 9 + k) * n + c] = (double)fn[k];
                p.dbg[(2 * 9 + k) * n + c] = (double)sFb[(2 * k) * NF + idx];
                p.dbg[(3 * 9 + k) * n + c] = (double)sFb[(2 * k + 1) * NF + idx];
            }
        }
    }
    __syncthreads();

    // S3: flux and update of the tile's own cells
    double msum = 0.0;
    for (int idx = tid; idx < TX * TY; idx += nt) {
        const int ly = idx / TX, lx = idx - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const size_t g = gidx(p, gx, gy);
        const int hidx = (ly + H) * WH + (lx + H);
        const int cidx = (ly + 1 + R) * WC + (lx + 1 + R);
        const int fidx = (ly + 1) * WF + (lx + 1);
        const T ph = sPhi[hidx], Px = sP[cidx], Py = sP[NC + cidx];
        // out = base + beta (g - X) + gamma L with base = X (alpha + beta = 1) or the
        // accumulator; the rest component is then set so that the new phi equals
        // sum(base) + gamma sum_k L_k (identical in exact arithmetic, since
        // sum_k g_k = sum_k X_k = phi), which keeps FP32 rounding from drifting
        // the conserved moment.
        T o1[9], o2[9];
        T sumL = T(0), sumB = T(0);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const T gk = wq<T>(k) * (ph + (T(ex(k)) * Px + T(ey(k)) * Py));
            const T *fE = sFb + (2 * k) * NF, *fN = sFb + (2 * k + 1) * NF;
            // Eq. (21) with the outward normal of a unit cell
            const T L = -(T(ex(k)) * (fE[fidx] - fE[fidx - 1]) + T(ey(k)) * (fN[fidx] - fN[fidx - WF]));
            const T Xk = sX[k * NH + hidx];
            T base = Xk;
            if constexpr (KIND == KIND_T3B) {
                base = static_cast<const T *>(p.acc)[k * plane + g];
                sumB += base;
            }
            o1[k] = base + p.be1 * (gk - Xk) + p.ga1 * L;
            if constexpr (KIND == KIND_T3A) o2[k] = Xk + p.be2 * (gk - Xk) + p.ga2 * L;
            sumL += L;
        }
        // phi planes: the base phi (T3B: the accumulator's, from its plane) plus the flux
        // sum, rounded without bias
        T phn;
        const uint32_t bits = PHIP ? sr_bits(p, gx, gy) : 0u;
        if constexpr (PHIP)
            phn = add_sr(KIND == KIND_T3B ? p.phi_acc[g] : ph, p.ga1 * sumL, bits);
        else
            phn = (KIND == KIND_T3B ? sumB : ph) + p.ga1 * sumL;
        {
            T r = T(0);
#pragma unroll
            for (int k = 1; k < 9; k++) r += o1[k];
            o1[0] = phn - r;
        }
        if constexpr (KIND == KIND_T3A) {
            T ph2;
            if constexpr (PHIP) ph2 = add_sr(ph, p.ga2 * sumL, mix32(bits));
            else ph2 = ph + p.ga2 * sumL;
            T r = T(0);
#pragma unroll
            for (int k = 1; k < 9; k++) r += o2[k];
            o2[0] = ph2 - r;
#pragma unroll
            for (int k = 0; k < 9; k++) put_cell(p, p.out2 + k * plane, gx, gy, o2[k]);
            if constexpr (PHIP) put_cell(p, p.phi_out2, gx, gy, ph2);
        }
        if constexpr (DEV) {
            __half *Oq = static_cast<__half *>(p.out1);
#pragma unroll
            for (int k = 0; k < 9; k++)
                put_cell(p, Oq + k * plane, gx, gy,
                         __float2half_rn((o1[k] - wq<T>(k) * phn) * (p.qscale * (T(1) / wq<T>(k)))));
            put_cell(p, p.phi_out, gx, gy, phn);
            msum += (double)phn;
        } else if constexpr (PHIP) {
            T *O = static_cast<T *>(p.out1);
#pragma unroll
            for (int k = 0; k < 9; k++) put_cell(p, O + k * plane, gx, gy, o1[k]);
            put_cell(p, p.phi_out, gx, gy, phn);
            msum += (double)phn;
        } else {
            T *O = static_cast<T *>(p.out1);
            T s = T(0);
#pragma unroll
            for (int k = 0; k < 9; k++) {
                put_cell(p, O + k * plane, gx, gy, o1[k]);
                s += o1[k];
            }
            if (KIND != KIND_T3B) put_cell(p, p.phi_out, gx, gy, ph);
            msum += (double)s;
        }
    }
    if (p.mass_partial != nullptr) {
        const double s = block_sum(msum, sred);
        if (tid == 0) p.mass_partial[blockIdx.y * p.tiles_x + blockIdx.x] = s;
    }
}

// ---- initial state: f = f^eq (Omega = 0), D = 0 ------------------------------
// X = f^eq - frac * dt * S with frac = 1/2 (two-stage tilde f) or 1/4 (hat f).
// phi0 uses the plane layout; only its cells (not its ghosts) are read.
template <typename T, typename ST, int ORDER>
__global__ void init_kernel(const StepParams<T> p, const T *phi0, T frac_dt) {
    constexpr bool DEV = Store<T, ST>::deviation;
    constexpr int R = ORDER == 4 ? 2 : 1;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= p.nx || gy >= p.ny) return;
    const int nx = p.nx, ny = p.ny;
    const size_t plane = p.plane;
    // gather the (2R+1)^2 neighbourhood of phi0 into registers
    T nb[(2 * R + 1) * (2 * R + 1)];
#pragma unroll
    for (int dy = -R; dy <= R; dy++)
#pragma unroll
        for (int dx = -R; dx <= R; dx++)
            nb[(dy + R) * (2 * R + 1) + (dx + R)] = phi0[gidx(p, wrapc(gx + dx, nx), wrapc(gy + dy, ny))];
    const T *c = nb + R * (2 * R + 1) + R;
    T gxp, gyp;
    grad_p<T, ORDER>(c, 2 * R + 1, gxp, gyp);
    const T ph = *c;
    const T g2 = gxp * gxp + gyp * gyp;
    T nxv = T(0), nyv = T(0);
    if (g2 > T(1e-24)) {
        const T inv = T(1) / sqrt(g2);
        nxv = gxp * inv;
        nyv = gyp * inv;
    }
    const T theta = p.theta_c * (ph - p.phiA) * (ph - p.phiB);
    T u, v;
    vel_cell(p, gx, gy, p.t, u, v);
    const T Vx = theta * nxv, Vy = theta * nyv;
    T fk[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const T exk = T(ex(k)), eyk = T(ey(k)), w = wq<T>(k);
        const T feq = w * ph * (T(1) + T(3) * (exk * u + eyk * v));
        const T S = w * (exk * Vx + eyk * Vy);
        fk[k] = feq - frac_dt * S;
    }
    if constexpr (DEV) {
        // phi of X: sum of the distribution (equals phi0 up to rounding)
        T phn = T(0);
#pragma unroll
        for (int k = 0; k < 9; k++) phn += fk[k];
        __half *Oq = static_cast<__half *>(p.out1);
#pragma unroll
        for (int k = 0; k < 9; k++)
            put_cell(p, Oq + k * plane, gx, gy,
                     __float2half_rn((fk[k] - wq<T>(k) * phn) * (p.qscale * (T(1) / wq<T>(k)))));
        put_cell(p, p.phi_out, gx, gy, phn);
    } else {
        T *O = static_cast<T *>(p.out1);
#pragma unroll
        for (int k = 0; k < 9; k++) put_cell(p, O + k * plane, gx, gy, fk[k]);
        // phi plane: phi of X; otherwise phi of the previous level for d(phi u)/dt
        put_cell(p, p.phi_out, gx, gy, ph);
    }
}

// sum_k X_k of one cell (the cell's phi), in the storage's arithmetic type
template <typename T, typename ST>
__device__ __forceinline__ T cell_phi(const StepParams<T> &p, size_t g) {
    if constexpr (Store<T, ST>::phi_plane) {
        return p.phi_cur[g];
    } else {
        const T *Xf = static_cast<const T *>(p.X);
        T s = T(0);
#pragma unroll
        for (int k = 0; k < 9; k++) s += Xf[k * p.plane + g];
        return s;
    }
}

// ---- mass: per-tile FP64 partials in the step kernel's tiling, then one CTA --
template <typename T, typename ST>
__global__ void __launch_bounds__(256) mass_partial_kernel(const StepParams<T> p) {
    __shared__ double sred[32];
    const int x0 = blockIdx.x * p.tile_w, y0 = blockIdx.y * p.tile_h;
    double msum = 0.0;
    for (int idx = threadIdx.x; idx < p.tile_w * p.tile_h; idx += blockDim.x) {
        const int ly = idx / p.tile_w, lx = idx - ly * p.tile_w;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= p.nx || gy >= p.ny) continue;
        msum += (double)cell_phi<T, ST>(p, gidx(p, gx, gy));
    }
    const double s = block_sum(msum, sred);
    if (threadIdx.x == 0) p.mass_partial[blockIdx.y * p.tiles_x + blockIdx.x] = s;
}

// phi of the state into a dense ny * nx array of T
template <typename T, typename ST, typename O = T>
__global__ void phi_kernel(const StepParams<T> p, O *out) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= p.nx || gy >= p.ny) return;
    out[(size_t)gy * p.nx + gx] = (O)cell_phi<T, ST>(p, gidx(p, gx, gy));
}

}  // namespace dugks
