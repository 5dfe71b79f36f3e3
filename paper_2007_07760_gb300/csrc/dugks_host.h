// dugks_host.h -- host helpers shared by the context API (dugks_api.cu) and the
// batch API (dugks_batch.cu): face-stencil coefficients of the fast kernel, TMA
// tensor maps of the ghost-bordered plane layout, and ghosted uploads.
#pragma once

#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_internal.h"

namespace dugks {
namespace host {

// ---- face stencils of the fast path ------------------------------------------
// The face value bar f_k(x_b) is a fixed linear combination of bar f^+_k at the
// cells around the face: the Taylor expansion of Eq. (26) about the upwind cell
// (value + d.grad + d d : H / 2, + d d d : T / 6 at order 4), or the central form
// of Eq. (25). Below: the weights at offset (a, b) from the expansion cell of the
// stencils the generic kernel applies (orders 2 and 3: 9-point lattice moments;
// order 4: the 21-point gradient, the Richardson Hessian (4 H_1 - H_2) / 3 and
// second-order central third derivatives).
inline double G9x(int a, int b) {
    if (a < -1 || a > 1 || b < -1 || b > 1) return 0.0;
    return a * (b == 0 ? 1.0 / 3.0 : 1.0 / 12.0);
}
inline double G9y(int a, int b) { return G9x(b, a); }
inline double G21x(int a, int b) {   // weights 13/30, 2/15, -1/60 at (1, +-2), -1/60 at (2, 0), -1/30 at (2, +-1)
    const int aa = a < 0 ? -a : a, bb = b < 0 ? -b : b, s = a < 0 ? -1 : 1;
    if (aa == 0 || aa > 2 || bb > 2) return 0.0;
    if (aa == 1) return s * (bb == 0 ? 13.0 / 30.0 : bb == 1 ? 2.0 / 15.0 : -1.0 / 60.0);
    return s * (bb == 0 ? -1.0 / 60.0 : bb == 1 ? -1.0 / 30.0 : 0.0);
}
inline double G21y(int a, int b) { return G21x(b, a); }
// 9-point lattice-moment Hessian with spacing S (points at S times the 3 x 3 block)
inline double H9s(int i, int j, int a, int b, int S) {   // i, j in {0: x, 1: y}
    if (a % S != 0 || b % S != 0) return 0.0;
    a /= S;
    b /= S;
    if (a < -1 || a > 1 || b < -1 || b > 1) return 0.0;
    const double inv = 1.0 / (S * S);
    if (i != j) return (a != 0 && b != 0) ? 0.25 * a * b * inv : 0.0;
    const int along = i == 0 ? a : b, across = i == 0 ? b : a;
    if (along == 0 && across == 0) return -4.0 / 3.0 * inv;
    if (across == 0) return 2.0 / 3.0 * inv;
    if (along == 0) return -1.0 / 3.0 * inv;
    return 1.0 / 6.0 * inv;
}
inline double Hp(int order, int i, int j, int a, int b) {
    return order == 4 ? 4.0 / 3.0 * H9s(i, j, a, b, 1) - 1.0 / 3.0 * H9s(i, j, a, b, 2) : H9s(i, j, a, b, 1);
}
// third derivatives: txxx = (F(2,0) - F(-2,0)) / 2 - (F(1,0) - F(-1,0)); txxy = ((F(1,1) - F(1,-1))
// + (F(-1,1) - F(-1,-1))) / 2 - (F(0,1) - F(0,-1)); tyyy, txyy by symmetry
inline double Txxx(int a, int b) {
    if (b != 0) return 0.0;
    return a == 2 ? 0.5 : a == -2 ? -0.5 : a == 1 ? -1.0 : a == -1 ? 1.0 : 0.0;
}
inline double Txxy(int a, int b) {
    if ((a == 1 || a == -1) && (b == 1 || b == -1)) return 0.5 * b;
    if (a == 0 && (b == 1 || b == -1)) return -1.0 * b;
    return 0.0;
}
inline double taylor_w(int order, double dx, double dy, int a, int b) {
    double w = (a == 0 && b == 0) ? 1.0 : 0.0;
    if (order == 4) w += dx * G21x(a, b) + dy * G21y(a, b);
    else w += dx * G9x(a, b) + dy * G9y(a, b);
    if (order >= 3)
        w += 0.5 * dx * dx * Hp(order, 0, 0, a, b) + dx * dy * Hp(order, 0, 1, a, b) +
             0.5 * dy * dy * Hp(order, 1, 1, a, b);
    if (order == 4)
        w += (dx * dx * dx * Txxx(a, b) + 3.0 * dx * dx * dy * Txxy(a, b) + 3.0 * dx * dy * dy * Txxy(b, a) +
              dy * dy * dy * Txxx(b, a)) / 6.0;
    return w;
}

// Face-stencil tables for stencil radius R (1: orders 2-3, 2: orders 4 and 5).
template <typename T, int R>
inline FaceCoefs<T, R> make_face_coefs_r(int order, int flux, double h) {
    constexpr int NE = 2 * R + 1, NA = 2 * R + 2;
    double e[9][NE][NA] = {}, n[9][NA][NA] = {};
    auto gx = [&](int a, int b) { return order == 4 ? G21x(a, b) : G9x(a, b); };
    auto gy = [&](int a, int b) { return order == 4 ? G21y(a, b) : G9y(a, b); };
    for (int k = 0; k < 9; k++) {
        const int kx = ex(k), ky = ey(k);
        // east face: taps (b, a) -> e[k][b + R][a + R], b in -R..R, a in -R..R+1
        auto addE = [&](int cx, double wgt, double dx, double dy) {   // expansion about cell (cx, 0)
            for (int b = -R; b <= R; b++)
                for (int a = -R; a <= R; a++) e[k][b + R][cx + a + R] += wgt * taylor_w(order, dx, dy, a, b);
        };
        auto addN = [&](int cy, double wgt, double dx, double dy) {   // expansion about cell (0, cy)
            for (int b = -R; b <= R; b++)
                for (int a = -R; a <= R; a++) n[k][cy + b + R][a + R] += wgt * taylor_w(order, dx, dy, a, b);
        };
        if (order == 5) {
            // DUGKS-T2S5: the degree-4 tensor-product Lagrange interpolant on the 5 x 5
            // cells centred at the cell nearest to x_b - xi h (ties averaged); it needs
            // R = 2 (a radius-1 table is never built for order 5)
            if constexpr (R >= 2) {
            auto L5 = [](int a, double sd) {
                double w = 1.0;
                for (int b = -2; b <= 2; b++)
                    if (b != a) w *= (sd - b) / (double)(a - b);
                return w;
            };
            auto lagE = [&](int cx, double wgt, double sx, double sy) {   // centred at cell (cx, 0)
                for (int b = -2; b <= 2; b++)
                    for (int a = -2; a <= 2; a++) e[k][b + R][cx + a + R] += wgt * L5(a, sx) * L5(b, sy);
            };
            auto lagN = [&](int cy, double wgt, double sx, double sy) {   // centred at cell (0, cy)
                for (int b = -2; b <= 2; b++)
                    for (int a = -2; a <= 2; a++) n[k][cy + b + R][a + R] += wgt * L5(a, sx) * L5(b, sy);
            };
            if (kx > 0) lagE(0, 1.0, 0.5 - h, -ky * h);
            else if (kx < 0) lagE(1, 1.0, h - 0.5, -ky * h);
            else { lagE(0, 0.5, 0.5, -ky * h); lagE(1, 0.5, -0.5, -ky * h); }
            if (ky > 0) lagN(0, 1.0, -kx * h, 0.5 - h);
            else if (ky < 0) lagN(1, 1.0, -kx * h, h - 0.5);
            else { lagN(0, 0.5, -kx * h, 0.5); lagN(1, 0.5, -kx * h, -0.5); }
            }
        } else if (flux == DUGKS_UPWIND) {
            if (kx > 0) addE(0, 1.0, 0.5 - h, -ky * h);
            else if (kx < 0) addE(1, 1.0, h - 0.5, -ky * h);
            else { addE(0, 0.5, 0.5, -ky * h); addE(1, 0.5, -0.5, -ky * h); }
            if (ky > 0) addN(0, 1.0, -kx * h, 0.5 - h);
            else if (ky < 0) addN(1, 1.0, -kx * h, h - 0.5);
            else { addN(0, 0.5, -kx * h, 0.5); addN(1, 0.5, -kx * h, -0.5); }
        } else {
            // east: (F_c + F_E)/2 - h [xi_x (F_E - F_c) + xi_y (dF/dy(c) + dF/dy(E))/2]
            e[k][R][R] += 0.5 + h * kx;
            e[k][R][R + 1] += 0.5 - h * kx;
            n[k][R][R] += 0.5 + h * ky;
            n[k][R + 1][R] += 0.5 - h * ky;
            for (int b = -R; b <= R; b++)
                for (int a = -R; a <= R; a++) {
                    e[k][b + R][a + R] += -0.5 * h * ky * gy(a, b);
                    e[k][b + R][a + R + 1] += -0.5 * h * ky * gy(a, b);
                    n[k][b + R][a + R] += -0.5 * h * kx * gx(a, b);
                    n[k][b + R + 1][a + R] += -0.5 * h * kx * gx(a, b);
                }
        }
    }
    FaceCoefs<T, R> cf;
    for (int k = 0; k < 9; k++) {
        for (int b = 0; b < NE; b++)
            for (int a = 0; a < NA; a++) cf.e[k][b][a] = (T)e[k][b][a];
        for (int b = 0; b < NA; b++)
            for (int a = 0; a < NA; a++) cf.n[k][b][a] = (T)n[k][b][a];
    }
    return cf;
}

template <typename T>
inline FaceCoefs<T> make_face_coefs(int order, int flux, double h) {
    return make_face_coefs_r<T, 1>(order, flux, h);
}

// ---- TMA tensor maps -----------------------------------------------------------
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    });
    return fn;
}

inline CUtensorMapDataType tma_type(size_t es, bool half) {
    if (half) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    return es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
}

// planes of `es`-byte elements at base: dims (pitch, ny + 2 GHOST[, nplanes]),
// box (bw, bh[, nplanes]); the fill of out-of-range elements is zero
inline bool encode_plane_map(CUtensorMap *m, void *base, size_t es, bool half, int pitch, int ny, size_t plane,
                             int nplanes, int bw, int bh) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)(ny + 2 * GHOST), (cuuint64_t)nplanes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)nplanes};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = nplanes > 1 ? 3 : 2;
    CUresult r = fn(m, tma_type(es, half), rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// host doubles (ny * nx, x fastest) -> device plane (double or float) with the
// periodic ghost border; synchronous
// A ny * nx field written into a ghost-bordered plane of (ny + 2 GHOST) rows of
// `pitch` elements of type O: the border holds the periodic images, the padding
// past nx + 2 GHOST is zero.
template <typename O>
inline void fill_ghosted_plane(O *pad, const double *src, int nx, int ny, int pitch) {
    const int G = GHOST;
    for (int y = -G; y < ny + G; y++) {
        const int sy = ((y % ny) + ny) % ny;
        const double *row = src + (size_t)sy * nx;
        O *out = pad + (size_t)(y + G) * pitch;
        for (int x = -G; x < 0; x++) out[x + G] = (O)row[((x % nx) + nx) % nx];
        for (int x = 0; x < nx; x++) out[x + G] = (O)row[x];
        for (int x = nx; x < nx + G; x++) out[x + G] = (O)row[x % nx];
        for (int x = nx + 2 * G; x < pitch; x++) out[x] = O(0);
    }
}

inline cudaError_t upload_ghosted_plane(void *dst, const double *src, int nx, int ny, int pitch, bool fp64) {
    const size_t n = (size_t)(ny + 2 * GHOST) * pitch;
    if (fp64) {
        std::vector<double> pad(n);
        fill_ghosted_plane(pad.data(), src, nx, ny, pitch);
        return cudaMemcpy(dst, pad.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    }
    std::vector<float> f(n);
    fill_ghosted_plane(f.data(), src, nx, ny, pitch);
    return cudaMemcpy(dst, f.data(), n * sizeof(float), cudaMemcpyHostToDevice);
}

}  // namespace host
}  // namespace dugks
