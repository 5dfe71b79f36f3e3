// dugks_api.cu -- the C ABI of libdugks.so (declared in include/dugks.h).
//
// Host logic only: parameter checks, the device memory of a context and its
// plane layout (ghost border of GHOST cells), TMA tensor maps, the per-step
// coefficients of the method, face-stencil coefficients, buffer rotation and
// error handling. All arithmetic of the time step runs in the kernels.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_dvm.cuh"
#include "dugks_host.h"
#include "dugks_internal.h"

using namespace dugks;
using namespace dugks::host;

struct dugks_ctx {
    dugks_params p{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int pitch = 0;
    size_t plane = 0;           // (ny + 2 GHOST) * pitch elements
    size_t tsize = 8, ssize = 8;
    int nsets = 2, nphi = 2;
    void *X[3] = {nullptr, nullptr, nullptr};
    void *phi[4] = {nullptr, nullptr, nullptr, nullptr};
    int cur = 0;                // current state set (two-stage)
    int pr[3] = {0, 1, 2};      // phi plane roles (see step_t2 / step_t3)
    void *phi0 = nullptr;       // initial phi (T, plane layout)
    void *ufield = nullptr, *vfield = nullptr;
    void *tmp = nullptr;        // ny * nx T, phi readout
    double *partial = nullptr;  // per-tile FP64 mass partials (scratch)
    double *dmass = nullptr;    // one double
    int *dstatus = nullptr;     // sticky device flags
    int tile_w = TILE_X, tile_h = TILE_Y, tiles_x = 0, ntiles = 0;
    // TMA-staged two-stage path (orders 2, 3)
    bool fast = false;
    int variant = 0;
    CUtensorMap tmX[2], tmPhi[4];
    double coef_h = -1.0;
    std::vector<unsigned char> coefs;   // FaceCoefs<T> of the current h
    double coef3_dt = -1.0;             // three-stage: FaceCoefs<T> at dt / 6 and 5 dt / 12
    std::vector<unsigned char> coefs3[2];
    int vel_kind = DUGKS_VEL_UNIFORM;
    double vel[4] = {0, 0, 0, 0};
    bool initialized = false;
    bool mass_valid = false;
    int64_t step = 0;
    int sticky = DUGKS_OK;
    std::string err;
};

namespace {

int fail(dugks_ctx *c, int code, const std::string &msg) {
    if (c) {
        if (c->sticky == DUGKS_OK) c->sticky = code;
        c->err = msg;
    }
    return code;
}

int cuda_fail(dugks_ctx *c, cudaError_t e, const char *where) {
    return fail(c, DUGKS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_fp64(const dugks_ctx *c) { return c->p.precision == DUGKS_FP64; }

int check_params(const dugks_params *p, std::string &why) {
    if (!p) { why = "params is NULL"; return DUGKS_EINVAL; }
    if (p->nx < 8 || p->ny < 8) { why = "nx and ny must be >= 8"; return DUGKS_EINVAL; }
    if ((int64_t)(p->nx + 2 * GHOST + 32) * (p->ny + 2 * GHOST) > (int64_t)1 << 31) { why = "grid too large"; return DUGKS_EINVAL; }
    if (!(p->W > 0) || !(p->M > 0)) { why = "W and M must be > 0"; return DUGKS_EINVAL; }
    if (!(p->cfl > 0) || p->cfl > 1.0) { why = "cfl must be in (0, 1]"; return DUGKS_EINVAL; }
    if (p->order < 2 || p->order > 5) { why = "order must be 2, 3, 4 or 5"; return DUGKS_EINVAL; }
    if (p->order == 5 && (p->flux != DUGKS_UPWIND || p->stages != 2)) {
        why = "order 5 (DUGKS-T2S5) is two-stage with upwind faces";
        return DUGKS_EINVAL;
    }
    if (p->flux != DUGKS_UPWIND && p->flux != DUGKS_CENTRAL) { why = "flux must be upwind or central"; return DUGKS_EINVAL; }
    if (p->stages < 1 || p->stages > 3) { why = "stages must be 1 (DVM), 2 or 3"; return DUGKS_EINVAL; }
    if (p->precision < DUGKS_FP64 || p->precision > DUGKS_FP16F) { why = "unknown precision"; return DUGKS_EINVAL; }
    if (p->precision == DUGKS_FP16F && p->stages != 2) { why = "FP16 storage is two-stage only"; return DUGKS_EINVAL; }
    if (!(p->phiA != p->phiB) || !std::isfinite(p->phiA) || !std::isfinite(p->phiB)) { why = "phiA must differ from phiB"; return DUGKS_EINVAL; }
    if (p->stages == 3 && !(p->cfl < 12.0 * 3.0 * p->M)) {
        why = "three-stage DUGKS needs dt < 12 tau = 36 M";
        return DUGKS_EINVAL;
    }
    return DUGKS_OK;
}

template <typename T>
StepParams<T> base_params(const dugks_ctx *c) {
    StepParams<T> q;
    std::memset(&q, 0, sizeof q);
    q.nx = c->p.nx;
    q.ny = c->p.ny;
    q.pitch = c->pitch;
    q.plane = c->plane;
    q.status = c->dstatus;
    q.tiles_x = c->tiles_x;
    q.tile_w = c->tile_w;
    q.tile_h = c->tile_h;
    q.ufield = static_cast<const T *>(c->ufield);
    q.vfield = static_cast<const T *>(c->vfield);
    const double tau = 3.0 * c->p.M;
    q.tau = (T)tau;
    q.theta_c = (T)(-4.0 / (c->p.W * (c->p.phiA - c->p.phiB)));
    q.phiA = (T)c->p.phiA;
    q.phiB = (T)c->p.phiB;
    q.vel_kind = c->vel_kind;
    q.vp0 = (T)c->vel[0];
    q.vp1 = (T)c->vel[1];
    q.vp2 = (T)c->vel[2];
    q.qscale = (T)256.0;
    q.qinv = (T)(1.0 / 256.0);
    return q;
}

// f_b = (2 tau bar f + h f^eq + tau h S) / (2 tau + h)        (Eq. (27))
template <typename T>
void face_coefs(StepParams<T> &q, double tau, double h) {
    q.h = (T)h;
    q.c1 = (T)(2.0 * tau / (2.0 * tau + h));
    q.c2 = (T)(h / (2.0 * tau + h));
    q.c3 = (T)(tau * h / (2.0 * tau + h));
}

bool encode_map(CUtensorMap *m, void *base, size_t es, bool half, const dugks_ctx *c, int nplanes, int bw, int bh) {
    return encode_plane_map(m, base, es, half, c->pitch, c->p.ny, c->plane, nplanes, bw, bh);
}

template <typename T, typename ST>
bool setup_fast(dugks_ctx *c) {
    const FastGeom g = Launch<T, ST>::fast_geom(c->variant, c->p.order, c->p.stages);
    const bool half = Store<T, ST>::deviation;
    for (int s = 0; s < 2; s++)
        if (!encode_map(&c->tmX[s], c->X[s], sizeof(ST), half, c, 9, g.box_w, g.box_h)) return false;
    for (int s = 0; s < c->nphi; s++)
        if (!encode_map(&c->tmPhi[s], c->phi[s], sizeof(T), false, c, 1, g.box_wt, g.box_h)) return false;
    c->tile_w = g.tile_w;
    c->tile_h = g.tile_h;
    return true;
}

template <typename T, typename ST>
int run_init(dugks_ctx *c) {
    StepParams<T> q = base_params<T>(c);
    q.t = (T)0;
    // tilde f = f - (dt/2)(Omega + S), hat f = f - (dt/4)(Omega + S); the DVM's
    // tilde f^+ = f + (dt/2)(Omega + S) (Eq. (9)); Omega = 0 at the start
    const double frac = c->p.stages == 2 ? 0.5 : c->p.stages == 3 ? 0.25 : -0.5;
    if (Store<T, ST>::phi_plane) {
        c->pr[0] = 0; c->pr[1] = 1; c->pr[2] = 2;
    }
    q.out1 = c->p.stages == 3 ? c->X[0] : c->X[c->cur];
    // a phi plane: phi of the state; otherwise phi0 as the previous level
    q.phi_out = static_cast<T *>(c->phi[c->pr[0]]);
    // (the initial source takes the gradient of the order; order 5 has the fourth-order one)
    cudaError_t e = Launch<T, ST>::init(q, static_cast<const T *>(c->phi0), (T)(frac * c->p.cfl),
                                        c->p.order == 5 ? 4 : c->p.order, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    c->initialized = true;
    c->mass_valid = false;
    return DUGKS_OK;
}

int ensure_init(dugks_ctx *c) {
    if (c->initialized) return DUGKS_OK;
    switch (c->p.precision) {
    case DUGKS_FP64: return run_init<double, double>(c);
    case DUGKS_FP32: return run_init<float, float>(c);
    default: return run_init<float, __half>(c);
    }
}

// Reversal factors cos(pi t / T) of the single vortex and of the deformation at
// the cell time, the older time of d(phi u)/dt and the face time (FP64 on the
// host); zero for other velocities.
template <typename T>
FastExtra<T> vortex_factors(const dugks_ctx *c, double t, double t_old, double t_face) {
    FastExtra<T> fx{};
    if (c->vel_kind == DUGKS_VEL_VORTEX || c->vel_kind == DUGKS_VEL_DEFORM) {
        const double PI = 3.14159265358979323846, Tp = c->vel[2];
        fx.vc_t = (T)std::cos(PI * t / Tp);
        fx.vc_told = (T)std::cos(PI * t_old / Tp);
        fx.vc_tface = (T)std::cos(PI * t_face / Tp);
    }
    return fx;
}

// One two-stage step, X[cur] -> X[1-cur]. phi as a sum of X (FP64): phi[pr0]
// holds phi^{n-1}, phi[pr1] receives phi^n. phi as a plane of its own (FP32,
// FP16F): phi[pr0] = phi^n (of X), phi[pr1] = phi^{n-1}, phi[pr2] receives phi^{n+1}.
// dbg (debug read-out): the generic kernel evaluates the step of the current state,
// writes its face values to dbg and its results only to scratch planes (the next
// state set and phi plane, no mass partials); the context does not advance.
template <typename T, typename ST>
int step_t2(dugks_ctx *c, double *dbg = nullptr) {
    StepParams<T> q = base_params<T>(c);
    const double dt = c->p.cfl, tau = 3.0 * c->p.M, h = 0.5 * dt;
    const double a = (2.0 * tau - h) / (2.0 * tau + dt), b = (dt + h) / (2.0 * tau + dt);
    const double t = (double)c->step * dt;
    q.a = (T)a;
    q.b = (T)b;
    face_coefs(q, tau, h);
    // tilde f^{n+1} = (4/3) bar f^+ - (1/3) tilde f + dt L = X + (4b/3)(g - X) + dt L
    q.al1 = (T)(4.0 / 3.0 * a - 1.0 / 3.0);
    q.be1 = (T)(4.0 / 3.0 * b);
    q.ga1 = (T)dt;
    q.t = (T)t;
    q.t_old = (T)(t - dt);
    q.t_face = (T)(t + h);
    q.seed = (uint32_t)c->step;
    q.useD = (c->p.dtphiu && c->step > 0) ? 1 : 0;
    q.inv_dtD = (T)(1.0 / dt);
    q.X = c->X[c->cur];
    q.out1 = c->X[1 - c->cur];
    q.mass_partial = c->partial;
    int iPc = 0, iPo, iOut;
    if (Store<T, ST>::phi_plane) {
        iPc = c->pr[0]; iPo = c->pr[1]; iOut = c->pr[2];
        q.phi_cur = static_cast<const T *>(c->phi[iPc]);
    } else {
        iPo = c->pr[0]; iOut = c->pr[1];
    }
    q.phi_old = static_cast<const T *>(c->phi[iPo]);
    q.phi_out = static_cast<T *>(c->phi[iOut]);
    cudaError_t e;
    if (dbg != nullptr) {
        q.dbg = dbg;
        q.mass_partial = nullptr;
        e = Launch<T, ST>::step(q, c->p.order, c->p.flux, KIND_T2, c->stream);
        return e == cudaSuccess ? DUGKS_OK : cuda_fail(c, e, "debug step kernel");
    }
    if (c->fast && c->p.order >= 4) {
        if (c->coef_h != h) {
            // (order 4: the Taylor stencils; order 5: the Lagrange ones)
            const FaceCoefs<T, 2> cf = make_face_coefs_r<T, 2>(c->p.order, c->p.flux, h);
            c->coefs.assign(reinterpret_cast<const unsigned char *>(&cf),
                            reinterpret_cast<const unsigned char *>(&cf) + sizeof cf);
            c->coef_h = h;
        }
        e = Launch<T, ST>::step_fast4(q, *reinterpret_cast<const FaceCoefs<T, 2> *>(c->coefs.data()),
                                      vortex_factors<T>(c, t, t - dt, t + h), c->tmX[c->cur], c->tmPhi[iPo],
                                      c->tmPhi[iPc], c->p.flux, KIND_T2, c->stream);
    } else if (c->fast) {
        if (c->coef_h != h) {
            FaceCoefs<T> cf = make_face_coefs<T>(c->p.order, c->p.flux, h);
            c->coefs.assign(reinterpret_cast<unsigned char *>(&cf), reinterpret_cast<unsigned char *>(&cf) + sizeof cf);
            c->coef_h = h;
        }
        const FaceCoefs<T> &cf = *reinterpret_cast<const FaceCoefs<T> *>(c->coefs.data());
        const FastExtra<T> fx = vortex_factors<T>(c, t, t - dt, t + h);
        e = Launch<T, ST>::step_fast(q, cf, fx, c->tmX[c->cur], c->tmPhi[iPo], c->tmPhi[iPc], c->p.order,
                                     c->p.flux, c->variant, c->stream);
    } else {
        if (c->p.order == 5) return fail(c, DUGKS_EINVAL, "order 5 needs the TMA-staged kernels");
        e = Launch<T, ST>::step(q, c->p.order, c->p.flux, KIND_T2, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
    c->cur = 1 - c->cur;
    if (Store<T, ST>::phi_plane) {
        const int a0 = c->pr[0], a1 = c->pr[1], a2 = c->pr[2];
        c->pr[0] = a2; c->pr[1] = a0; c->pr[2] = a1;
    } else {
        std::swap(c->pr[0], c->pr[1]);
    }
    return DUGKS_OK;
}

// One three-stage step (Sec. II.B.2): X[0] = hat f, X[1] = tilde f at t',
// X[2] = accumulator f^n + (3 dt / 7) L*.
template <typename T>
int step_t3(dugks_ctx *c) {
    constexpr bool PHIP = Store<T, T>::phi_plane;
    const double dt = c->p.cfl, tau = 3.0 * c->p.M;
    const double t = (double)c->step * dt;
    // (i)-(ii): bar f^{+, dt/6} (Eq. (31)), flux at t_n + dt/6, tilde f(t') and accumulator
    StepParams<T> A = base_params<T>(c);
    const double a1 = (12.0 * tau - dt) / (12.0 * tau + 3.0 * dt), b1 = 4.0 * dt / (12.0 * tau + 3.0 * dt);
    A.a = (T)a1;
    A.b = (T)b1;
    face_coefs(A, tau, dt / 6.0);
    A.al1 = (T)(1.25 * a1 - 0.25);   // tilde f^+ = (5/4) A - (1/4) hat f   (Eq. (33))
    A.be1 = (T)(1.25 * b1);
    A.ga1 = (T)(dt / 3.0);           // Eq. (15)
    A.al2 = (T)(0.75 * a1 + 0.25);   // f^n = (3/4) A + (1/4) hat f         (Eq. (32))
    A.be2 = (T)(0.75 * b1);
    A.ga2 = (T)(3.0 * dt / 7.0);     // Eq. (16)
    A.t = (T)t;
    A.t_old = (T)(t - dt);
    A.t_face = (T)(t + dt / 6.0);
    A.useD = (c->p.dtphiu && c->step > 0) ? 1 : 0;
    A.inv_dtD = (T)(1.0 / dt);
    A.X = c->X[0];
    A.out1 = c->X[1];
    A.out2 = static_cast<T *>(c->X[2]);
    A.seed = (uint32_t)(2 * c->step);
    // phi planes (FP32): pr0 = phi^n (of X), pr1 = phi^{n-1}; plane 2 receives phi of
    // tilde f', plane 3 phi of the accumulator, and kernel B writes phi^{n+1} over
    // pr1. Otherwise (FP64): pr0 = phi^{n-1}; kernel A writes phi^n to pr1.
    int aPo = c->pr[0], aPc = c->pr[0], bPo = c->pr[1], bPc = c->pr[1];
    if (PHIP) {
        aPc = c->pr[0];
        aPo = c->pr[1];
        bPc = 2;
        bPo = c->pr[0];
        A.phi_cur = static_cast<const T *>(c->phi[aPc]);
        A.phi_out = static_cast<T *>(c->phi[2]);
        A.phi_out2 = static_cast<T *>(c->phi[3]);
    } else {
        A.phi_out = static_cast<T *>(c->phi[c->pr[1]]);
    }
    A.phi_old = static_cast<const T *>(c->phi[aPo]);
    cudaError_t e;
    if (c->fast && c->coef3_dt != dt) {
        auto keep = [](std::vector<unsigned char> &v, const auto &cf) {
            v.assign(reinterpret_cast<const unsigned char *>(&cf), reinterpret_cast<const unsigned char *>(&cf) + sizeof cf);
        };
        if (c->p.order == 4) {
            keep(c->coefs3[0], make_face_coefs_r<T, 2>(4, c->p.flux, dt / 6.0));
            keep(c->coefs3[1], make_face_coefs_r<T, 2>(4, c->p.flux, 5.0 * dt / 12.0));
        } else {
            keep(c->coefs3[0], make_face_coefs<T>(c->p.order, c->p.flux, dt / 6.0));
            keep(c->coefs3[1], make_face_coefs<T>(c->p.order, c->p.flux, 5.0 * dt / 12.0));
        }
        c->coef3_dt = dt;
    }
    if (c->fast && c->p.order >= 4) {
        e = Launch<T, T>::step_fast4(A, *reinterpret_cast<const FaceCoefs<T, 2> *>(c->coefs3[0].data()),
                                     vortex_factors<T>(c, t, t - dt, t + dt / 6.0), c->tmX[0], c->tmPhi[aPo],
                                     c->tmPhi[aPc], c->p.flux, KIND_T3A, c->stream);
    } else if (c->fast) {
        const FaceCoefs<T> &cf = *reinterpret_cast<const FaceCoefs<T> *>(c->coefs3[0].data());
        e = Launch<T, T>::step_fast3(A, cf, vortex_factors<T>(c, t, t - dt, t + dt / 6.0), c->tmX[0],
                                     c->tmPhi[aPo], c->tmPhi[aPc], c->p.order, c->p.flux, KIND_T3A, c->stream);
    } else {
        e = Launch<T, T>::step(A, c->p.order, c->p.flux, KIND_T3A, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "three-stage kernel A");
    // (iii)-(iv): bar f^{+, 5dt/12}(t') (Eq. (34)), flux at t_n + 3dt/4, hat f^{n+1}
    StepParams<T> B = base_params<T>(c);
    const double a2 = (24.0 * tau - 5.0 * dt) / (24.0 * tau + 4.0 * dt), b2 = 9.0 * dt / (24.0 * tau + 4.0 * dt);
    const double cos_ = -6.0 / (6.0 * tau + dt);   // Eq. (29), stray dt read as a typo
    B.a = (T)a2;
    B.b = (T)b2;
    face_coefs(B, tau, 5.0 * dt / 12.0);
    B.al1 = (T)(0.75 * dt * cos_);
    B.be1 = (T)(-0.75 * dt * cos_);
    B.ga1 = (T)(4.0 * dt / 7.0);
    B.t = (T)(t + dt / 3.0);
    B.t_old = (T)t;
    B.t_face = (T)(t + 0.75 * dt);
    B.useD = c->p.dtphiu ? 1 : 0;
    B.inv_dtD = (T)(3.0 / dt);
    B.X = c->X[1];
    B.acc = c->X[2];
    B.out1 = c->X[0];
    B.seed = (uint32_t)(2 * c->step + 1);
    B.phi_old = static_cast<const T *>(c->phi[bPo]);
    if (PHIP) {
        B.phi_cur = static_cast<const T *>(c->phi[bPc]);
        B.phi_acc = static_cast<const T *>(c->phi[3]);
        B.phi_out = static_cast<T *>(c->phi[c->pr[1]]);
    }
    B.mass_partial = c->partial;
    if (c->fast && c->p.order >= 4) {
        e = Launch<T, T>::step_fast4(B, *reinterpret_cast<const FaceCoefs<T, 2> *>(c->coefs3[1].data()),
                                     vortex_factors<T>(c, t + dt / 3.0, t, t + 0.75 * dt), c->tmX[1],
                                     c->tmPhi[bPo], c->tmPhi[bPc], c->p.flux, KIND_T3B, c->stream);
    } else if (c->fast) {
        const FaceCoefs<T> &cf = *reinterpret_cast<const FaceCoefs<T> *>(c->coefs3[1].data());
        e = Launch<T, T>::step_fast3(B, cf, vortex_factors<T>(c, t + dt / 3.0, t, t + 0.75 * dt), c->tmX[1],
                                     c->tmPhi[bPo], c->tmPhi[bPc], c->p.order, c->p.flux, KIND_T3B, c->stream);
    } else {
        e = Launch<T, T>::step(B, c->p.order, c->p.flux, KIND_T3B, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "three-stage kernel B");
    std::swap(c->pr[0], c->pr[1]);
    return DUGKS_OK;
}

// One step of the streaming-collision DVM (Sec. II.B.1; the LBM at dt = 1):
// X[cur] -> X[1-cur]. phi as a sum of X (FP64): phi[pr0] holds phi^n (of X),
// phi[pr1] receives phi^{n+1}. phi as a plane of its own (FP32): phi[pr0] = phi^n,
// phi[pr2] receives phi^{n+1}, the roles rotating as in step_t2.
template <typename T>
int step_dvm(dugks_ctx *c) {
    constexpr bool PHIP = Store<T, T>::phi_plane;
    StepParams<T> q = base_params<T>(c);
    const double dt = c->p.cfl, tau = 3.0 * c->p.M, t = (double)c->step * dt;
    q.t_old = (T)t;          // time of the state and of phi_old
    q.t = (T)(t + dt);       // time of the new cell quantities
    q.inv_dtD = (T)(1.0 / dt);
    q.useD = c->p.dtphiu ? 1 : 0;
    q.X = c->X[c->cur];
    q.out1 = c->X[1 - c->cur];
    q.mass_partial = c->partial;
    q.phi_old = static_cast<const T *>(c->phi[c->pr[0]]);
    q.phi_out = static_cast<T *>(c->phi[PHIP ? c->pr[2] : c->pr[1]]);
    DvmExtra<T> dv;
    dv.s = dt >= 0.5 ? 1 : 0;
    dv.d = (T)(dv.s - dt);
    dv.beta = (T)(2.0 * dt / (2.0 * tau + dt));
    cudaError_t e = launch_dvm<T>(q, dv, c->p.order, dt == 1.0, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "DVM kernel");
    c->cur = 1 - c->cur;
    if (PHIP) {
        const int a0 = c->pr[0], a1 = c->pr[1], a2 = c->pr[2];
        c->pr[0] = a2; c->pr[1] = a0; c->pr[2] = a1;
    } else {
        std::swap(c->pr[0], c->pr[1]);
    }
    return DUGKS_OK;
}

int step_once(dugks_ctx *c) {
    int r;
    if (c->p.stages == 1) {
        r = is_fp64(c) ? step_dvm<double>(c) : step_dvm<float>(c);
    } else if (c->p.stages == 3) {
        r = is_fp64(c) ? step_t3<double>(c) : step_t3<float>(c);
    } else {
        switch (c->p.precision) {
        case DUGKS_FP64: r = step_t2<double, double>(c); break;
        case DUGKS_FP32: r = step_t2<float, float>(c); break;
        default: r = step_t2<float, __half>(c); break;
        }
    }
    if (r == DUGKS_OK) {
        c->step++;
        c->mass_valid = true;
    }
    return r;
}

template <typename T, typename ST>
StepParams<T> state_view(const dugks_ctx *c) {
    StepParams<T> q = base_params<T>(c);
    q.X = c->p.stages == 3 ? c->X[0] : c->X[c->cur];
    if (Store<T, ST>::phi_plane) q.phi_cur = static_cast<const T *>(c->phi[c->pr[0]]);
    q.mass_partial = c->partial;
    return q;
}

int enqueue_mass(dugks_ctx *c, double *dev_out) {
    cudaError_t e;
    if (!c->mass_valid) {
        switch (c->p.precision) {
        case DUGKS_FP64: e = Launch<double, double>::mass_partial(state_view<double, double>(c), c->stream); break;
        case DUGKS_FP32: e = Launch<float, float>::mass_partial(state_view<float, float>(c), c->stream); break;
        default: e = Launch<float, __half>::mass_partial(state_view<float, __half>(c), c->stream); break;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "mass partial kernel");
        c->mass_valid = true;
    }
    e = launch_mass_final(c->partial, c->ntiles, dev_out, c->dstatus, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "mass kernel");
    return DUGKS_OK;
}

int enqueue_phi(dugks_ctx *c, void *dev_out) {
    cudaError_t e;
    switch (c->p.precision) {
    case DUGKS_FP64: e = Launch<double, double>::phi(state_view<double, double>(c), static_cast<double *>(dev_out), c->stream); break;
    case DUGKS_FP32: e = Launch<float, float>::phi(state_view<float, float>(c), static_cast<float *>(dev_out), c->stream); break;
    default: e = Launch<float, __half>::phi(state_view<float, __half>(c), static_cast<float *>(dev_out), c->stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "phi kernel");
    return DUGKS_OK;
}

int sync_ctx(dugks_ctx *c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    return c->sticky;
}

void free_ctx(dugks_ctx *c) {
    for (void *q : {c->X[0], c->X[1], c->X[2], c->phi[0], c->phi[1], c->phi[2], c->phi[3], c->phi0, c->ufield,
                    c->vfield, c->tmp, (void *)c->partial, (void *)c->dmass, (void *)c->dstatus})
        if (q) cudaFree(q);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// host doubles (ny * nx, x fastest) -> device plane of T with the periodic ghost border
int upload_plane(dugks_ctx *c, void *dst, const double *src) {
    cudaError_t e = upload_ghosted_plane(dst, src, c->p.nx, c->p.ny, c->pitch, is_fp64(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "upload");
    return DUGKS_OK;
}

}  // namespace

namespace dugks {
// allocation test hook: the next g_alloc_skip allocations proceed, the g_alloc_fail
// after them fail
static std::atomic<int> g_alloc_skip{0}, g_alloc_fail{0};

static bool alloc_hook_fails() {
    if (g_alloc_fail.load(std::memory_order_relaxed) > 0) {
        if (g_alloc_skip.fetch_sub(1, std::memory_order_relaxed) <= 0) {
            g_alloc_skip.store(0, std::memory_order_relaxed);
            g_alloc_fail.fetch_sub(1, std::memory_order_relaxed);
            return true;
        }
    }
    return false;
}

cudaError_t dev_malloc_raw(void **p, size_t bytes) {
    if (alloc_hook_fails()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_pool(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t s) {
    if (alloc_hook_fails()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// Fixed-order sum of the per-tile partials (deterministic); flags NaN / Inf.
// Thread t adds partials t, t + 256, ... in index order with 8 independent loads
// in flight (one memory latency per 8 partials), then the fixed tree of block_sum.
// One small CTA: it finds a free slot while the step kernel drains.
__global__ void __launch_bounds__(256) mass_final_kernel(const double *partial, int n, double *out, int *status) {
    __shared__ double sred[32];
    pdl_trigger();
    pdl_wait();   // the partials of the step kernel ahead of it
    constexpr int U = 8;
    double s = 0.0;
    for (int base = threadIdx.x; base < n; base += U * 256) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; u++) v[u] = base + u * 256 < n ? partial[base + u * 256] : 0.0;
#pragma unroll
        for (int u = 0; u < U; u++) s += v[u];
    }
    s = block_sum(s, sred);
    if (threadIdx.x == 0) {
        *out = s;
        if (!isfinite(s)) atomicOr(status, 1);
    }
}

cudaError_t launch_mass_final(const double *partial, int n, double *out, int *status, cudaStream_t s) {
    // programmatic dependent launch: resident while the step kernel drains, it
    // waits for the partials in the kernel itself
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, mass_final_kernel, partial, n, out, status);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
}  // namespace dugks

extern "C" {

int dugks_create(const dugks_params *p, const double *phi0_host, void *cuda_stream, dugks_ctx **out) {
    if (!out) return DUGKS_EINVAL;
    *out = nullptr;
    std::string why;
    int r = check_params(p, why);
    if (r != DUGKS_OK) return r;
    if (!phi0_host) return DUGKS_EINVAL;
    for (size_t i = 0; i < (size_t)p->nx * p->ny; i++)
        if (!std::isfinite(phi0_host[i])) return DUGKS_ENONFINITE;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DUGKS_ECUDA;
    }
    dugks_ctx *c = new dugks_ctx();
    c->p = *p;
    cudaGetDevice(&c->dev);
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            free_ctx(c);
            return DUGKS_ECUDA;
        }
        c->own_stream = true;
    }
    c->tsize = is_fp64(c) ? 8 : 4;
    c->ssize = p->precision == DUGKS_FP64 ? 8 : p->precision == DUGKS_FP32 ? 4 : 2;
    c->pitch = (p->nx + 2 * GHOST + 31) / 32 * 32;
    c->plane = (size_t)(p->ny + 2 * GHOST) * c->pitch;
    c->nsets = p->stages == 3 ? 3 : 2;
    // FP32 and FP16F keep phi as a plane of its own: three rotating roles (two-stage), or
    // the state's and the previous level's plus phi of tilde f' and of the accumulator
    // (three-stage); FP64: the previous level for d(phi u)/dt (and phi^n, three-stage)
    c->nphi = p->precision == DUGKS_FP64 ? 2 : p->stages == 3 ? 4 : 3;
    // the TMA-staged kernels serve every order and both schemes (three-stage: full
    // storage; orders 4-5 and the three-stage scheme: one tile shape each)
    // (the DVM has one kernel of its own)
    c->fast = p->stages != 1 && (p->stages == 2 || p->precision != DUGKS_FP16F) && encode_fn() != nullptr;
    if (c->fast && (p->stages == 3 || p->order >= 4)) {
        c->variant = 2;
    } else if (c->fast) {
        // measured (FP32, L2 flushed between steps): 8 warps x 2 rows per thread fastest
        // on grids that fill about one wave of tiles (256^2), 8 x 3 from 1024^2 up
        c->variant = (int64_t)p->nx * p->ny >= 512 * 512 ? 4 : 2;
        // tuning override: DUGKS_FAST_VARIANT = 0..FAST_VARIANTS-1
        if (const char *ev = std::getenv("DUGKS_FAST_VARIANT")) {
            const int v = std::atoi(ev);
            if (v >= 0 && v < FAST_VARIANTS) c->variant = v;
        }
    }
    bool ok = true;
    for (int s = 0; s < c->nsets && ok; s++) {
        // the three-stage accumulator (set 2) is always in the arithmetic type
        size_t es = (p->stages == 3) ? c->tsize : c->ssize;
        ok = dev_malloc(&c->X[s], 9 * c->plane * es) == cudaSuccess;
    }
    for (int s = 0; s < c->nphi && ok; s++) ok = dev_malloc(&c->phi[s], c->plane * c->tsize) == cudaSuccess;
    if (ok) ok = dev_malloc(&c->phi0, c->plane * c->tsize) == cudaSuccess;
    if (ok) ok = dev_malloc(&c->tmp, (size_t)p->nx * p->ny * sizeof(double)) == cudaSuccess;
    if (ok) ok = dev_malloc(&c->dmass, sizeof(double)) == cudaSuccess;
    if (ok) ok = dev_malloc(&c->dstatus, sizeof(int)) == cudaSuccess;
    if (ok && c->fast) {
        bool enc = p->precision == DUGKS_FP64 ? setup_fast<double, double>(c)
                   : p->precision == DUGKS_FP32 ? setup_fast<float, float>(c)
                                                : setup_fast<float, __half>(c);
        if (!enc) {   // use the generic CUDA kernel instead
            c->fast = false;
            c->tile_w = TILE_X;
            c->tile_h = TILE_Y;
        }
    }
    c->tiles_x = (p->nx + c->tile_w - 1) / c->tile_w;
    c->ntiles = c->tiles_x * ((p->ny + c->tile_h - 1) / c->tile_h);
    if (ok) ok = dev_malloc(&c->partial, (size_t)c->ntiles * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        return DUGKS_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream);
    // zero everything so raw checkpoints and the pitch padding are deterministic
    for (int s = 0; s < c->nsets && e == cudaSuccess; s++)
        e = cudaMemsetAsync(c->X[s], 0, 9 * c->plane * ((p->stages == 3) ? c->tsize : c->ssize), c->stream);
    for (int s = 0; s < c->nphi && e == cudaSuccess; s++) e = cudaMemsetAsync(c->phi[s], 0, c->plane * c->tsize, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_ctx(c);
        return DUGKS_ECUDA;
    }
    r = upload_plane(c, c->phi0, phi0_host);
    if (r == DUGKS_OK) r = sync_ctx(c);
    if (r != DUGKS_OK) {
        free_ctx(c);
        return r;
    }
    *out = c;
    return DUGKS_OK;
}

int dugks_set_velocity(dugks_ctx *c, int kind, const double *params, const double *u_host, const double *v_host) {
    if (!c) return DUGKS_EINVAL;
    cudaSetDevice(c->dev);
    double v[4] = {0, 0, 0, 0};
    switch (kind) {
    case DUGKS_VEL_UNIFORM:
        if (!params) return fail(c, DUGKS_EINVAL, "uniform velocity needs (ux, uy)");
        v[0] = params[0]; v[1] = params[1];
        break;
    case DUGKS_VEL_ROTATION:
        if (!params) return fail(c, DUGKS_EINVAL, "rotation needs (cx, cy, omega)");
        v[0] = params[0]; v[1] = params[1]; v[2] = params[2];
        break;
    case DUGKS_VEL_VORTEX:
        if (!params || !(params[0] > 0) || !(params[2] > 0)) return fail(c, DUGKS_EINVAL, "vortex needs (L > 0, U, T > 0)");
        v[0] = params[0]; v[1] = params[1]; v[2] = params[2];
        break;
    case DUGKS_VEL_DEFORM:
        if (!params || !(params[0] > 0) || !(params[2] > 0))
            return fail(c, DUGKS_EINVAL, "deformation needs (L > 0, U, T > 0)");
        v[0] = params[0]; v[1] = params[1]; v[2] = params[2];
        break;
    case DUGKS_VEL_FIELD: {
        if (!u_host || !v_host) return fail(c, DUGKS_EINVAL, "field velocity needs u and v arrays");
        for (size_t i = 0; i < (size_t)c->p.nx * c->p.ny; i++)
            if (!std::isfinite(u_host[i]) || !std::isfinite(v_host[i]))
                return fail(c, DUGKS_EINVAL, "velocity field must be finite");
        cudaStreamSynchronize(c->stream);   // the field may be in use by queued steps
        if (!c->ufield) {
            if (dev_malloc(&c->ufield, c->plane * c->tsize) != cudaSuccess ||
                dev_malloc(&c->vfield, c->plane * c->tsize) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, DUGKS_ENOMEM, "velocity field allocation");
            }
        }
        int r = upload_plane(c, c->ufield, u_host);
        if (r == DUGKS_OK) r = upload_plane(c, c->vfield, v_host);
        if (r != DUGKS_OK) return r;
        break;
    }
    default:
        return fail(c, DUGKS_EINVAL, "unknown velocity kind");
    }
    for (int i = 0; i < 4; i++)
        if (!std::isfinite(v[i])) return fail(c, DUGKS_EINVAL, "velocity parameters must be finite");
    c->vel_kind = kind;
    std::memcpy(c->vel, v, sizeof v);
    if (c->step == 0) c->initialized = false;   // the initial equilibrium depends on u(0)
    return DUGKS_OK;
}

int dugks_step(dugks_ctx *c, int64_t nsteps) {
    if (!c || nsteps < 0) return c ? fail(c, DUGKS_EINVAL, "nsteps < 0") : DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    cudaSetDevice(c->dev);
    int r = ensure_init(c);
    for (int64_t s = 0; s < nsteps && r == DUGKS_OK; s++) r = step_once(c);
    return r;
}

int dugks_read_phi_device(dugks_ctx *c, void *dev_out) {
    if (!c || !dev_out) return DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    cudaSetDevice(c->dev);
    int r = ensure_init(c);
    if (r == DUGKS_OK) r = enqueue_phi(c, dev_out);
    return r;
}

int dugks_read_phi(dugks_ctx *c, double *out_host) {
    if (!c || !out_host) return DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    cudaSetDevice(c->dev);
    int r = ensure_init(c);
    if (r != DUGKS_OK) return r;
    // phi widened to double on the device, then one copy into the caller's buffer
    // (at full link speed when that buffer is pinned)
    cudaError_t e;
    switch (c->p.precision) {
    case DUGKS_FP64: e = Launch<double, double>::phi64(state_view<double, double>(c), static_cast<double *>(c->tmp), c->stream); break;
    case DUGKS_FP32: e = Launch<float, float>::phi64(state_view<float, float>(c), static_cast<double *>(c->tmp), c->stream); break;
    default: e = Launch<float, __half>::phi64(state_view<float, __half>(c), static_cast<double *>(c->tmp), c->stream); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "phi kernel");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    e = cudaMemcpyAsync(out_host, c->tmp, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read phi");
    return sync_ctx(c);
}

int dugks_debug_faces(dugks_ctx *c, double *fbar_E, double *fbar_N, double *f_E, double *f_N) {
    // (argument errors leave the context usable: they are not sticky)
    if (!c || !fbar_E || !fbar_N || !f_E || !f_N) return DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    if (c->p.stages != 2 || c->p.order == 5) {
        c->err = "face read-out serves the two-stage scheme at orders 2-4";
        return DUGKS_EINVAL;
    }
    cudaSetDevice(c->dev);
    int r = ensure_init(c);
    if (r != DUGKS_OK) return r;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    double *d = nullptr;
    if (dev_malloc(&d, 4 * 9 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "face read-out buffer";
        return DUGKS_ENOMEM;
    }
    switch (c->p.precision) {
    case DUGKS_FP64: r = step_t2<double, double>(c, d); break;
    case DUGKS_FP32: r = step_t2<float, float>(c, d); break;
    default: r = step_t2<float, __half>(c, d); break;
    }
    double *outs[4] = {fbar_E, fbar_N, f_E, f_N};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && r == DUGKS_OK && e == cudaSuccess; i++)
        e = cudaMemcpyAsync(outs[i], d + (size_t)i * 9 * n, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (r == DUGKS_OK && e == cudaSuccess) r = sync_ctx(c);
    else if (r == DUGKS_OK) r = cuda_fail(c, e, "face read-out copy");
    cudaStreamSynchronize(c->stream);
    cudaFree(d);
    return r;
}

int dugks_mass_device(dugks_ctx *c, double *dev_out) {
    if (!c || !dev_out) return DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    cudaSetDevice(c->dev);
    int r = ensure_init(c);
    if (r == DUGKS_OK) r = enqueue_mass(c, dev_out);
    return r;
}

int dugks_mass(dugks_ctx *c, double *out) {
    if (!c || !out) return DUGKS_EINVAL;
    int r = dugks_mass_device(c, c->dmass);
    if (r != DUGKS_OK) return r;
    cudaError_t e = cudaMemcpyAsync(out, c->dmass, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read mass");
    r = sync_ctx(c);
    if (r != DUGKS_OK) return r;
    if (!std::isfinite(*out)) return fail(c, DUGKS_ENONFINITE, "the field holds NaN or Inf");
    return DUGKS_OK;
}

int dugks_status(dugks_ctx *c) {
    if (!c) return DUGKS_EINVAL;
    cudaSetDevice(c->dev);
    int r = sync_ctx(c);
    if (r != DUGKS_OK) return r;
    int flags = 0;
    cudaError_t e = cudaMemcpy(&flags, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read status");
    if (flags & 2) return fail(c, DUGKS_ETIMEOUT, "a device wait ran out");
    if (flags & 1) return fail(c, DUGKS_ENONFINITE, "the field holds NaN or Inf");
    return DUGKS_OK;
}

namespace {
// one CTA waiting (bounded) on an mbarrier whose expected bytes never arrive
__global__ void wait_timeout_kernel(uint32_t polls, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 16);   // the arrival, with 16 bytes pending that nothing sends
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, polls) && threadIdx.x == 0) atomicOr(status, 2);
}
}  // namespace

int dugks_selftest_wait_timeout(dugks_ctx *c, uint32_t max_polls) {
    if (!c || max_polls < 1 || max_polls > (1u << 20)) return DUGKS_EINVAL;
    cudaSetDevice(c->dev);
    wait_timeout_kernel<<<1, 32, 0, c->stream>>>(max_polls, c->dstatus);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "self-test kernel");
    return DUGKS_OK;
}

int dugks_selftest_fail_allocs(int32_t skip, int32_t count) {
    if (skip < 0 || count < 0) return DUGKS_EINVAL;
    dugks::g_alloc_fail.store(0, std::memory_order_relaxed);
    dugks::g_alloc_skip.store(skip, std::memory_order_relaxed);
    dugks::g_alloc_fail.store(count, std::memory_order_relaxed);
    return DUGKS_OK;
}

int dugks_set_variant(dugks_ctx *c, int variant) {
    if (!c || variant < -1 || variant >= FAST_VARIANTS) return DUGKS_EINVAL;
    const bool fast_capable =
        c->p.stages != 1 && (c->p.stages == 2 || c->p.precision != DUGKS_FP16F) && encode_fn() != nullptr;
    if (!fast_capable) return DUGKS_OK;
    // order 4 and the three-stage kernels have one tile shape
    if ((c->p.stages == 3 || c->p.order >= 4) && variant >= 0) variant = 2;
    // order 5 exists on the TMA-staged path only
    if (c->p.order == 5 && variant < 0) return DUGKS_EINVAL;
    cudaSetDevice(c->dev);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    if (variant < 0) {   // the generic kernel (the plain reference GPU step)
        c->fast = false;
        c->tile_w = TILE_X;
        c->tile_h = TILE_Y;
    } else {
        c->fast = true;
        c->variant = variant;
        const bool ok = c->p.precision == DUGKS_FP64 ? setup_fast<double, double>(c)
                        : c->p.precision == DUGKS_FP32 ? setup_fast<float, float>(c)
                                                       : setup_fast<float, __half>(c);
        if (!ok) return fail(c, DUGKS_ECUDA, "tensor map encoding failed");
    }
    c->tiles_x = (c->p.nx + c->tile_w - 1) / c->tile_w;
    const int ntiles = c->tiles_x * ((c->p.ny + c->tile_h - 1) / c->tile_h);
    if (ntiles > c->ntiles) {
        cudaFree(c->partial);
        c->partial = nullptr;
        if (dev_malloc(&c->partial, (size_t)ntiles * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, DUGKS_ENOMEM, "mass partials");
        }
    }
    c->ntiles = ntiles;
    c->mass_valid = false;
    return DUGKS_OK;
}

int dugks_get_variant(const dugks_ctx *c) { return c ? (c->fast ? c->variant : -1) : -1; }

const char *dugks_last_error(const dugks_ctx *c) { return c ? c->err.c_str() : "null context"; }

int64_t dugks_step_index(const dugks_ctx *c) { return c ? c->step : -1; }

// phi of the state and of the previous level where phi is a plane of its own
static int saved_phi_planes(const dugks_ctx *c) { return c->p.precision == DUGKS_FP64 ? 1 : 2; }

size_t dugks_state_bytes(const dugks_ctx *c) {
    if (!c) return 0;
    return 9 * c->plane * c->ssize + (size_t)saved_phi_planes(c) * c->plane * c->tsize;
}

int dugks_save_state(dugks_ctx *c, void *host, size_t bytes, int64_t *step_index) {
    if (!c || !host || bytes != dugks_state_bytes(c)) return c ? fail(c, DUGKS_EINVAL, "bad checkpoint buffer") : DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    cudaSetDevice(c->dev);
    int r = ensure_init(c);
    if (r != DUGKS_OK) return r;
    char *h = static_cast<char *>(host);
    const size_t xs = 9 * c->plane * c->ssize;
    const void *X = c->p.stages == 3 ? c->X[0] : c->X[c->cur];
    cudaError_t e = cudaMemcpyAsync(h, X, xs, cudaMemcpyDeviceToHost, c->stream);
    for (int i = 0; i < saved_phi_planes(c) && e == cudaSuccess; i++)
        e = cudaMemcpyAsync(h + xs + i * c->plane * c->tsize, c->phi[c->pr[i]], c->plane * c->tsize,
                            cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "save state");
    if (step_index) *step_index = c->step;
    return sync_ctx(c);
}

int dugks_load_state(dugks_ctx *c, const void *host, size_t bytes, int64_t step_index) {
    if (!c || !host || bytes != dugks_state_bytes(c) || step_index < 0)
        return c ? fail(c, DUGKS_EINVAL, "bad checkpoint buffer") : DUGKS_EINVAL;
    if (c->sticky != DUGKS_OK) return c->sticky;
    cudaSetDevice(c->dev);
    const char *h = static_cast<const char *>(host);
    const size_t xs = 9 * c->plane * c->ssize;
    void *X = c->p.stages == 3 ? c->X[0] : c->X[c->cur];
    cudaError_t e = cudaMemcpyAsync(X, h, xs, cudaMemcpyHostToDevice, c->stream);
    for (int i = 0; i < saved_phi_planes(c) && e == cudaSuccess; i++)
        e = cudaMemcpyAsync(c->phi[c->pr[i]], h + xs + i * c->plane * c->tsize, c->plane * c->tsize,
                            cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "load state");
    c->step = step_index;
    c->initialized = true;
    c->mass_valid = false;
    return sync_ctx(c);
}

void dugks_destroy(dugks_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

}  // extern "C"
