// dugks_fast.cuh -- the DUGKS step staged by TMA (sm_103a): the two-stage step
// and the two kernels of the three-stage step, stencil orders 2 to 4.
//
// Same arithmetic as step_kernel (dugks_kernels.cuh), organised for throughput:
//  * the tile's 9 distribution planes plus a halo of 1 + 2R cells (stencil radius
//    R = 1 for orders 2-3, 2 for order 4) arrive in shared memory as ONE 3D TMA
//    box (the ghost border of the plane layout makes every halo a plain
//    rectangle), the older phi plane as a 2D box (and, where phi is a plane of its
//    own -- FP32, FP16 storage -- phi of the state as a second one); one mbarrier,
//    bounded wait;
//  * the loop over the 9 velocities is outermost and unrolled (lattice constants,
//    stencil coefficients and the stencils' structural zeros are compile-time per
//    direction): per direction k, bar f^+_k on the tile + R + 1 cells, then bar
//    f_k at the east and north faces of every face-owner cell as fixed linear
//    stencils of bar f^+_k ((2R+1) x (2R+2) taps; coefficients depend only on k
//    and h: computed on the host);
//  * the flux of Eq. (21) is split as
//      L_k = -[(1 - c2) Dbar_k + c2 w_k Phi_k + c3 w_k Psi_k]
//    with Dbar_k the face-difference of bar f_k, Phi_k that of
//    f^eq_b / w_k = phi_b + 3 xi_k.(phi_b u_b) and Psi_k that of xi_k.V_b.
//    During the direction loop each cell's X_k + beta (g_k - X_k) + gamma L_k
//    minus its phi_b part is written over X_k in the TMA buffer (dead by then);
//    once phi_b is known, a second loop adds the phi_b part (in closed form over
//    k) and stores; a phi plane receives phi + the flux sum, stochastically
//    rounded (add_sr).
// Thread layout: a warp owns 32 consecutive face-owner columns (lane l is column
// l - 1) and MR consecutive rows; the CTA's face owners are 32 x (NW * MR), its
// cells TX = 31 by TY = NW * MR - 1.
#pragma once

#include <cuda.h>

#include "dugks_kernels.cuh"

namespace dugks {

// Face stencils of one reconstruction time h, for stencils of radius R (1 for
// orders 2 and 3, 2 for order 4): east face of cell c over rows -R..R and
// columns -R..R+1 around c, north face over rows -R..R+1 and columns -R..R
// (stored with a zero last column). Index = offset + R.
template <typename T, int R = 1>
struct FaceCoefs {
    T e[9][2 * R + 1][2 * R + 2];
    T n[9][2 * R + 2][2 * R + 2];
};

// structural non-zeros of the face stencils (the host fills the same pattern);
// b, a are row and column offsets from the face-owner cell. Upwind: the taps of
// the expansion cell (c or its east / north neighbour, both for a tie). Central:
// the two face cells, plus the tangential derivatives when xi has a tangential part
// (radius 2: the whole box).
__host__ __device__ constexpr bool tapE(int flux, int k, int b, int a, int R = 1) {
    // b in -R..R, a in -R..R+1
    return flux == 0 ? (ex(k) > 0 ? a <= R : ex(k) < 0 ? a >= 1 - R : true)
                     : (ey(k) == 0 ? (b == 0 && (a == 0 || a == 1))
                                   : (R > 1 || b != 0 || a == 0 || a == 1));
}
__host__ __device__ constexpr bool tapN(int flux, int k, int b, int a, int R = 1) {
    // b in -R..R+1, a in -R..R
    return flux == 0 ? (ey(k) > 0 ? b <= R : ey(k) < 0 ? b >= 1 - R : true)
                     : (ex(k) == 0 ? (a == 0 && (b == 0 || b == 1))
                                   : (R > 1 || a != 0 || b == 0 || b == 1));
}

// Per-step scalars of the fast kernel that the generic parameters do not carry.
template <typename T>
struct FastExtra {
    T vc_t, vc_told, vc_tface;   // reversal factors cos(pi t / T) at t, t_old, t_face (vortex, deformation)
};

// ---- TMA and mbarrier (inline PTX) -------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return done != 0;
}
// Bounded wait: gives up after max_iter polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t max_iter) {
    for (uint32_t i = 0; i < max_iter; i++)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

constexpr uint32_t MBAR_MAX_POLLS = 1u << 22;

// 1 / sqrt(g): correctly rounded in FP64; the hardware reciprocal square root in
// FP32 (a few ulp, far inside the FP32 tolerance, and no division slow path)
__device__ __forceinline__ double rnorm(double g) { return 1.0 / sqrt(g); }
__device__ __forceinline__ float rnorm(float g) { return rsqrtf(g); }

// wrap a tile-relative index into [0, n) (at most a few periods away)
__device__ __forceinline__ int wrap_small(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// four consecutive shared-memory values (16-B aligned for float, two 16-B loads for double)
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 q0 = reinterpret_cast<const double2 *>(p)[0], q1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// Plane geometry for the ghost writer: passed by value, so that a caller whose
// parameters are a local struct (the many-grid kernel) does not have to keep that
// struct in local memory for the call.
struct GhostGeom {
    int nx, ny, pitch;
    size_t plane;
};

// ghost images of the 9 distribution values and phi of one cell near an edge
// (values by argument so that the caller's registers stay registers)
template <typename T, typename V>
__device__ __noinline__ void put_ghosts9(GhostGeom gg, T *phi_out, V *out, int x, int y, T phi, V v0, V v1, V v2,
                                         V v3, V v4, V v5, V v6, V v7, V v8) {
#pragma unroll 1
    for (int ay = -1; ay <= 1; ay++) {
        const int yy = y + ay * gg.ny;
        if (yy < -GHOST || yy >= gg.ny + GHOST) continue;
#pragma unroll 1
        for (int ax = -1; ax <= 1; ax++) {
            const int xx = x + ax * gg.nx;
            if ((ax == 0 && ay == 0) || xx < -GHOST || xx >= gg.nx + GHOST) continue;
            const size_t g = (size_t)(yy + GHOST) * gg.pitch + (size_t)(xx + GHOST), pl = gg.plane;
            out[g] = v0;
            out[pl + g] = v1;
            out[2 * pl + g] = v2;
            out[3 * pl + g] = v3;
            out[4 * pl + g] = v4;
            out[5 * pl + g] = v5;
            out[6 * pl + g] = v6;
            out[7 * pl + g] = v7;
            out[8 * pl + g] = v8;
            if (phi_out != nullptr) phi_out[g] = phi;
        }
    }
}

// Tile of the TMA-staged kernel for stencils of radius R: state region with a
// halo of H = 1 + 2R, cell-quantity region (bar f^+, V) with a halo of R + 1.
template <typename T, typename ST, int NW, int MR, int R = 1>
struct FastTile {
    static constexpr int NT = NW * 32;
    static constexpr int H = 1 + 2 * R, C1 = R + 1;
    static constexpr int TX = 31, TY = NW * MR - 1;         // cells written
    static constexpr int RW = TX + 2 * H, RH = TY + 2 * H;  // state region
    static constexpr int CW = TX + 2 * C1, CH = TY + 2 * C1;   // cell-quantity region
    static constexpr int NC = CW * CH;
    // cell-quantity cells not owned by a thread: columns -R-1 .. -2 and TX .. TX + R
    // (all rows), rows -R-1 .. -2 and TY .. TY + R (columns -1 .. TX - 1)
    static constexpr int NE = (2 * R + 1) * (CH + 32);
    static constexpr int NXS = (NE + NT - 1) / NT;          // extra slots per thread
    static constexpr int AS = 16 / (int)sizeof(ST);         // TMA x alignment of the state (elements)
    static constexpr int AT = 16 / (int)sizeof(T);          // ... of the phi planes
    static constexpr int BW = (RW + AS - 1 + AS - 1) / AS * AS;   // state box width
    static constexpr int BWT = (RW + AT - 1 + AT - 1) / AT * AT;  // phi box width
    static constexpr bool DEV = Store<T, ST>::deviation, PHIP = Store<T, ST>::phi_plane;
    // shared-memory carve-up (byte offsets, 128-B aligned TMA destinations first)
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t oX = 0;
    static constexpr size_t oPo = al(oX + sizeof(ST) * 9 * BW * RH);
    static constexpr size_t oPc = al(oPo + sizeof(T) * BWT * RH);
    static constexpr size_t oPhi = al(oPc + (PHIP ? sizeof(T) * BWT * RH : 0));
    static constexpr size_t oPart = al(oPhi + (PHIP ? 0 : sizeof(T) * RW * RH));
    static constexpr size_t oV = al(oPart + (DEV ? sizeof(T) * 9 * 32 * (TY + 1) : 0));
    static constexpr size_t oF = al(oV + sizeof(T) * 2 * NC);
    static constexpr size_t oNB = al(oF + sizeof(T) * 2 * NC);
    static constexpr size_t oQ = al(oNB + sizeof(T) * 2 * NW * 32);
    static constexpr size_t oVel = al(oQ + sizeof(T) * 3 * NW * 32);
    static constexpr size_t oRed = al(oVel + sizeof(T) * 4 * (CW + CH));
    static constexpr size_t oBar = oRed + sizeof(double) * 32;
    static constexpr size_t smem_bytes = oBar + 16;
    static constexpr uint32_t tx_bytes =
        (uint32_t)(sizeof(ST) * 9 * BW * RH + sizeof(T) * BWT * RH * (PHIP ? 2 : 1));
    // resident CTAs per SM that shared memory allows (228 KiB per SM, 1 KiB reserved
    // per CTA) and threads allow, without asking for fewer than 64 registers per thread:
    // the register target of the launch bounds, so that registers never cut occupancy
    // below what shared memory gives
    static constexpr int cmin(int a, int b) { return a < b ? a : b; }
    static constexpr int min_blocks =
        cmin(cmin((int)((228u * 1024u) / (smem_bytes + 1024u)), 2048 / NT), 65536 / (NT * 64));
    // first kernel of the three-stage scheme: a second per-direction partial (the
    // accumulator output) after the common layout
    static constexpr size_t oPart2 = al(smem_bytes);
    static constexpr size_t smem_bytes_t3a = oPart2 + sizeof(T) * 9 * 32 * (TY + 1);
    static constexpr int min_blocks_t3a =
        cmin(cmin((int)((228u * 1024u) / (smem_bytes_t3a + 1024u)), 2048 / NT), 65536 / (NT * 64));
};

// One tile (bx, by) of one grid. The caller initialised the mbarrier `bar`
// (count 1) and passes the parity of its next phase. Returns false if the TMA
// copy never arrived (status flagged). mass_out: where the tile's FP64 partial
// goes (may be null).
template <typename T, typename ST, int ORDER, int FLUX, int NW, int MR, int KIND = KIND_T2>
__device__ __forceinline__ bool fast_tile(const StepParams<T> &p, const FaceCoefs<T, (ORDER == 4 ? 2 : 1)> &cf,
                                          const FastExtra<T> &fe_,
                                          const CUtensorMap *tmX, const CUtensorMap *tmPo, const CUtensorMap *tmPc,
                                          int bx, int by, double *mass_out, unsigned char *smem, uint64_t *bar,
                                          uint32_t phase) {
    constexpr int R = ORDER == 4 ? 2 : 1;   // stencil radius
    using FT = FastTile<T, ST, NW, MR, R>;
    constexpr int TX = FT::TX, TY = FT::TY, RW = FT::RW, CW = FT::CW, CH = FT::CH, NC = FT::NC;
    constexpr int NT = FT::NT, BW = FT::BW, BWT = FT::BWT, RH = FT::RH, NE = FT::NE, NXS = FT::NXS;
    constexpr int H = FT::H, C1 = FT::C1;
    constexpr bool DEV = FT::DEV, PHIP = FT::PHIP;
    static_assert(ORDER >= 2 && ORDER <= 4, "stencil orders 2 to 4");
    // KIND_T2: the two-stage step. KIND_T3A / KIND_T3B: the two kernels of the
    // three-stage step (Sec. II.B.2), full storage only:
    //   T3A  out1 = X + be1 (g - X) + ga1 L (tilde f at t'), out2 = X + be2 (g - X) + ga2 L
    //        (the accumulator, in T); phi_out = phi of X, or with phi planes phi of out1
    //        (phi_out) and of out2 (phi_out2);
    //   T3B  out1 = acc + be1 (g - X) + ga1 L (hat f at t_n + dt; al1 = -be1), mass partial;
    //        with phi planes phi of acc from phi_acc and phi of out1 to phi_out.
    static_assert(KIND == KIND_T2 ? Store<T, ST>::t2 : Store<T, ST>::t3, "scheme not served by this storage");
    constexpr bool T3A = KIND == KIND_T3A, T3B = KIND == KIND_T3B;

    ST *sX = reinterpret_cast<ST *>(smem + FT::oX);
    T *sPo = reinterpret_cast<T *>(smem + FT::oPo);
    T *sPc = reinterpret_cast<T *>(smem + FT::oPc);
    T *sPhi = reinterpret_cast<T *>(smem + FT::oPhi);
    T *sPart = reinterpret_cast<T *>(smem + FT::oPart);
    T *sV = reinterpret_cast<T *>(smem + FT::oV);
    T *sF = reinterpret_cast<T *>(smem + FT::oF);
    T *sNB = reinterpret_cast<T *>(smem + FT::oNB);
    T *sQ = reinterpret_cast<T *>(smem + FT::oQ);
    T *sVel = reinterpret_cast<T *>(smem + FT::oVel);   // vortex factors, see below
    double *sred = reinterpret_cast<double *>(smem + FT::oRed);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = p.nx, ny = p.ny;
    const GhostGeom gg{nx, ny, p.pitch, p.plane};
    const int x0 = bx * TX, y0 = by * TY;
    // padded-plane coordinates of the state box; ox = offset of relative x = -H in the box
    const int xs_raw = x0 - H + GHOST, ys = y0 - H + GHOST;
    const int xs = xs_raw / FT::AS * FT::AS, ox = xs_raw - xs;
    const int xst = xs_raw / FT::AT * FT::AT, oxt = xs_raw - xst;

    // ---- S0: one TMA box for the 9 planes (+ phi planes) --------------------
    // (the barrier also orders this tile's copy after the previous tile's
    // shared-memory accesses when a CTA processes several tiles)
    __syncthreads();
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, FT::tx_bytes);
        tma_load_3d(sX, tmX, xs, ys, 0, bar);
        tma_load_2d(sPo, tmPo, xst, ys, bar);
        if constexpr (PHIP) tma_load_2d(sPc, tmPc, xst, ys, bar);
    }
    // while the copy is in flight: velocity tables
    // single vortex u = -U A(x) B(y) c(t), v = U A(y) B(x) c(t), with
    // A(s) = sin^2(pi s / L), B(s) = sin(2 pi s / L) at cell centres (s = i + 1/2)
    // and at faces (s = i + 1) of the wrapped cells of this tile (+ R + 1 halo)
    T *sAxc = sVel, *sBxc = sAxc + CW, *sAxf = sBxc + CW, *sBxf = sAxf + CW;
    T *sAyc = sBxf + CW, *sByc = sAyc + CH, *sAyf = sByc + CH, *sByf = sAyf + CH;
    if (p.vel_kind == VEL_VORTEX) {
        const T L = p.vp0;
        for (int i = tid; i < 2 * (CW + CH); i += NT) {
            const bool isx = i < 2 * CW;
            const int j = isx ? (i >> 1) : ((i - 2 * CW) >> 1);
            const bool face = (i & 1) != 0;
            const int g = isx ? wrap_small(x0 + j - C1, nx) : wrap_small(y0 + j - C1, ny);
            const T s = T(g) + (face ? T(1) : T(0.5));
            const T sn = sinpi_(s / L);
            const T A = sn * sn, B = sinpi_(T(2) * s / L);
            if (isx) {
                (face ? sAxf : sAxc)[j] = A;
                (face ? sBxf : sBxc)[j] = B;
            } else {
                (face ? sAyf : sAyc)[j] = A;
                (face ? sByf : sByc)[j] = B;
            }
        }
    }
    if (!mbar_wait_bounded(bar, phase, MBAR_MAX_POLLS)) {
        // the copy never completed: flag it, give it one more bounded chance to
        // land (it targets this CTA's shared memory), and leave
        if (tid == 0) atomicOr(p.status, 2);
        mbar_wait_bounded(bar, phase, MBAR_MAX_POLLS);
        return false;
    }

    // accessors (relative cell coordinates x, y of the tile)
    auto xidx = [&](int x, int y) { return (y + H) * BW + (x + H + ox); };   // + k * RH * BW
    auto PHI = [&](int x, int y) -> T {
        if constexpr (PHIP) return sPc[(y + H) * BWT + (x + H + oxt)];
        else return sPhi[(y + H) * RW + (x + H)];
    };
    // velocity of a cell centre (where = 0), east face (1) or north face (2)
    auto vel = [&](int x, int y, int where, T t, T vc, T &u, T &v) {
        if (p.vel_kind == VEL_UNIFORM) {
            u = p.vp0;
            v = p.vp1;
        } else if (p.vel_kind == VEL_VORTEX) {
            const int i = x + C1, j = y + C1;
            const T Ax = where == 1 ? sAxf[i] : sAxc[i], Bx = where == 1 ? sBxf[i] : sBxc[i];
            const T Ay = where == 2 ? sAyf[j] : sAyc[j], By = where == 2 ? sByf[j] : sByc[j];
            u = -p.vp1 * Ax * By * vc;
            v = p.vp1 * Ay * Bx * vc;
        } else if (p.vel_kind == VEL_DEFORM) {   // spatial part times the reversal factor vc
            const int gx = wrap_small(x0 + x, nx), gy = wrap_small(y0 + y, ny);
            deform_spatial(p, T(gx) + (where == 1 ? T(1) : T(0.5)), T(gy) + (where == 2 ? T(1) : T(0.5)), u, v);
            u *= vc;
            v *= vc;
        } else {
            const int gx = wrap_small(x0 + x, nx), gy = wrap_small(y0 + y, ny);
            if (where == 0) vel_cell(p, gx, gy, t, u, v);
            else vel_face(p, gx, gy, where - 1, t, u, v);
        }
    };
    // cell quantities of cell (x, y): phi, P = 3 phi u + tau V (g_k = w_k (phi + xi_k.P)),
    // and V = theta n + 3 D into shared memory (face sources)
    auto cell_q = [&](int x, int y, T &ph, T &Px, T &Py) {
        ph = PHI(x, y);
        T gxp, gyp;
        if constexpr (ORDER == 4) {   // the order's own gradient (Sec. II.B.1)
            if constexpr (PHIP) grad21(sPc + (y + H) * BWT + (x + H + oxt), BWT, gxp, gyp);
            else grad21(sPhi + (y + H) * RW + (x + H), RW, gxp, gyp);
        } else {
            const T ne = PHI(x + 1, y + 1), nw = PHI(x - 1, y + 1), se = PHI(x + 1, y - 1), sw = PHI(x - 1, y - 1);
            gxp = (PHI(x + 1, y) - PHI(x - 1, y)) * T(1.0 / 3.0) + ((ne - nw) + (se - sw)) * T(1.0 / 12.0);
            gyp = (PHI(x, y + 1) - PHI(x, y - 1)) * T(1.0 / 3.0) + ((ne - se) + (nw - sw)) * T(1.0 / 12.0);
        }
        const T g2 = gxp * gxp + gyp * gyp;
        T nxv = T(0), nyv = T(0);
        if (g2 > T(1e-24)) {  // Eq. (2); n = 0 where grad phi vanishes
            const T inv = rnorm(g2);
            nxv = gxp * inv;
            nyv = gyp * inv;
        }
        const T theta = p.theta_c * (ph - p.phiA) * (ph - p.phiB);  // Eq. (4)
        // the velocity at the cell centre at both time levels: the spatial part of the
        // vortex and of the deformation once, scaled by their reversal factors; the
        // other kinds do not depend on t
        const bool vortex = p.vel_kind == VEL_VORTEX || p.vel_kind == VEL_DEFORM;
        T u0, v0;
        vel(x, y, 0, p.t, vortex ? T(1) : fe_.vc_t, u0, v0);
        const T u = vortex ? u0 * fe_.vc_t : u0, v = vortex ? v0 * fe_.vc_t : v0;
        T Dx = T(0), Dy = T(0);
        if (p.useD) {  // d(phi u)/dt, backward difference
            const T uo = vortex ? u0 * fe_.vc_told : u0, vo = vortex ? v0 * fe_.vc_told : v0;
            const T po = sPo[(y + H) * BWT + (x + H + oxt)];
            Dx = (ph * u - po * uo) * p.inv_dtD;
            Dy = (ph * v - po * vo) * p.inv_dtD;
        }
        const T Vx = theta * nxv + T(3) * Dx, Vy = theta * nyv + T(3) * Dy;  // Eq. (14b)
        Px = T(3) * ph * u + p.tau * Vx;
        Py = T(3) * ph * v + p.tau * Vy;
        const int j = (y + C1) * CW + (x + C1);
        sV[j] = Vx;
        sV[NC + j] = Vy;
    };

    // ---- S1: phi = sum_k X_k on the state region (Eq. (30)) ------------------
    // (a phi plane already holds it)
    if constexpr (!PHIP) {
        for (int y = warp - H; y < RH - H; y += NW)
            for (int x = lane - H; x < RW - H; x += 32) {
                const int xi = xidx(x, y);
                T s = T(0);
#pragma unroll
                for (int k = 0; k < 9; k++) s += (T)sX[k * RH * BW + xi];
                sPhi[(y + H) * RW + (x + H)] = s;
            }
    }
    __syncthreads();

    // ---- S2: cell quantities: my MR cells and up to NXS halo cells ----------
    const int fx = lane - 1;                // face-owner column
    const int fy0 = warp * MR - 1;          // first face-owner row of this thread
    T cg[MR], cPx[MR], cPy[MR];
#pragma unroll
    for (int r = 0; r < MR; r++) cell_q(fx, fy0 + r, cg[r], cPx[r], cPy[r]);
    // extra cells are clamped to the last one: surplus threads recompute it and
    // store identical values (no divergent branch in the direction loop)
    int exj[NXS], exX[NXS];
    T eg[NXS], ePx[NXS], ePy[NXS];
    // a warp whose first slot lies beyond the halo has nothing to do there (warp-uniform)
    bool exw[NXS];
#pragma unroll
    for (int s = 0; s < NXS; s++) exw[s] = warp * 32 + s * NT < NE;
#pragma unroll
    for (int s = 0; s < NXS; s++) {
        exj[s] = exX[s] = 0;
        eg[s] = ePx[s] = ePy[s] = T(0);
        if (!exw[s]) continue;
        const int e = min(tid + s * NT, NE - 1);
        int x, y;
        if (e < (2 * R + 1) * CH) {
            const int c = e / CH;   // columns -R-1 .. -2, then TX .. TX + R
            x = c < R ? c - C1 : TX + c - R;
            y = e - c * CH - C1;
        } else {
            const int e2 = e - (2 * R + 1) * CH, c = e2 >> 5;
            y = c < R ? c - C1 : TY + c - R;
            x = (e2 & 31) - 1;
        }
        exj[s] = (y + C1) * CW + (x + C1);
        exX[s] = xidx(x, y);
        cell_q(x, y, eg[s], ePx[s], ePy[s]);
    }

    // ---- S3: directions ------------------------------------------------------
    T phbE[MR], phbN[MR], sumD[MR];
#pragma unroll
    for (int r = 0; r < MR; r++) phbE[r] = phbN[r] = sumD[r] = T(0);
    const T gmc = p.ga1 * (T(1) - p.c2);    // gamma (1 - c2)
    T fn0Prev = T(0);                       // pending south difference of my first row
    const int fbase = (fy0 + C1) * CW + (fx + C1);   // my first cell in the cell-quantity region
    const int xbase = xidx(fx, fy0);                 // ... in the state box

    // partial update of my cell r, direction k: X + beta (g - X) - gamma (1 - c2) Dbar
    auto part_ref = [&](int k, int r) -> T & {
        if constexpr (DEV) return sPart[(k * (TY + 1) + (fy0 + 1 + r)) * 32 + lane];
        else return reinterpret_cast<T *>(sX)[k * RH * BW + xbase + r * BW];
    };
    // T3A: the accumulator's partial
    T *sPart2 = reinterpret_cast<T *>(smem + FT::oPart2);
    auto part2_ref = [&](int k, int r) -> T & { return sPart2[(k * (TY + 1) + (fy0 + 1 + r)) * 32 + lane]; };
    const T gmc2 = p.ga2 * (T(1) - p.c2);

    // The direction loop is unrolled: xi_k, w_k, the stencil coefficients (kernel
    // parameters, i.e. constant-bank operands) and the structural zeros of each
    // face stencil are compile-time per direction.
#pragma unroll
    for (int k = 0; k < 9; k++) {
        T *F = sF + (k & 1) * NC;
        constexpr T one = T(1);
        const int kx = ex(k), ky = ey(k);
        const T wk = wq<T>(k);
        // xi_k . P without multiplications by 0 or +-1
        auto xiP = [&](T px, T py) -> T {
            T v = T(0);
            if (kx > 0) v = px;
            if (kx < 0) v = -px;
            if (ky > 0) v = (kx != 0) ? v + py : py;
            if (ky < 0) v = (kx != 0) ? v - py : -py;
            return v;
        };
        // S3a: bar f^+_k = X_k + b (g_k - X_k) (increment form; a + b = 1)
        T xk[MR], gk[MR], fo[MR];
#pragma unroll
        for (int r = 0; r < MR; r++) {
            const ST v = sX[k * RH * BW + xbase + r * BW];
            if constexpr (DEV) xk[r] = wk * (cg[r] + to_f(v) * p.qinv);
            else xk[r] = (T)v;
            gk[r] = wk * (cg[r] + xiP(cPx[r], cPy[r]));
            fo[r] = xk[r] + p.b * (gk[r] - xk[r]);
            F[fbase + r * CW] = fo[r];
        }
#pragma unroll
        for (int s = 0; s < NXS; s++) {
            if (!exw[s]) continue;
            const ST v = sX[k * RH * BW + exX[s]];
            T xe;
            if constexpr (DEV) xe = wk * (eg[s] + to_f(v) * p.qinv);
            else xe = (T)v;
            const T ge = wk * (eg[s] + xiP(ePx[s], ePy[s]));
            F[exj[s]] = xe + p.b * (ge - xe);
        }
        __syncthreads();
        // finish the previous direction's first-row partial with its south difference
        if (k > 1 && ey(k - 1) != 0) {   // (warp 0 reads a neighbour slot; its row -1 result is never stored)
            const T below = sNB[((k - 1) & 1) * NW * 32 + (warp > 0 ? warp - 1 : 0) * 32 + lane];
            const T d = ey(k - 1) > 0 ? (fn0Prev - below) : (below - fn0Prev);
            part_ref(k - 1, 0) -= gmc * d;
            if constexpr (T3A) part2_ref(k - 1, 0) -= gmc2 * d;
            sumD[0] += d;
        }
        // S3b: face values of my MR cells from an (MR + 2R + 1) x (2R + 2) window of
        // bar f^+_k, rows -R .. MR + R, columns -R .. R + 1 (entries no tap uses are
        // never loaded; my own column of rows 0 .. MR - 1 is in registers)
        T win[MR + 2 * R + 1][2 * R + 2];
#pragma unroll
        for (int i = 0; i < MR + 2 * R + 1; i++)
#pragma unroll
            for (int a = 0; a < 2 * R + 2; a++)
                win[i][a] = (a == R && i >= R && i < R + MR) ? fo[i - R] : F[fbase + (i - R) * CW + (a - R)];
        T fe[MR], fn[MR];
#pragma unroll
        for (int r = 0; r < MR; r++) {
            T se = T(0), sn = T(0);
#pragma unroll
            for (int b = 0; b < 2 * R + 1; b++)
#pragma unroll
                for (int a = 0; a < 2 * R + 2; a++)
                    if (tapE(FLUX, k, b - R, a - R, R)) se += cf.e[k][b][a] * win[r + b][a];
#pragma unroll
            for (int b = 0; b < 2 * R + 2; b++)
#pragma unroll
                for (int a = 0; a < 2 * R + 1; a++)
                    if (tapN(FLUX, k, b - R, a - R, R)) sn += cf.n[k][b][a] * win[r + b][a];
            fe[r] = se;
            fn[r] = sn;
            phbE[r] += se;
            phbN[r] += sn;
        }
        // Dbar_k = xi_x (f_E(c) - f_E(c - E)) + xi_y (f_N(c) - f_N(c - N)); partial update
        // (direction 0 has xi = 0 and is completed from phi in S4)
        if (k > 0) {
#pragma unroll
            for (int r = 0; r < MR; r++) {
                T d = T(0);
                if (kx != 0) {
                    const T left = __shfl_up_sync(0xffffffffu, fe[r], 1);
                    d = kx > 0 ? fe[r] - left : left - fe[r];
                }
                if (ky != 0 && r > 0) d = ky > 0 ? d + (fn[r] - fn[r - 1]) : d - (fn[r] - fn[r - 1]);
                // cells outside the tile write harmless values
                part_ref(k, r) = (T3B ? T(0) : xk[r]) + p.be1 * (gk[r] - xk[r]) - gmc * d;
                if constexpr (T3A) part2_ref(k, r) = xk[r] + p.be2 * (gk[r] - xk[r]) - gmc2 * d;
                sumD[r] += d;
            }
        }
        (void)one;
        fn0Prev = fn[0];
        if (ky != 0) sNB[(k & 1) * NW * 32 + warp * 32 + lane] = fn[MR - 1];
    }
    __syncthreads();
    if (ey(8) != 0) {
        const T below = sNB[(8 & 1) * NW * 32 + (warp > 0 ? warp - 1 : 0) * 32 + lane];
        const T d = ey(8) > 0 ? (fn0Prev - below) : (below - fn0Prev);
        part_ref(8, 0) -= gmc * d;
        if constexpr (T3A) part2_ref(8, 0) -= gmc2 * d;
        sumD[0] += d;
    }

    // ---- S4: face scalars, flux completion and store -------------------------
    T qE[MR][3], qN[MR][3];
#pragma unroll
    for (int r = 0; r < MR; r++) {
        T u, v;
        vel(fx, fy0 + r, 1, p.t_face, fe_.vc_tface, u, v);
        qE[r][0] = phbE[r];
        qE[r][1] = phbE[r] * u;
        qE[r][2] = phbE[r] * v;
        vel(fx, fy0 + r, 2, p.t_face, fe_.vc_tface, u, v);
        qN[r][0] = phbN[r];
        qN[r][1] = phbN[r] * u;
        qN[r][2] = phbN[r] * v;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) sQ[c * NW * 32 + warp * 32 + lane] = qN[MR - 1][c];
    __syncthreads();

    double msum = 0.0;
    const size_t plane = p.plane;
    const T ga = p.ga1, gc2 = p.ga1 * p.c2, gc3 = p.ga1 * p.c3;
#pragma unroll
    for (int r = 0; r < MR; r++) {
        const int x = fx, y = fy0 + r;
        // east differences from the lane to the west, north from the row below
        T dE[3], dN[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            dE[c] = qE[r][c] - __shfl_up_sync(0xffffffffu, qE[r][c], 1);
            const T below = r > 0 ? qN[r - 1][c] : (warp > 0 ? sQ[c * NW * 32 + (warp - 1) * 32 + lane] : T(0));
            dN[c] = qN[r][c] - below;
        }
        const int gx = x0 + x, gy = y0 + y;
        if (x < 0 || y < 0 || gx >= nx || gy >= ny) continue;
        const int cj = fbase + r * CW;
        // Delta V_b = (V(c + E) - V(c - E)) / 2 and likewise north
        const T dVEx = T(0.5) * (sV[cj + 1] - sV[cj - 1]), dVEy = T(0.5) * (sV[NC + cj + 1] - sV[NC + cj - 1]);
        const T dVNx = T(0.5) * (sV[cj + CW] - sV[cj - CW]), dVNy = T(0.5) * (sV[NC + cj + CW] - sV[NC + cj - CW]);
        if constexpr (KIND != KIND_T2) {
            // out = part_k - w_k (xi_x A1 + xi_y A2 + xi_x^2 B1 + xi_x xi_y B2 + xi_y^2 B3), all scaled
            // by the output's gamma; its rest component from phi_base + gamma sum_k L_k (a phi
            // plane: that sum added with stochastic rounding, uniform bits `bits`)
            auto combine = [&](T gam, T gmcX, T phib, auto part, T (&o)[9], uint32_t bits) -> T {
                const T g2 = gam * p.c2, g3 = gam * p.c3;
                const T A1 = g2 * dE[0], A2 = g2 * dN[0];
                const T B1 = T(3) * g2 * dE[1] + g3 * dVEx;
                const T B2 = T(3) * g2 * (dE[2] + dN[1]) + g3 * (dVEy + dVNx);
                const T B3 = T(3) * g2 * dN[2] + g3 * dVNy;
                const T dph = -gmcX * sumD[r] - (B1 + B3) * T(1.0 / 3.0);
                T ph;
                if constexpr (PHIP) ph = add_sr(phib, dph, bits);
                else ph = phib + dph;
                const T S13 = B1 + B3;
                o[1] = part(1) - wq<T>(1) * (A1 + B1);
                o[5] = part(5) - wq<T>(5) * (B1 - A1);
                o[3] = part(3) - wq<T>(3) * (A2 + B3);
                o[7] = part(7) - wq<T>(7) * (B3 - A2);
                o[2] = part(2) - wq<T>(2) * ((A1 + A2) + (S13 + B2));
                o[4] = part(4) - wq<T>(4) * ((A2 - A1) + (S13 - B2));
                o[6] = part(6) - wq<T>(6) * ((S13 + B2) - (A1 + A2));
                o[8] = part(8) - wq<T>(8) * ((A1 - A2) + (S13 - B2));
                T rsum = T(0);
#pragma unroll
                for (int k = 1; k < 9; k++) rsum += o[k];
                o[0] = ph - rsum;
                return ph;
            };
            const bool edge = gx < GHOST || gx >= nx - GHOST || gy < GHOST || gy >= ny - GHOST;
            const size_t g = gidx(p, gx, gy);
            T *O = static_cast<T *>(p.out1);
            T o[9];
            const uint32_t bits = PHIP ? sr_bits(p, gx, gy) : 0u;
            if constexpr (T3A) {
                // phi plane: phi of tilde f' (with ghosts: kernel B stages it) and of the
                // accumulator; otherwise phi of X (the older level of kernel B's d(phi u)/dt)
                const T ph1 = combine(p.ga1, gmc, cg[r], [&](int k) { return part_ref(k, r); }, o, bits);
                const T pho = PHIP ? ph1 : cg[r];
#pragma unroll
                for (int k = 0; k < 9; k++) O[k * plane + g] = o[k];
                p.phi_out[g] = pho;
                if (edge) put_ghosts9(gg, p.phi_out, O, gx, gy, pho,
                                      o[0], o[1], o[2], o[3], o[4], o[5], o[6], o[7], o[8]);
                T o2[9];
                const T ph2 = combine(p.ga2, gmc2, cg[r], [&](int k) { return part2_ref(k, r); }, o2, mix32(bits));
#pragma unroll
                for (int k = 0; k < 9; k++) p.out2[k * plane + g] = o2[k];   // read per cell only: no ghosts
                if constexpr (PHIP) p.phi_out2[g] = ph2;
            } else {
                const T *Acc = static_cast<const T *>(p.acc);
                T a[9], pha = T(0);
#pragma unroll
                for (int k = 0; k < 9; k++) {
                    a[k] = Acc[k * plane + g];
                    if constexpr (!PHIP) pha += a[k];
                }
                if constexpr (PHIP) pha = p.phi_acc[g];
                const T phn = combine(p.ga1, gmc, pha, [&](int k) { return a[k] + part_ref(k, r); }, o, bits);
#pragma unroll
                for (int k = 0; k < 9; k++) O[k * plane + g] = o[k];
                if constexpr (PHIP) p.phi_out[g] = phn;   // phi^{n+1} (else phi_out is null)
                if (edge) put_ghosts9(gg, p.phi_out, O, gx, gy, phn,
                                      o[0], o[1], o[2], o[3], o[4], o[5], o[6], o[7], o[8]);
                msum += (double)phn;
            }
            continue;
        }
        // gamma w_k (c2 Phi_k + c3 Psi_k) = w_k (xi_x A1 + xi_y A2 + xi_x^2 B1 + xi_x xi_y B2 + xi_y^2 B3)
        const T A1 = gc2 * dE[0], A2 = gc2 * dN[0];
        const T B1 = T(3) * gc2 * dE[1] + gc3 * dVEx;
        const T B2 = T(3) * gc2 * (dE[2] + dN[1]) + gc3 * (dVEy + dVNx);
        const T B3 = T(3) * gc2 * dN[2] + gc3 * dVNy;
        // new phi = phi + gamma sum_k L_k (sum_k w_k xi_k = 0, sum_k w_k xi_a xi_b = delta_ab / 3)
        // (a phi plane: the flux sum added with unbiased stochastic rounding)
        const T dphi = -gmc * sumD[r] - (B1 + B3) * T(1.0 / 3.0);
        T phn;
        if constexpr (PHIP) phn = add_sr(cg[r], dphi, sr_bits(p, gx, gy));
        else phn = cg[r] + dphi;
        const bool edge = gx < GHOST || gx >= nx - GHOST || gy < GHOST || gy >= ny - GHOST;
        const size_t g = gidx(p, gx, gy);
        T o[9];
        const T S13 = B1 + B3;
        o[1] = part_ref(1, r) - wq<T>(1) * (A1 + B1);
        o[5] = part_ref(5, r) - wq<T>(5) * (B1 - A1);
        o[3] = part_ref(3, r) - wq<T>(3) * (A2 + B3);
        o[7] = part_ref(7, r) - wq<T>(7) * (B3 - A2);
        o[2] = part_ref(2, r) - wq<T>(2) * ((A1 + A2) + (S13 + B2));
        o[4] = part_ref(4, r) - wq<T>(4) * ((A2 - A1) + (S13 - B2));
        o[6] = part_ref(6, r) - wq<T>(6) * ((S13 + B2) - (A1 + A2));
        o[8] = part_ref(8, r) - wq<T>(8) * ((A1 - A2) + (S13 - B2));
        // rest component: the new phi is exactly phn (up to this subtraction)
        T rsum = T(0);
#pragma unroll
        for (int k = 1; k < 9; k++) rsum += o[k];
        o[0] = phn - rsum;
        if constexpr (DEV) {
            __half *Oq = static_cast<__half *>(p.out1);
            __half qv[9];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                qv[k] = __float2half_rn((o[k] - wq<T>(k) * phn) * (p.qscale / wq<T>(k)));
                Oq[k * plane + g] = qv[k];
            }
            p.phi_out[g] = phn;
            if (edge)
                put_ghosts9(gg, p.phi_out, Oq, gx, gy, phn,
                            qv[0], qv[1], qv[2], qv[3], qv[4], qv[5], qv[6], qv[7], qv[8]);
        } else {
            // a phi plane receives the new phi; otherwise phi_out is phi of X (the
            // older level of the next step's d(phi u)/dt)
            const T pho = PHIP ? phn : cg[r];
            T *O = static_cast<T *>(p.out1);
#pragma unroll
            for (int k = 0; k < 9; k++) O[k * plane + g] = o[k];
            p.phi_out[g] = pho;
            if (edge) put_ghosts9(gg, p.phi_out, O, gx, gy, pho,
                                  o[0], o[1], o[2], o[3], o[4], o[5], o[6], o[7], o[8]);
        }
        msum += (double)phn;
    }
    if (mass_out != nullptr) {
        const double s = block_sum(msum, sred);
        if (tid == 0) *mass_out = s;
    }
    return true;
}

template <typename T, typename ST, int NW, int MR, int R = 1>
__device__ __forceinline__ uint64_t *fast_bar(unsigned char *smem) {
    return reinterpret_cast<uint64_t *>(smem + FastTile<T, ST, NW, MR, R>::oBar);
}

// One grid, one tile per CTA.
template <typename T, typename ST, int ORDER, int FLUX, int NW, int MR, int KIND = KIND_T2>
__global__ void __launch_bounds__(NW * 32,
                                  (KIND == KIND_T3A ? FastTile<T, ST, NW, MR, (ORDER == 4 ? 2 : 1)>::min_blocks_t3a
                                                    : FastTile<T, ST, NW, MR, (ORDER == 4 ? 2 : 1)>::min_blocks))
step_fast_kernel(const __grid_constant__ StepParams<T> p,
                 const __grid_constant__ FaceCoefs<T, (ORDER == 4 ? 2 : 1)> cf,
                 const __grid_constant__ FastExtra<T> fe_, const __grid_constant__ CUtensorMap tmX,
                 const __grid_constant__ CUtensorMap tmPo, const __grid_constant__ CUtensorMap tmPc) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = fast_bar<T, ST, NW, MR, (ORDER == 4 ? 2 : 1)>(smem);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    pdl_wait();   // the previous kernel's output (launched with programmatic serialization)
    double *mo = p.mass_partial ? p.mass_partial + blockIdx.y * p.tiles_x + blockIdx.x : nullptr;
    fast_tile<T, ST, ORDER, FLUX, NW, MR, KIND>(p, cf, fe_, &tmX, &tmPo, &tmPc, blockIdx.x, blockIdx.y, mo, smem, bar,
                                                0);
    // the next kernel may be scheduled once every tile is done with its work (a
    // trigger at entry would place its waiting CTAs while this grid still runs,
    // unevenly when the grid is a single wave)
    pdl_trigger();
}

// ---- many grids per launch ----------------------------------------------------
// Per-grid descriptor of a batch, in device memory. The tensor maps are read by
// TMA from global memory. `step` counts the grid's steps; it selects the
// ping-pong state set and the phi plane roles, and it is advanced by
// batch_advance_kernel, so a captured sequence of launches stays valid while
// grids join and leave (their step counters differ).
template <typename T>
struct alignas(64) BatchGrid {
    CUtensorMap tmX[2];      // state sets 0, 1
    CUtensorMap tmPhi[3];    // phi planes
    void *X[2];
    T *phi[3];
    long long step, target;  // steps taken; the grid is frozen once step == target
    size_t plane;
    int nx, ny, pitch, tiles_x;
    int item0, nitems;       // its tiles in the work list
    int vel_kind, pad_;
    double vp[3];            // velocity parameters (FP64; rounded per precision in the kernel)
    T tl[3];                 // time levels of the current step: t, t - dt, t + dt/2
    T vc[3];                 // single vortex: cos(pi t / T) at those levels
};

// Time levels of a grid's current step and, for the single vortex, its reversal
// factors, in FP64 (FP64 is slow on this chip: evaluated once per grid and step,
// by the advance kernel and after each upload of the descriptors, never per tile).
template <typename T>
__device__ inline void batch_time_factors(BatchGrid<T> *G, double dt) {
    const double t = (double)G->step * dt;
    G->tl[0] = (T)t;
    G->tl[1] = (T)(t - dt);
    G->tl[2] = (T)(t + 0.5 * dt);
    if (G->vel_kind != VEL_VORTEX) return;
    const double Tp = G->vp[2];
    G->vc[0] = (T)cospi(t / Tp);
    G->vc[1] = (T)cospi((t - dt) / Tp);
    G->vc[2] = (T)cospi((t + 0.5 * dt) / Tp);
}

// Parameters common to every grid of a batch (same W, M, cfl, order, flux, precision).
template <typename T>
struct BatchUniform {
    T b, h, c1, c2, c3, be1, ga1, tau, theta_c, phiA, phiB, inv_dt, qscale, qinv;
    double dt;
    int dtphiu, tile_w, tile_h;
    int *status;
};

template <typename T, typename ST, int ORDER, int FLUX, int NW, int MR>
__global__ void __launch_bounds__(NW * 32, (FastTile<T, ST, NW, MR>::min_blocks))
batch_fast_kernel(const __grid_constant__ BatchUniform<T> u, const __grid_constant__ FaceCoefs<T> cf,
                  const BatchGrid<T> *__restrict__ grids, const int4 *__restrict__ items, int nitems,
                  double *__restrict__ partials) {
    constexpr bool PHIP = Store<T, ST>::phi_plane;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = fast_bar<T, ST, NW, MR>(smem);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    uint32_t phase = 0;
    int fenced = -1;   // grid whose tensor maps this CTA has acquired in this launch
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        const BatchGrid<T> *G = grids + w.x;
        const long long step = G->step;
        if (step >= G->target) continue;   // frozen grid (uniform for the CTA)
        StepParams<T> p;
        p.nx = G->nx;
        p.ny = G->ny;
        p.pitch = G->pitch;
        p.plane = G->plane;
        p.status = u.status;
        p.tiles_x = G->tiles_x;
        p.tile_w = u.tile_w;
        p.tile_h = u.tile_h;
        p.acc = nullptr;
        p.out2 = nullptr;
        p.mass_partial = nullptr;
        p.ufield = p.vfield = nullptr;
        p.a = T(1) - u.b;
        p.b = u.b;
        p.h = u.h;
        p.c1 = u.c1;
        p.c2 = u.c2;
        p.c3 = u.c3;
        p.al1 = T(1) - u.be1;
        p.be1 = u.be1;
        p.ga1 = u.ga1;
        p.al2 = p.be2 = p.ga2 = T(0);
        p.tau = u.tau;
        p.theta_c = u.theta_c;
        p.phiA = u.phiA;
        p.phiB = u.phiB;
        p.inv_dtD = u.inv_dt;
        p.useD = (u.dtphiu && step > 0) ? 1 : 0;
        p.seed = (uint32_t)step;
        p.vel_kind = G->vel_kind;
        p.vp0 = (T)G->vp[0];
        p.vp1 = (T)G->vp[1];
        p.vp2 = (T)G->vp[2];
        p.t = G->tl[0];
        p.t_old = G->tl[1];
        p.t_face = G->tl[2];
        p.qscale = u.qscale;
        p.qinv = u.qinv;
        FastExtra<T> fe;
        fe.vc_t = G->vc[0];
        fe.vc_told = G->vc[1];
        fe.vc_tface = G->vc[2];
        const int cur = (int)(step & 1);
        p.X = G->X[cur];
        p.out1 = G->X[1 - cur];
        int iPc = 0, iPo, iOut;
        if constexpr (PHIP) {   // roles rotate with period 3 (see the context API)
            iPc = (3 - (int)(step % 3)) % 3;
            iPo = (iPc + 1) % 3;
            iOut = (iPc + 2) % 3;
            p.phi_cur = G->phi[iPc];
        } else {
            iPo = cur;
            iOut = 1 - cur;
            p.phi_cur = nullptr;
        }
        p.phi_old = G->phi[iPo];
        p.phi_out = G->phi[iOut];
        if (threadIdx.x == 0 && w.x != fenced) {
            // tensor maps written to global memory by the host: order them for the TMA
            // unit (once per grid: the descriptors do not change during a launch)
            fenced = w.x;
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&G->tmX[cur]) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&G->tmPhi[iPo]) : "memory");
            if constexpr (PHIP)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&G->tmPhi[iPc]) : "memory");
        }
        if (!fast_tile<T, ST, ORDER, FLUX, NW, MR>(p, cf, fe, &G->tmX[cur], &G->tmPhi[iPo], &G->tmPhi[iPc], w.y, w.z,
                                                  partials + it, smem, bar, phase))
            return;
        phase ^= 1u;
    }
}

// After a batch step: per-grid FP64 mass (fixed-order sum of its tile partials)
// and the step counter. One CTA per grid.
template <typename T>
__global__ void __launch_bounds__(256)
batch_advance_kernel(BatchGrid<T> *grids, const double *partials, double *mass, int *status, double dt) {
    __shared__ double sred[32];
    BatchGrid<T> *G = grids + blockIdx.x;
    if (G->step >= G->target) return;   // uniform for the CTA
    double s = 0.0;
    for (int i = threadIdx.x; i < G->nitems; i += blockDim.x) s += partials[G->item0 + i];
    s = block_sum(s, sred);
    if (threadIdx.x == 0) {
        mass[blockIdx.x] = s;
        if (!isfinite(s)) atomicOr(status, 1);
        G->step = G->step + 1;
        batch_time_factors(G, dt);
    }
}

// The factors of every grid after an upload of the descriptors (one thread per grid).
template <typename T>
__global__ void __launch_bounds__(128) batch_factors_kernel(BatchGrid<T> *grids, int n, double dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) batch_time_factors(grids + i, dt);
}

}  // namespace dugks
