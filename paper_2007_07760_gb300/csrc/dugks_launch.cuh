// dugks_launch.cuh -- launchers of one precision; included once by each
// dugks_inst_*.cu so the three precisions compile in parallel.
#pragma once

#include <atomic>

#include "dugks_internal.h"

namespace dugks {

// Raises a kernel's dynamic shared-memory limit once per device (the attribute is
// per function and device); `done` is the kernel's own bit set of devices.
template <typename K>
static cudaError_t smem_attr_once(K kern, int bytes, std::atomic<uint64_t> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

template <typename T, typename ST, int ORDER, int FLUX, int KIND>
static cudaError_t launch_step_t(const StepParams<T> &p, cudaStream_t s) {
    using TL = Tile<T, ST, ORDER, FLUX, KIND, TILE_X, TILE_Y>;
    auto kern = step_kernel<T, ST, ORDER, FLUX, KIND, TILE_X, TILE_Y>;
    static std::atomic<uint64_t> configured{0};
    if (cudaError_t e = smem_attr_once(kern, (int)TL::smem_bytes, configured); e != cudaSuccess) return e;
    dim3 grid((p.nx + TILE_X - 1) / TILE_X, (p.ny + TILE_Y - 1) / TILE_Y);
    kern<<<grid, STEP_THREADS, TL::smem_bytes, s>>>(p);
    return cudaGetLastError();
}

// (each storage compiles only the schemes it serves)
template <typename T, typename ST, int ORDER, int FLUX>
static cudaError_t launch_kind(const StepParams<T> &p, int kind, cudaStream_t s) {
    if constexpr (Store<T, ST>::t2)
        if (kind == KIND_T2) return launch_step_t<T, ST, ORDER, FLUX, KIND_T2>(p, s);
    if constexpr (Store<T, ST>::t3) {
        if (kind == KIND_T3A) return launch_step_t<T, ST, ORDER, FLUX, KIND_T3A>(p, s);
        if (kind == KIND_T3B) return launch_step_t<T, ST, ORDER, FLUX, KIND_T3B>(p, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, typename ST, int ORDER>
static cudaError_t launch_flux(const StepParams<T> &p, int flux, int kind, cudaStream_t s) {
    return flux == 0 ? launch_kind<T, ST, ORDER, 0>(p, kind, s) : launch_kind<T, ST, ORDER, 1>(p, kind, s);
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::step(const StepParams<T> &p, int order, int flux, int kind, cudaStream_t s) {
    switch (order) {
    case 2: return launch_flux<T, ST, 2>(p, flux, kind, s);
    case 3: return launch_flux<T, ST, 3>(p, flux, kind, s);
    case 4: return launch_flux<T, ST, 4>(p, flux, kind, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::init(const StepParams<T> &p, const T *phi0, T frac_dt, int order, cudaStream_t s) {
    dim3 block(128), grid((p.nx + 127) / 128, p.ny);
    switch (order) {
    case 2: init_kernel<T, ST, 2><<<grid, block, 0, s>>>(p, phi0, frac_dt); break;
    case 3: init_kernel<T, ST, 3><<<grid, block, 0, s>>>(p, phi0, frac_dt); break;
    case 4: init_kernel<T, ST, 4><<<grid, block, 0, s>>>(p, phi0, frac_dt); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::mass_partial(const StepParams<T> &p, cudaStream_t s) {
    dim3 grid((p.nx + p.tile_w - 1) / p.tile_w, (p.ny + p.tile_h - 1) / p.tile_h);
    mass_partial_kernel<T, ST><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// rows of cells per thread in the fast kernel: 4 (FP32 arithmetic) or 2 (FP64)
template <typename T>
constexpr int fast_mr() { return sizeof(T) == 8 ? 2 : 4; }

template <typename T, typename ST, int NW, int MR, int R = 1>
static FastGeom geom_t() {
    using FT = FastTile<T, ST, NW, MR, R>;
    return FastGeom{FT::NT, FT::TX, FT::TY, FT::BW, FT::RH, FT::BWT};
}

// Tile of the radius-2 (orders 4 and 5) two-stage kernel: 10 warps x 3 rows in FP32
// and FP16 storage (measured in FP32 at 4096^2: 893 us against 1159 us for 8 x 2;
// at 1024^2 78 against 84 us), 8 x 2 in FP64. The three-stage kernels keep 8 x 2.
template <typename T>
constexpr int o4_nw() { return sizeof(T) == 8 ? 8 : 10; }
template <typename T>
constexpr int o4_mr() { return sizeof(T) == 8 ? 2 : 3; }

template <typename T, typename ST>
FastGeom Launch<T, ST>::fast_geom(int variant, int order, int stages) {
    if (order >= 4) {   // one tile shape per scheme for radius-2 stencils (orders 4 and 5)
        if (stages == 2) return geom_t<T, ST, o4_nw<T>(), o4_mr<T>(), 2>();
        return geom_t<T, ST, 8, 2, 2>();
    }
    switch (variant) {
    case 1: return geom_t<T, ST, 16, 1>();
    case 2: return geom_t<T, ST, 8, 2>();
    case 3: return geom_t<T, ST, 12, 3>();
    case 4: return geom_t<T, ST, 8, 3>();
    case 5: return geom_t<T, ST, 10, 4>();
    default: return geom_t<T, ST, 8, fast_mr<T>()>();
    }
}

template <typename T, typename ST, int ORDER, int FLUX, int NW, int MR>
static cudaError_t launch_fast_t(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe, const CUtensorMap &tmX,
                                 const CUtensorMap &tmPo, const CUtensorMap &tmPc, cudaStream_t s) {
    using FT = FastTile<T, ST, NW, MR>;
    auto kern = step_fast_kernel<T, ST, ORDER, FLUX, NW, MR>;
    static std::atomic<uint64_t> configured{0};
    if (cudaError_t e = smem_attr_once(kern, (int)FT::smem_bytes, configured); e != cudaSuccess) return e;
    // programmatic dependent launch: scheduled while the previous kernel drains
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nx + FT::TX - 1) / FT::TX, (p.ny + FT::TY - 1) / FT::TY);
    cfg.blockDim = dim3(FT::NT);
    cfg.dynamicSmemBytes = FT::smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p, cf, fe, tmX, tmPo, tmPc);
}

template <typename T, typename ST, int ORDER, int FLUX>
static cudaError_t launch_fast_v(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe,
                                 const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc, int variant,
                                 cudaStream_t s) {
    switch (variant) {
    case 1: return launch_fast_t<T, ST, ORDER, FLUX, 16, 1>(p, cf, fe, tmX, tmPo, tmPc, s);
    case 2: return launch_fast_t<T, ST, ORDER, FLUX, 8, 2>(p, cf, fe, tmX, tmPo, tmPc, s);
    case 3: return launch_fast_t<T, ST, ORDER, FLUX, 12, 3>(p, cf, fe, tmX, tmPo, tmPc, s);
    case 4: return launch_fast_t<T, ST, ORDER, FLUX, 8, 3>(p, cf, fe, tmX, tmPo, tmPc, s);
    case 5: return launch_fast_t<T, ST, ORDER, FLUX, 10, 4>(p, cf, fe, tmX, tmPo, tmPc, s);
    default: return launch_fast_t<T, ST, ORDER, FLUX, 8, fast_mr<T>()>(p, cf, fe, tmX, tmPo, tmPc, s);
    }
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::step_fast(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe, const CUtensorMap &tmX,
                                     const CUtensorMap &tmPo, const CUtensorMap &tmPc, int order, int flux,
                                     int variant, cudaStream_t s) {
    if (order == 2)
        return flux == 0 ? launch_fast_v<T, ST, 2, 0>(p, cf, fe, tmX, tmPo, tmPc, variant, s)
                         : launch_fast_v<T, ST, 2, 1>(p, cf, fe, tmX, tmPo, tmPc, variant, s);
    if (order == 3)
        return flux == 0 ? launch_fast_v<T, ST, 3, 0>(p, cf, fe, tmX, tmPo, tmPc, variant, s)
                         : launch_fast_v<T, ST, 3, 1>(p, cf, fe, tmX, tmPo, tmPc, variant, s);
    return cudaErrorInvalidValue;
}

template <typename T, int ORDER, int FLUX, int KIND>
static cudaError_t launch_fast3_t(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe,
                                  const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc,
                                  cudaStream_t s) {
    using FT = FastTile<T, T, 8, 2>;
    constexpr size_t smem = KIND == KIND_T3A ? FT::smem_bytes_t3a : FT::smem_bytes;
    auto kern = step_fast_kernel<T, T, ORDER, FLUX, 8, 2, KIND>;
    static std::atomic<uint64_t> configured{0};
    if (cudaError_t e = smem_attr_once(kern, (int)smem, configured); e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nx + FT::TX - 1) / FT::TX, (p.ny + FT::TY - 1) / FT::TY);
    cfg.blockDim = dim3(FT::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p, cf, fe, tmX, tmPo, tmPc);
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::step_fast3(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe,
                                      const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc,
                                      int order, int flux, int kind, cudaStream_t s) {
#define DUGKS_T3(O, F)                                                                        \
    return kind == KIND_T3A ? launch_fast3_t<T, O, F, KIND_T3A>(p, cf, fe, tmX, tmPo, tmPc, s) \
                            : launch_fast3_t<T, O, F, KIND_T3B>(p, cf, fe, tmX, tmPo, tmPc, s)
    if (kind != KIND_T3A && kind != KIND_T3B) return cudaErrorInvalidValue;
    if (order == 2) {
        if (flux == 0) DUGKS_T3(2, 0);
        DUGKS_T3(2, 1);
    }
    if (order == 3) {
        if (flux == 0) DUGKS_T3(3, 0);
        DUGKS_T3(3, 1);
    }
#undef DUGKS_T3
    return cudaErrorInvalidValue;
}

template <typename T, typename ST, int FLUX, int KIND>
static cudaError_t launch_fast4_t(const StepParams<T> &p, const FaceCoefs<T, 2> &cf, const FastExtra<T> &fe,
                                  const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc,
                                  cudaStream_t s) {
    constexpr int NW = KIND == KIND_T2 ? o4_nw<T>() : 8, MR = KIND == KIND_T2 ? o4_mr<T>() : 2;
    using FT = FastTile<T, ST, NW, MR, 2>;
    constexpr size_t smem = KIND == KIND_T3A ? FT::smem_bytes_t3a : FT::smem_bytes;
    auto kern = step_fast_kernel<T, ST, 4, FLUX, NW, MR, KIND>;
    static std::atomic<uint64_t> configured{0};
    if (cudaError_t e = smem_attr_once(kern, (int)smem, configured); e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nx + FT::TX - 1) / FT::TX, (p.ny + FT::TY - 1) / FT::TY);
    cfg.blockDim = dim3(FT::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p, cf, fe, tmX, tmPo, tmPc);
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::step_fast4(const StepParams<T> &p, const FaceCoefs<T, 2> &cf, const FastExtra<T> &fe,
                                      const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc,
                                      int flux, int kind, cudaStream_t s) {
    if constexpr (Store<T, ST>::t2)
        if (kind == KIND_T2)
            return flux == 0 ? launch_fast4_t<T, ST, 0, KIND_T2>(p, cf, fe, tmX, tmPo, tmPc, s)
                             : launch_fast4_t<T, ST, 1, KIND_T2>(p, cf, fe, tmX, tmPo, tmPc, s);
    if constexpr (Store<T, ST>::t3) {
        if (kind == KIND_T3A)
            return flux == 0 ? launch_fast4_t<T, ST, 0, KIND_T3A>(p, cf, fe, tmX, tmPo, tmPc, s)
                             : launch_fast4_t<T, ST, 1, KIND_T3A>(p, cf, fe, tmX, tmPo, tmPc, s);
        if (kind == KIND_T3B)
            return flux == 0 ? launch_fast4_t<T, ST, 0, KIND_T3B>(p, cf, fe, tmX, tmPo, tmPc, s)
                             : launch_fast4_t<T, ST, 1, KIND_T3B>(p, cf, fe, tmX, tmPo, tmPc, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::phi(const StepParams<T> &p, T *out, cudaStream_t s) {
    dim3 block(128), grid((p.nx + 127) / 128, p.ny);
    phi_kernel<T, ST><<<grid, block, 0, s>>>(p, out);
    return cudaGetLastError();
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::phi64(const StepParams<T> &p, double *out, cudaStream_t s) {
    dim3 block(128), grid((p.nx + 127) / 128, p.ny);
    phi_kernel<T, ST, double><<<grid, block, 0, s>>>(p, out);
    return cudaGetLastError();
}


template <typename T, typename ST, int ORDER, int FLUX, int NW, int MR>
static cudaError_t launch_batch_t(const BatchUniform<T> &u, const FaceCoefs<T> &cf, const BatchGrid<T> *grids,
                                  const int4 *items, int nitems, double *partials, int ctas, cudaStream_t s) {
    using FT = FastTile<T, ST, NW, MR>;
    auto kern = batch_fast_kernel<T, ST, ORDER, FLUX, NW, MR>;
    // (the shared-memory attribute was set by batch_ctas_per_sm, outside any capture)
    if (nitems <= 0) return cudaSuccess;
    kern<<<ctas < nitems ? ctas : nitems, FT::NT, FT::smem_bytes, s>>>(u, cf, grids, items, nitems, partials);
    return cudaGetLastError();
}

template <typename T, typename ST, int ORDER, int FLUX, int NW, int MR>
static int batch_occupancy_t() {
    using FT = FastTile<T, ST, NW, MR>;
    auto kern = batch_fast_kernel<T, ST, ORDER, FLUX, NW, MR>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FT::smem_bytes);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, FT::NT, FT::smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 0 ? n : 1;
}

#define DUGKS_BATCH_DISPATCH(CALL)                                                            \
    switch (variant) {                                                                        \
    case 1: return CALL(16, 1);                                                               \
    case 2: return CALL(8, 2);                                                                \
    case 3: return CALL(12, 3);                                                               \
    case 4: return CALL(8, 3);                                                                \
    case 5: return CALL(10, 4);                                                               \
    default: return CALL(8, fast_mr<T>());                                                    \
    }

template <typename T, typename ST, int ORDER, int FLUX>
static cudaError_t launch_batch_v(const BatchUniform<T> &u, const FaceCoefs<T> &cf, const BatchGrid<T> *grids,
                                  const int4 *items, int nitems, double *partials, int variant, int ctas,
                                  cudaStream_t s) {
#define CALL(NW, MR) launch_batch_t<T, ST, ORDER, FLUX, NW, MR>(u, cf, grids, items, nitems, partials, ctas, s)
    DUGKS_BATCH_DISPATCH(CALL)
#undef CALL
}

template <typename T, typename ST, int ORDER, int FLUX>
static int batch_occ_v(int variant) {
#define CALL(NW, MR) batch_occupancy_t<T, ST, ORDER, FLUX, NW, MR>()
    DUGKS_BATCH_DISPATCH(CALL)
#undef CALL
}

template <typename T, typename ST>
cudaError_t Launch<T, ST>::batch_step(const BatchUniform<T> &u, const FaceCoefs<T> &cf, const BatchGrid<T> *grids,
                                      const int4 *items, int nitems, double *partials, int order, int flux,
                                      int variant, int ctas, cudaStream_t s) {
    switch (order * 2 + flux) {
    case 4: return launch_batch_v<T, ST, 2, 0>(u, cf, grids, items, nitems, partials, variant, ctas, s);
    case 5: return launch_batch_v<T, ST, 2, 1>(u, cf, grids, items, nitems, partials, variant, ctas, s);
    case 6: return launch_batch_v<T, ST, 3, 0>(u, cf, grids, items, nitems, partials, variant, ctas, s);
    case 7: return launch_batch_v<T, ST, 3, 1>(u, cf, grids, items, nitems, partials, variant, ctas, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, typename ST>
int Launch<T, ST>::batch_ctas_per_sm(int order, int flux, int variant) {
    switch (order * 2 + flux) {
    case 4: return batch_occ_v<T, ST, 2, 0>(variant);
    case 5: return batch_occ_v<T, ST, 2, 1>(variant);
    case 6: return batch_occ_v<T, ST, 3, 0>(variant);
    case 7: return batch_occ_v<T, ST, 3, 1>(variant);
    default: return 1;
    }
}

template <typename T>
cudaError_t launch_batch_advance(BatchGrid<T> *grids, int ngrids, const double *partials, double *mass, int *status,
                                 double dt, cudaStream_t s) {
    if (ngrids <= 0) return cudaSuccess;
    batch_advance_kernel<T><<<ngrids, 256, 0, s>>>(grids, partials, mass, status, dt);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_factors(BatchGrid<T> *grids, int ngrids, double dt, cudaStream_t s) {
    if (ngrids <= 0) return cudaSuccess;
    batch_factors_kernel<T><<<(ngrids + 127) / 128, 128, 0, s>>>(grids, ngrids, dt);
    return cudaGetLastError();
}

}  // namespace dugks
