// dugks_internal.h -- host-side launch interface between the C ABI (dugks_api.cu)
// and the per-precision kernel instantiations (dugks_inst_*.cu).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dugks_fast.cuh"
#include "dugks_kernels.cuh"

namespace dugks {

// Tile of one CTA of the generic fused step kernel.
constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;
constexpr int STEP_THREADS = 256;

// Fast-kernel variants (warps per CTA x rows per thread): 0 = 8 x 4 (FP64: 8 x 2),
// 1 = 16 x 1, 2 = 8 x 2, 3 = 12 x 3, 4 = 8 x 3, 5 = 10 x 4. Fewer rows per thread:
// fewer registers and more resident warps, more halo overhead; taller tiles (3, 5):
// less halo per cell, fewer resident CTAs.
constexpr int FAST_VARIANTS = 6;

// Geometry of a TMA-staged (fast) variant.
struct FastGeom {
    int threads, tile_w, tile_h;   // cells written per CTA
    int box_w, box_h;              // state box (elements, rows)
    int box_wt;                    // phi box width (elements)
};

template <typename T, typename ST>
struct Launch {
    static cudaError_t step(const StepParams<T> &p, int order, int flux, int kind, cudaStream_t s);
    static cudaError_t init(const StepParams<T> &p, const T *phi0, T frac_dt, int order, cudaStream_t s);
    static cudaError_t mass_partial(const StepParams<T> &p, cudaStream_t s);
    static cudaError_t phi(const StepParams<T> &p, T *out, cudaStream_t s);
    // phi widened to double on the device (host read-out: one copy, no host conversion)
    static cudaError_t phi64(const StepParams<T> &p, double *out, cudaStream_t s);
    static FastGeom fast_geom(int variant, int order = 3, int stages = 2);
    static cudaError_t batch_step(const BatchUniform<T> &u, const FaceCoefs<T> &cf, const BatchGrid<T> *grids,
                                  const int4 *items, int nitems, double *partials, int order, int flux, int variant,
                                  int ctas, cudaStream_t s);
    static int batch_ctas_per_sm(int order, int flux, int variant);
    static cudaError_t step_fast(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe, const CUtensorMap &tmX,
                                 const CUtensorMap &tmPo, const CUtensorMap &tmPc, int order, int flux,
                                 int variant, cudaStream_t s);
    // order 4 (radius-2 stencils) on the TMA-staged path, tile 8 warps x 2 rows: the
    // two-stage step (KIND_T2) or a kernel of the three-stage step (full storage only)
    static cudaError_t step_fast4(const StepParams<T> &p, const FaceCoefs<T, 2> &cf, const FastExtra<T> &fe,
                                  const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc, int flux,
                                  int kind, cudaStream_t s);
    // one kernel of the three-stage step (kind KIND_T3A or KIND_T3B) on the TMA-staged
    // path, tile 8 warps x 2 rows (full storage only: ST == T); tmPc maps the plane of
    // phi of X where phi is a plane of its own (FP32)
    static cudaError_t step_fast3(const StepParams<T> &p, const FaceCoefs<T> &cf, const FastExtra<T> &fe,
                                  const CUtensorMap &tmX, const CUtensorMap &tmPo, const CUtensorMap &tmPc, int order,
                                  int flux, int kind, cudaStream_t s);
};

template <typename T>
cudaError_t launch_batch_advance(BatchGrid<T> *grids, int ngrids, const double *partials, double *mass, int *status,
                                 double dt, cudaStream_t s);
template <typename T>
cudaError_t launch_batch_factors(BatchGrid<T> *grids, int ngrids, double dt, cudaStream_t s);

cudaError_t launch_mass_final(const double *partial, int n, double *out, int *status, cudaStream_t s);

// One step of the streaming-collision DVM (dugks_inst_dvm.cu); lbm: the plain
// streaming of dt = 1 (T = double or float, full storage).
template <typename T>
struct DvmExtra;
template <typename T>
cudaError_t launch_dvm(const StepParams<T> &p, const DvmExtra<T> &dv, int order, bool lbm, cudaStream_t s);

// Every device allocation of the library goes through dev_malloc: cudaMalloc
// behind a host-side test hook (dugks_selftest_fail_allocs) that can make chosen
// allocations report cudaErrorMemoryAllocation without touching the device.
cudaError_t dev_malloc_raw(void **p, size_t bytes);
// The same hook in front of a stream-ordered allocation from `pool` on stream `s`
// (cudaMallocFromPoolAsync): the memory is usable in the order of `s`.
cudaError_t dev_malloc_pool(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t s);
template <typename P>
inline cudaError_t dev_malloc(P **p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

}  // namespace dugks
