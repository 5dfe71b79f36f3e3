// dugks_internal.h -- host-side launch interface between the C ABI (dugks_api.cu)
// and the per-precision kernel instantiations (dugks_inst_*.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dugks_kernels.cuh"

namespace dugks {

// Tile of one CTA of the fused step kernel.
constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;
constexpr int STEP_THREADS = 256;

// Precision tags: 0 = FP64, 1 = FP32, 2 = FP32 arithmetic with FP16 deviation storage.
template <typename T, typename ST>
struct Launch {
    static cudaError_t step(const StepParams<T> &p, int order, int flux, int kind, cudaStream_t s);
    static cudaError_t init(const StepParams<T> &p, const T *phi0, T frac_dt, int order, cudaStream_t s);
    static cudaError_t mass_partial(const StepParams<T> &p, cudaStream_t s);
    static cudaError_t phi(const StepParams<T> &p, T *out, cudaStream_t s);
};

cudaError_t launch_mass_final(const double *partial, int n, double *out, int *status, cudaStream_t s);

}  // namespace dugks
