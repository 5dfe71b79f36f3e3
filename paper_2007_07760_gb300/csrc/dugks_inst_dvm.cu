// Streaming-collision DVM / LBM step kernels (dugks_dvm.cuh), FP64 and FP32.
// (One translation unit per kernel family, so they compile in parallel.)
#include <atomic>

#include "dugks_dvm.cuh"
#include "dugks_internal.h"

namespace dugks {

namespace {

template <typename T, int ORDER, bool LBM>
cudaError_t launch_dvm_t(const StepParams<T> &p, const DvmExtra<T> &dv, cudaStream_t s) {
    using DT = DvmTile<T, ORDER, LBM>;
    auto kern = dvm_step_kernel<T, ORDER, LBM>;
    // the dynamic shared-memory limit is a per-function, per-device attribute
    static std::atomic<uint64_t> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (!bit || !(configured.load(std::memory_order_relaxed) & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DT::smem_bytes);
        if (e != cudaSuccess) return e;
        if (bit) configured.fetch_or(bit, std::memory_order_relaxed);
    }
    const dim3 grid((p.nx + DT::TX - 1) / DT::TX, (p.ny + DT::TY - 1) / DT::TY);
    kern<<<grid, DT::NT, DT::smem_bytes, s>>>(p, dv);
    return cudaGetLastError();
}

template <typename T, bool LBM>
cudaError_t launch_dvm_o(const StepParams<T> &p, const DvmExtra<T> &dv, int order, cudaStream_t s) {
    switch (order) {
    case 2: return launch_dvm_t<T, 2, LBM>(p, dv, s);
    case 3: return launch_dvm_t<T, 3, LBM>(p, dv, s);
    case 4: return launch_dvm_t<T, 4, LBM>(p, dv, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_dvm(const StepParams<T> &p, const DvmExtra<T> &dv, int order, bool lbm, cudaStream_t s) {
    return lbm ? launch_dvm_o<T, true>(p, dv, order, s) : launch_dvm_o<T, false>(p, dv, order, s);
}
template cudaError_t launch_dvm<double>(const StepParams<double> &, const DvmExtra<double> &, int, bool, cudaStream_t);
template cudaError_t launch_dvm<float>(const StepParams<float> &, const DvmExtra<float> &, int, bool, cudaStream_t);

}  // namespace dugks
