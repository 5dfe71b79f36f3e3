// generic fused step, initial state, mass and phi kernels; FP32 arithmetic, distribution stored as half-precision deviations from w_k phi.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<float,__half>::step(const StepParams<float> &, int, int, int, cudaStream_t);
template cudaError_t Launch<float,__half>::init(const StepParams<float> &, const float *, float, int, cudaStream_t);
template cudaError_t Launch<float,__half>::mass_partial(const StepParams<float> &, cudaStream_t);
template cudaError_t Launch<float,__half>::phi(const StepParams<float> &, float *, cudaStream_t);
template cudaError_t Launch<float,__half>::phi64(const StepParams<float> &, double *, cudaStream_t);
}  // namespace dugks
