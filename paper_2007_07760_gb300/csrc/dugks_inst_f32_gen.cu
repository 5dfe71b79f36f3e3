// generic fused step, initial state, mass and phi kernels of the two-stage scheme; state and arithmetic in float,
// phi a plane of its own.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<float,PhiF32>::step(const StepParams<float> &, int, int, int, cudaStream_t);
template cudaError_t Launch<float,PhiF32>::init(const StepParams<float> &, const float *, float, int, cudaStream_t);
template cudaError_t Launch<float,PhiF32>::mass_partial(const StepParams<float> &, cudaStream_t);
template cudaError_t Launch<float,PhiF32>::phi(const StepParams<float> &, float *, cudaStream_t);
template cudaError_t Launch<float,PhiF32>::phi64(const StepParams<float> &, double *, cudaStream_t);
}  // namespace dugks
