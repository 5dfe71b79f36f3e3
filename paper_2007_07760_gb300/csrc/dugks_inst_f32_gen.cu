// generic fused step, initial state, mass and phi kernels; state and arithmetic in float.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<float,float>::step(const StepParams<float> &, int, int, int, cudaStream_t);
template cudaError_t Launch<float,float>::init(const StepParams<float> &, const float *, float, int, cudaStream_t);
template cudaError_t Launch<float,float>::mass_partial(const StepParams<float> &, cudaStream_t);
template cudaError_t Launch<float,float>::phi(const StepParams<float> &, float *, cudaStream_t);
template cudaError_t Launch<float,float>::phi64(const StepParams<float> &, double *, cudaStream_t);
}  // namespace dugks
