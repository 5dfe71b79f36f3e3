// generic fused step, initial state, mass and phi kernels; state and arithmetic in double.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<double,double>::step(const StepParams<double> &, int, int, int, cudaStream_t);
template cudaError_t Launch<double,double>::init(const StepParams<double> &, const double *, double, int, cudaStream_t);
template cudaError_t Launch<double,double>::mass_partial(const StepParams<double> &, cudaStream_t);
template cudaError_t Launch<double,double>::phi(const StepParams<double> &, double *, cudaStream_t);
template cudaError_t Launch<double,double>::phi64(const StepParams<double> &, double *, cudaStream_t);
}  // namespace dugks
