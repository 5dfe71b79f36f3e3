// TMA-staged kernels for order 4 (radius-2 stencils); state double, arithmetic double.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<double,double>::step_fast4(const StepParams<double> &, const FaceCoefs<double, 2> &, const FastExtra<double> &, const CUtensorMap &, const CUtensorMap &, const CUtensorMap &, int, int, cudaStream_t);
}  // namespace dugks
