// TMA-staged kernels for order 4 (radius-2 stencils); state float, arithmetic float.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<float,float>::step_fast4(const StepParams<float> &, const FaceCoefs<float, 2> &, const FastExtra<float> &, const CUtensorMap &, const CUtensorMap &, const CUtensorMap &, int, int, cudaStream_t);
}  // namespace dugks
