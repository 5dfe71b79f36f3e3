// TMA-staged kernels of the three-stage step; state and arithmetic in double.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<double,double>::step_fast3(const StepParams<double> &, const FaceCoefs<double> &, const FastExtra<double> &, const CUtensorMap &, const CUtensorMap &, const CUtensorMap &, int, int, int, cudaStream_t);
}  // namespace dugks
