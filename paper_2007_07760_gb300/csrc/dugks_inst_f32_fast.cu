// TMA-staged single-grid step kernels; state and arithmetic in float.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template FastGeom Launch<float,float>::fast_geom(int, int, int);
template cudaError_t Launch<float,float>::step_fast(const StepParams<float> &, const FaceCoefs<float> &, const FastExtra<float> &, const CUtensorMap &, const CUtensorMap &, const CUtensorMap &, int, int, int, cudaStream_t);
}  // namespace dugks
