// TMA-staged single-grid step kernels; FP32 arithmetic, distribution stored as half-precision deviations from w_k phi.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template FastGeom Launch<float,__half>::fast_geom(int, int, int);
template cudaError_t Launch<float,__half>::step_fast(const StepParams<float> &, const FaceCoefs<float> &, const FastExtra<float> &, const CUtensorMap &, const CUtensorMap &, const CUtensorMap &, int, int, int, cudaStream_t);
}  // namespace dugks
